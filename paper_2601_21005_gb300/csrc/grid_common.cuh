// Device helpers shared by the grid kernels (plane path and row path).
#pragma once
#include <cuda_runtime.h>

namespace sgw {

__device__ __forceinline__ int sfreq(int i, int n) { return i < n / 2 ? i : i - n; }

__device__ __forceinline__ float4 ld4(const float2* p) { return __ldg(reinterpret_cast<const float4*>(p)); }

// Bulk prefetch of `bytes` (multiple of 16) at a 16-byte aligned global address into L2; no data
// reaches the SM, the later loads of the same lines hit L2.
__device__ __forceinline__ void l2_prefetch(const void* p, unsigned bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}
__device__ __forceinline__ void st4(float2* p, float2 a, float2 b) {
    *reinterpret_cast<float4*>(p) = make_float4(a.x, a.y, b.x, b.y);
}
// Streaming forms (data read or written once per launch): the lines are cached evict-first, so
// they displace neither the operands prefetched into L2 for later blocks nor the data shared by
// the vectors of one unit.
__device__ __forceinline__ float4 ldcs4(const float2* p) { return __ldcs(reinterpret_cast<const float4*>(p)); }
__device__ __forceinline__ void stcs4(float2* p, float2 a, float2 b) {
    __stcs(reinterpret_cast<float4*>(p), make_float4(a.x, a.y, b.x, b.y));
}

// Sum 8 per-lane values over a warp by halving exchanges at lane distances 16, 8, 4 (each lane keeps
// the half selected by its lane bit and adds its partner's copy of that half), then a plain
// reduction over distances 2 and 1; returns the total of value 4 bit4 + 2 bit3 + bit2 of the lane.
__device__ __forceinline__ float warp_reduce_scatter8(const float (&v)[8], int lane) {
    float a4[4], a2[2];
    const bool h4 = (lane >> 4) & 1;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const float keep = h4 ? v[4 + i] : v[i], give = h4 ? v[i] : v[4 + i];
        a4[i] = keep + __shfl_xor_sync(0xffffffffu, give, 16);
    }
    const bool h3 = (lane >> 3) & 1;
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const float keep = h3 ? a4[2 + i] : a4[i], give = h3 ? a4[i] : a4[2 + i];
        a2[i] = keep + __shfl_xor_sync(0xffffffffu, give, 8);
    }
    const bool h2 = (lane >> 2) & 1;
    const float keep = h2 ? a2[1] : a2[0], give = h2 ? a2[0] : a2[1];
    float t = keep + __shfl_xor_sync(0xffffffffu, give, 4);
    t += __shfl_xor_sync(0xffffffffu, t, 2);
    t += __shfl_xor_sync(0xffffffffu, t, 1);
    return t;
}

// k-space factor of grid point (kx, ky, kz) of an N^3 transform, divided by N^3 (the inverse's
// normalisation): KIND 0 kinetic |k|^2/2 (capped at ecut if ecut > 0), KIND 1 Coulomb 4 pi/|k|^2
// (0 at k = 0)
template <int N, int KIND>
__device__ __forceinline__ float kspace_factor(int kx, int ky, int kz, float kscale, float ecut) {
    const int mx = sfreq(kx, N), my = sfreq(ky, N), mz = sfreq(kz, N);
    const float k2 = kscale * (float)(mx * mx + my * my + mz * mz);
    float f;
    if (KIND == 0) {
        f = 0.5f * k2;
        if (ecut > 0.f) f = fminf(f, ecut);
    } else {
        f = k2 > 0.f ? 12.566370614359172f / k2 : 0.f;   // 4 pi / k^2
    }
    return f * (1.0f / ((float)N * N * N));
}

}  // namespace sgw
