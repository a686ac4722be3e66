// A 288-point complex FFT of one line held by one warp (no shared-memory stages, no barriers).
//
// 288 = 32 x 9 (Cooley-Tukey): X[k2 + 9 k1] = sum_n1 W32^(n1 k1) W288^(n1 k2) sum_n2 x[n1 + 32 n2] W9^(n2 k2).
// Each lane holds the 9 points of one n1, does the 9-point DFT (3 x 3) in registers, multiplies by
// W288^(n1 k2), and the 32-point DFTs over n1 run across the lanes as five radix-2
// decimation-in-time stages with shuffle partners (bit-reversed input, natural output).
//
// Lane relabelling: physical lane p acts as logical lane L = p ^ ((p & 1) << 4).  Logical lane L
// holds input n1 = bitrev5(L) and ends with output k1 = L.  With it every half-warp covers 16
// different n1 and 16 different k1 modulo 16, so both the loads (rows x = n1 + 32 n2, stride 1) and
// the stores (x = k2 + 9 k1, stride 9) hit 16 distinct bank pairs; logical partner L ^ m is
// physical p ^ m for m > 1 and p ^ 17 for m = 1.
//
// Twiddles come from the table tws[m] = exp(-2 pi i m / 288) (m < 288) in shared memory.
#pragma once
#include "fft_smem.cuh"

namespace sgw {

__device__ __forceinline__ int wfft_logical_lane(int p) { return p ^ ((p & 1) << 4); }
// the input index n1 of physical lane p: the line's points n1 + 32 n2, n2 = 0..8, go to v[n2]
__device__ __forceinline__ int wfft_n1(int p) { return (int)(__brev((unsigned)wfft_logical_lane(p)) >> 27); }
// the output index k1 of physical lane p: on return v[k2] = X[k2 + 9 k1]
__device__ __forceinline__ int wfft_k1(int p) { return wfft_logical_lane(p); }

// exp(DIR 2 pi i m / 288) from the table of exp(-2 pi i m / 288)
template <int DIR>
__device__ __forceinline__ float2 wfft_tw(const float2* tws, int m) {
    float2 w = tws[m];
    if (DIR > 0) w.y = -w.y;
    return w;
}

// 9-point DFT of v in place, as 3 x 3: n = c + 3 d, k = a + 3 b
template <int DIR>
__device__ __forceinline__ void wfft_dft9(float2 (&v)[9], const float2* tws) {
    float2 t[3][3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        t[c][0] = v[c];
        t[c][1] = v[c + 3];
        t[c][2] = v[c + 6];
        Dft<3, DIR>::run(t[c]);
    }
    // W9^(c a) = W288^(32 c a)
    t[1][1] = cmul(t[1][1], wfft_tw<DIR>(tws, 32));
    t[1][2] = cmul(t[1][2], wfft_tw<DIR>(tws, 64));
    t[2][1] = cmul(t[2][1], wfft_tw<DIR>(tws, 64));
    t[2][2] = cmul(t[2][2], wfft_tw<DIR>(tws, 128));
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        float2 s[3] = {t[0][a], t[1][a], t[2][a]};
        Dft<3, DIR>::run(s);
        v[a] = s[0];
        v[a + 3] = s[1];
        v[a + 6] = s[2];
    }
}

// v[n2] = x[wfft_n1(lane) + 32 n2] on entry; v[k2] = X[k2 + 9 wfft_k1(lane)] on return, X the
// unnormalised DFT with exp(DIR 2 pi i n k / 288).  All 32 lanes must call it together.
template <int DIR>
__device__ __forceinline__ void warp_fft288(float2 (&v)[9], int lane, const float2* tws) {
    const int L = wfft_logical_lane(lane);
    const int n1 = wfft_n1(lane);
    wfft_dft9<DIR>(v, tws);
#pragma unroll
    for (int k = 1; k < 9; ++k) v[k] = cmul(v[k], wfft_tw<DIR>(tws, n1 * k));
#pragma unroll
    for (int m = 1; m < 32; m <<= 1) {
        const bool hi = (L & m) != 0;
        const float2 w = wfft_tw<DIR>(tws, (L & (m - 1)) * (144 / m));
        const int sx = m == 1 ? 17 : m;
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            const float2 u = hi ? cmul(v[k], w) : v[k];
            float2 p;
            p.x = __shfl_xor_sync(0xffffffffu, u.x, sx);
            p.y = __shfl_xor_sync(0xffffffffu, u.y, sx);
            v[k] = hi ? csub(p, u) : cadd(u, p);
        }
    }
}

}  // namespace sgw
