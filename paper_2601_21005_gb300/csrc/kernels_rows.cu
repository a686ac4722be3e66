// Grid kernels of the row path: grids whose side is not a power of two (n = 2^a 3^b: 48, 96 and
// 288 here), in particular those whose xy plane does not fit one CTA's shared memory (a 288^2
// complex plane is 663 KB against 227 KB per CTA).  The passes of the plane path, with the 2D plane
// transform split into a transform along x of units of RR consecutive rows (one CTA per unit) and a
// transform along y of tiles of LT x-columns:
//   H b = [z lines: FFT z, * T(k)/n^3, inverse FFT z] -> [y lines: inverse FFT y] ->
//         [rows: inverse FFT x, + V b + V_NL b, Chebyshev combine, write, per-slot KB partials,
//          FFT x] -> [y lines: FFT y]
// i.e. four HBM passes per Chebyshev term instead of two (Sec. 2.2: the cost of each H application
// is dominated by the FFTs; the potential multiply and the KB apply are fused into the row pass).
// The KB tables are those of the plane path built per unit instead of per plane (see KBDev).
#include "fft_smem.cuh"
#include "grid_common.cuh"
#include "kb_unit.cuh"
#include "sgw_internal.cuh"

namespace sgw {

constexpr int RR = 8;      // x rows per unit of the row kernels
constexpr int RNT = 256;   // threads of the row and line kernels
constexpr int LT = 16;     // x columns per y- or z-line tile (16 x 8 B = 128 B rows)

bool rows_path(int n) { return n == 48 || n == 96 || n == 288; }
// KB unit: an xy plane on the plane path, RR x rows on the row path, a CTA's rows of a plane when a
// cluster of CTAs holds the plane (288)
int64_t unit_points(int n) {
    if (cluster_plane(n)) return (int64_t)cluster_unit_rows() * n;
    return rows_path(n) ? (int64_t)RR * n : (int64_t)n * n;
}

// ------------------------------------------------------------------ units of rows <-> smem
// A unit is RR consecutive x rows (RR N points, contiguous in memory); in shared memory row y of
// the unit starts at y (N + 1).
template <int N>
__device__ __forceinline__ void load_rows(float2* sm, const float2* __restrict__ src) {
    constexpr int P = N + 1;
    for (int q = threadIdx.x; q < RR * N / 2; q += RNT) {
        const int y = q / (N / 2), x = 2 * (q % (N / 2));
        const float4 v = ld4(src + y * N + x);
        sm[y * P + x] = make_float2(v.x, v.y);
        sm[y * P + x + 1] = make_float2(v.z, v.w);
    }
}

template <int N>
__device__ __forceinline__ void store_rows(float2* __restrict__ dst, const float2* sm) {
    constexpr int P = N + 1;
    for (int q = threadIdx.x; q < RR * N / 2; q += RNT) {
        const int y = q / (N / 2), x = 2 * (q % (N / 2));
        st4(dst + y * N + x, sm[y * P + x], sm[y * P + x + 1]);
    }
}

template <int N>
__device__ __forceinline__ TwShared stage_twiddles(float2* stw, const float2* __restrict__ tw) {
    for (int i = threadIdx.x; i < N; i += RNT) stw[i] = __ldg(tw + i);
    return TwShared{stw};
}

// ------------------------------------------------------------------ forward transform along x
template <int N>
__global__ void __launch_bounds__(RNT) k_rows_fwd(const float2* __restrict__ in, float2* __restrict__ W,
                                                  const float2* __restrict__ tw) {
    extern __shared__ float2 sm[];
    constexpr int P = N + 1;
    const TwShared tws = stage_twiddles<N>(sm + RR * P, tw);
    const size_t off = ((size_t)blockIdx.y * (N * N / RR) + blockIdx.x) * RR * N;
    load_rows<N>(sm, in + off);
    __syncthreads();
    fft_lines<N, RR, P, 1, RNT, -1>(sm, tws);
    store_rows<N>(W + off, sm);
}

// ------------------------------------------------------------------ transforms along y, in place
// One CTA per (LT x-columns, z) of a vector: the tile [y][LT] is loaded with 128-byte rows,
// transformed along y in shared memory (consecutive threads on consecutive columns) and stored.
template <int N, int DIR>
__global__ void __launch_bounds__(RNT) k_ylines(float2* __restrict__ W, const float2* __restrict__ tw) {
    extern __shared__ float2 sm[];
    const TwShared tws = stage_twiddles<N>(sm + N * LT, tw);
    const int xt = blockIdx.x % (N / LT), z = blockIdx.x / (N / LT);
    float2* base = W + (size_t)blockIdx.y * N * N * N + (size_t)z * N * N + xt * LT;
    for (int q = threadIdx.x; q < N * LT / 2; q += RNT) {
        const int y = q / (LT / 2), x = 2 * (q % (LT / 2));
        const float4 v = ld4(base + (size_t)y * N + x);
        sm[y * LT + x] = make_float2(v.x, v.y);
        sm[y * LT + x + 1] = make_float2(v.z, v.w);
    }
    __syncthreads();
    fft_lines<N, LT, 1, LT, RNT, DIR>(sm, tws);
    for (int q = threadIdx.x; q < N * LT / 2; q += RNT) {
        const int y = q / (LT / 2), x = 2 * (q % (LT / 2));
        st4(base + (size_t)y * N + x, sm[y * LT + x], sm[y * LT + x + 1]);
    }
}

// ------------------------------------------------------------------ z lines
// One CTA per (LT kx-columns, ky) of a vector whose planes are xy-transformed: FFT along z, the
// diagonal k-space factor (KIND 0 kinetic, 1 Coulomb; / n^3), inverse FFT along z, in place.
template <int N>
__device__ __forceinline__ void zlines_load_fwd(const float2* __restrict__ base, float2* sm, TwShared tws) {
    for (int q = threadIdx.x; q < N * LT / 2; q += RNT) {
        const int z = q / (LT / 2), x = 2 * (q % (LT / 2));
        const float4 v = ld4(base + (size_t)z * N * N + x);
        sm[z * LT + x] = make_float2(v.x, v.y);
        sm[z * LT + x + 1] = make_float2(v.z, v.w);
    }
    __syncthreads();
    fft_lines<N, LT, 1, LT, RNT, -1>(sm, tws);
}

// Compiled for 3 resident CTAs per SM (80 registers): at 288 the pass is latency-bound, and the
// third CTA made it 31% faster than the unconstrained 93-register build.
template <int N, int KIND>
__global__ void __launch_bounds__(RNT, 3) k_zlines(float2* __restrict__ W, float kscale, float ecut,
                                                const float2* __restrict__ tw) {
    extern __shared__ float2 sm[];
    const TwShared tws = stage_twiddles<N>(sm + N * LT, tw);
    const int xt = blockIdx.x % (N / LT), ky = blockIdx.x / (N / LT);
    float2* base = W + (size_t)blockIdx.y * N * N * N + (size_t)ky * N + xt * LT;
    zlines_load_fwd<N>(base, sm, tws);
    for (int q = threadIdx.x; q < N * LT; q += RNT) {
        const int kz = q / LT, l = q % LT;
        sm[q] = cscale(sm[q], kspace_factor<N, KIND>(xt * LT + l, ky, kz, kscale, ecut));
    }
    __syncthreads();
    fft_lines<N, LT, 1, LT, RNT, +1>(sm, tws);
    for (int q = threadIdx.x; q < N * LT / 2; q += RNT) {
        const int z = q / (LT / 2), x = 2 * (q % (LT / 2));
        st4(base + (size_t)z * N * N + x, sm[z * LT + x], sm[z * LT + x + 1]);
    }
}

// Coulomb energy partial of a tile after the z transform: part[b][block] = sum_k 4 pi/k^2 |F(k)|^2
// (FP64, fixed order: per-thread sums, warp shuffles, then the warps in order).
template <int N>
__global__ void __launch_bounds__(RNT) k_zlines_energy(const float2* __restrict__ W, float kscale,
                                                       const float2* __restrict__ tw, double* __restrict__ part) {
    extern __shared__ float2 sm[];
    __shared__ double red[RNT / 32];
    const TwShared tws = stage_twiddles<N>(sm + N * LT, tw);
    const int xt = blockIdx.x % (N / LT), ky = blockIdx.x / (N / LT);
    const float2* base = W + (size_t)blockIdx.y * N * N * N + (size_t)ky * N + xt * LT;
    zlines_load_fwd<N>(base, sm, tws);
    const int my = sfreq(ky, N);
    double s = 0.0;
    for (int q = threadIdx.x; q < N * LT; q += RNT) {
        const int kz = q / LT, l = q % LT;
        const int mx = sfreq(xt * LT + l, N), mz = sfreq(kz, N);
        const double k2 = (double)kscale * (double)(mx * mx + my * my + mz * mz);
        if (k2 > 0.0) s += 12.566370614359172 / k2 * ((double)sm[q].x * sm[q].x + (double)sm[q].y * sm[q].y);
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        double t = threadIdx.x < RNT / 32 ? red[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (threadIdx.x == 0) part[(size_t)blockIdx.y * gridDim.x + blockIdx.x] = t;
    }
}

// ------------------------------------------------------------------ inverse transform along x
// After the inverse y lines: mode 0 -> out_c = the unit's points; mode 1 (Poisson of TDH densities)
// -> vtot = vloc + Re, dv = Im, uR = Im (if uR); mode 2 -> out_re = Re.
template <int N>
__global__ void __launch_bounds__(RNT) k_rows_inv(const float2* __restrict__ W, const float2* __restrict__ tw,
                                                  int mode, float2* out_c, const float* __restrict__ vloc,
                                                  float* vtot, float* dv, float* uR, int64_t uR_stride,
                                                  float* out_re) {
    extern __shared__ float2 sm[];
    constexpr int P = N + 1;
    constexpr size_t NG = (size_t)N * N * N;
    const TwShared tws = stage_twiddles<N>(sm + RR * P, tw);
    const int b = blockIdx.y;
    const size_t uoff = (size_t)blockIdx.x * RR * N;
    load_rows<N>(sm, W + (size_t)b * NG + uoff);
    __syncthreads();
    fft_lines<N, RR, P, 1, RNT, +1>(sm, tws);
    if (mode == 0) {
        store_rows<N>(out_c + (size_t)b * NG + uoff, sm);
        return;
    }
    for (int q = threadIdx.x; q < RR * N; q += RNT) {
        const size_t g = uoff + q;
        const float2 c = sm[(q / N) * P + (q % N)];
        if (mode == 1) {
            vtot[(size_t)b * NG + g] = __ldg(vloc + g) + c.x;
            dv[(size_t)b * NG + g] = c.y;
            if (uR != nullptr) uR[(size_t)b * uR_stride + g] = c.y;
        } else {
            out_re[(size_t)b * NG + g] = c.x;
        }
    }
}

// ------------------------------------------------------------------ TDH density
// Sample s owns batch vectors [s 2 n_eta, (s+1) 2 n_eta): eta_l then d eta_l.  The unit's
// (rho - rho0) + i d rho, transformed along x, goes to Wp (the y lines follow).
template <int N>
__global__ void __launch_bounds__(RNT) k_rows_density(const float2* __restrict__ psi, int n_eta, float weight,
                                                      float* rho0, int store_rho0, float2* __restrict__ Wp,
                                                      const float2* __restrict__ tw) {
    extern __shared__ float2 sm[];
    constexpr int P = N + 1;
    constexpr size_t NG = (size_t)N * N * N;
    const TwShared tws = stage_twiddles<N>(sm + RR * P, tw);
    const int s = blockIdx.y;
    const size_t uoff = (size_t)blockIdx.x * RR * N;
    for (int q = threadIdx.x; q < RR * N / 2; q += RNT) {
        const int y = q / (N / 2), x = 2 * (q % (N / 2));
        const size_t g = uoff + y * N + x;
        float r0 = 0.f, r1 = 0.f, d0 = 0.f, d1 = 0.f;
        for (int l = 0; l < n_eta; ++l) {
            const float4 e = ld4(psi + ((size_t)s * 2 * n_eta + l) * NG + g);
            const float4 de = ld4(psi + ((size_t)s * 2 * n_eta + n_eta + l) * NG + g);
            r0 += e.x * e.x + e.y * e.y;
            r1 += e.z * e.z + e.w * e.w;
            d0 += 2.f * (e.x * de.x + e.y * de.y);
            d1 += 2.f * (e.z * de.z + e.w * de.w);
        }
        r0 *= weight; r1 *= weight; d0 *= weight; d1 *= weight;
        float* rz = rho0 + (size_t)s * NG + g;
        if (store_rho0) {
            rz[0] = r0;
            rz[1] = r1;
        }
        const float q0 = store_rho0 ? r0 : rz[0], q1 = store_rho0 ? r1 : rz[1];
        sm[y * P + x] = make_float2(r0 - q0, d0);
        sm[y * P + x + 1] = make_float2(r1 - q1, d1);
    }
    __syncthreads();
    fft_lines<N, RR, P, 1, RNT, -1>(sm, tws);
    store_rows<N>(Wp + (size_t)s * NG + uoff, sm);
}

// ------------------------------------------------------------------ fused Chebyshev step
// The row-path form of the plane path's fused step on unit u of vector b (after the inverse y
// lines): inverse x transform of W -> KB apply colour by colour (unit tables, projections staged
// in shared memory) -> + (V - Ebar) b1 (+ dv b1_partner for tangents) -> combine with psi and b2 ->
// write out -> per-slot partial projections of out -> forward x transform -> Wout.
template <int N>
__global__ void __launch_bounds__(RNT) k_rows_step(StepArgs a, const float2* __restrict__ tw) {
    extern __shared__ float2 sm[];
    constexpr int P = N + 1;
    constexpr size_t NG = (size_t)N * N * N;
    float2* kcs = sm + RR * P + N;
    const TwShared tws = stage_twiddles<N>(sm + RR * P, tw);
    const int u = blockIdx.x, b = blockIdx.y;
    const size_t uoff = (size_t)u * RR * N;
    const size_t off = (size_t)b * NG + uoff;
    const VecInfo inf = a.info[b];
    const float2* kc = a.kbc != nullptr ? a.kbc + (size_t)b * a.n_proj : nullptr;
    if (kc != nullptr) kb_stage_coeffs<RNT>(a, kc, u, kcs);
    load_rows<N>(sm, a.W + off);
    __syncthreads();
    fft_lines<N, RR, P, 1, RNT, +1>(sm, tws);
    if (kc != nullptr) kb_apply_unit<N, P, RNT>(a, u, kcs, sm);
    step_pointwise<N, RR, P, RNT>(a, inf, off, uoff, sm);
    if (a.Wout == nullptr) return;
    __syncthreads();
    if (a.kbp != nullptr) kb_project_unit<N, P, RNT>(a, u, b, sm);
    fft_lines<N, RR, P, 1, RNT, -1>(sm, tws);
    store_rows<N>(a.Wout + off, sm);
}

// ------------------------------------------------------------------ launchers
#define SGW_DISPATCH_ROWS(n, ...)                                \
    switch (n) {                                                 \
        case 48: { constexpr int N = 48; __VA_ARGS__; } break;   \
        case 96: { constexpr int N = 96; __VA_ARGS__; } break;   \
        case 288: { constexpr int N = 288; __VA_ARGS__; } break; \
        default: break;                                          \
    }

static size_t rows_smem(int n) { return sizeof(float2) * ((size_t)RR * (n + 1) + n); }
static size_t lines_smem(int n) { return sizeof(float2) * ((size_t)n * LT + n); }
size_t rows_step_smem(int n, int max_unit_slots) {
    if (cluster_plane(n)) return cplane_smem(max_unit_slots);
    return rows_smem(n) + sizeof(float2) * 4 * (size_t)max_unit_slots;
}
int rows_units(int n) { return n * n / RR; }

template <int N> static cudaError_t rows_attrs(int slots) {
    cudaError_t e = cudaSuccess;
    const int mx = (int)cudaSharedmemCarveoutMaxShared;
    if ((e = cudaFuncSetAttribute(k_rows_step<N>, cudaFuncAttributePreferredSharedMemoryCarveout, mx))) return e;
    if ((e = cudaFuncSetAttribute(k_rows_step<N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)rows_step_smem(N, slots))))
        return e;
    if ((e = cudaFuncSetAttribute(k_zlines<N, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lines_smem(N))))
        return e;
    if ((e = cudaFuncSetAttribute(k_zlines<N, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lines_smem(N))))
        return e;
    if ((e = cudaFuncSetAttribute(k_zlines_energy<N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)lines_smem(N))))
        return e;
    if ((e = cudaFuncSetAttribute(k_ylines<N, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lines_smem(N))))
        return e;
    return cudaFuncSetAttribute(k_ylines<N, -1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lines_smem(N));
}

cudaError_t rows_init_attributes(int n) {
    cudaError_t e = cudaErrorInvalidValue;
    SGW_DISPATCH_ROWS(n, e = rows_attrs<N>(0));
    if (e == cudaSuccess && cluster_plane(n)) e = cluster_init_attributes(0);
    return e;
}

cudaError_t rows_step_reserve_smem(int n, int max_unit_slots) {
    if (cluster_plane(n)) return cluster_init_attributes(max_unit_slots);
    cudaError_t e = cudaErrorInvalidValue;
    SGW_DISPATCH_ROWS(n, e = cudaFuncSetAttribute(k_rows_step<N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                  (int)rows_step_smem(N, max_unit_slots)));
    return e;
}

int rows_step_blocks_per_sm(int n, int variant, int max_unit_slots) {
    if (cluster_plane(n)) return cplane_blocks_per_sm(variant, max_unit_slots);
    int r = 0;
    SGW_DISPATCH_ROWS(n, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&r, k_rows_step<N>, RNT,
                                                                       rows_step_smem(N, max_unit_slots)));
    return r;
}

int zlines_blocks_per_sm(int n) {
    if (cluster_plane(n)) return zlines_reg_blocks_per_sm(0);
    int r = 0;
    SGW_DISPATCH_ROWS(n, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&r, k_zlines<N, 0>, RNT, lines_smem(N)));
    return r;
}

static void ylines(int n, float2* W, int batch, int dir, const float2* tw, cudaStream_t st) {
    SGW_DISPATCH_ROWS(n, {
        const dim3 grid((N / LT) * N, batch);
        if (dir > 0)
            k_ylines<N, 1><<<grid, RNT, lines_smem(N), st>>>(W, tw);
        else
            k_ylines<N, -1><<<grid, RNT, lines_smem(N), st>>>(W, tw);
    });
}

void rows_plane_fwd(int n, const float2* in, float2* W, int batch, const float2* tw, cudaStream_t st) {
    if (batch == 0) return;
    SGW_DISPATCH_ROWS(n, k_rows_fwd<N><<<dim3(N * N / RR, batch), RNT, rows_smem(N), st>>>(in, W, tw));
    ylines(n, W, batch, -1, tw, st);
}

void rows_pencil(int n, float2* W, int batch, int kind, float kscale, float ecut, const float2* tw, cudaStream_t st,
                 int line_form) {
    if (batch == 0) return;
    if (cluster_plane(n)) return zlines_reg(W, batch, kind, line_form, kscale, ecut, tw, st);
    SGW_DISPATCH_ROWS(n, {
        const dim3 grid((N / LT) * N, batch);
        if (kind == 0)
            k_zlines<N, 0><<<grid, RNT, lines_smem(N), st>>>(W, kscale, ecut, tw);
        else if (kind == 1)
            k_zlines<N, 1><<<grid, RNT, lines_smem(N), st>>>(W, kscale, ecut, tw);
    });
}

void rows_zlines_energy(int n, const float2* W, int batch, float kscale, const float2* tw, double* part,
                        cudaStream_t st) {
    if (batch == 0) return;
    SGW_DISPATCH_ROWS(n, k_zlines_energy<N><<<dim3((N / LT) * N, batch), RNT, lines_smem(N), st>>>(W, kscale, tw,
                                                                                                     part));
}

// The W input of the step is transformed back along y in place (the plane path leaves it intact;
// every caller overwrites W afterwards).  At 288 one cluster of CTAs per plane does the whole pass.
void rows_plane_step(int n, const StepArgs& a, int batch, const float2* tw, cudaStream_t st, int variant, int line_form) {
    if (batch == 0) return;
    if (cluster_plane(n)) return cplane_step(a, batch, tw, st, variant, line_form);
    ylines(n, const_cast<float2*>(a.W), batch, +1, tw, st);
    const int slots = a.kbc != nullptr ? a.max_plane_slots : 0;
    SGW_DISPATCH_ROWS(n, k_rows_step<N><<<dim3(N * N / RR, batch), RNT, rows_step_smem(N, slots), st>>>(a, tw));
    if (a.Wout != nullptr) ylines(n, a.Wout, batch, -1, tw, st);
}

void rows_plane_inv(int n, const float2* W, int batch, const float2* tw, int mode, float2* out_c, const float* vloc,
                    float* vtot, float* dv, float* uR, int64_t uR_stride, float* out_re, cudaStream_t st) {
    if (batch == 0) return;
    ylines(n, const_cast<float2*>(W), batch, +1, tw, st);
    SGW_DISPATCH_ROWS(n, k_rows_inv<N><<<dim3(N * N / RR, batch), RNT, rows_smem(N), st>>>(
                             W, tw, mode, out_c, vloc, vtot, dv, uR, uR_stride, out_re));
}

void rows_density_fwd(int n, const float2* psi, int n_samples, int n_eta, float weight, float* rho0, int store_rho0,
                      float2* Wp, const float2* tw, cudaStream_t st) {
    if (n_samples == 0) return;
    SGW_DISPATCH_ROWS(n, k_rows_density<N><<<dim3(N * N / RR, n_samples), RNT, rows_smem(N), st>>>(
                             psi, n_eta, weight, rho0, store_rho0, Wp, tw));
    ylines(n, Wp, n_samples, -1, tw, st);
}

}  // namespace sgw
