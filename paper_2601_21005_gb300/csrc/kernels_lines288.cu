// Two-stage 288-point line transforms for the 288^3 grid (the y and z passes of the row form).
//
// 288 = 16 x 18, Cooley-Tukey with n = 18 n1 + n2 (n1 < 16, n2 < 18), k = k1 + 16 k2 (k1 < 16,
// k2 < 18) and W_M = exp(dir 2 pi i / M):
//   X[k1 + 16 k2] = sum_n2 W18^(n2 k2) W288^(n2 k1) sum_n1 x[18 n1 + n2] W16^(n1 k1).
// Stage A: for each n2 a 16-point DFT over n1, times W288^(n2 k1).  Stage B: for each k1 an
// 18-point DFT over n2.  The same identity read backwards is the inverse with the stages swapped:
//   x[18 n1 + n2] = sum_k1 W16^(n1 k1) W288^(n2 k1) sum_k2 X[k1 + 16 k2] W18^(n2 k2)   (dir = +1),
// so a forward transform, a diagonal factor and an inverse (the z lines) keep the 18 values of
// one k1 in one thread's registers from the forward stage B through the inverse's first stage.
//
// A tile is 16 columns of one plane (y lines) or of one ky row (z lines), 288 threads: in stage A
// thread (column l, n2) owns one 16-point butterfly, in stage B thread (l, k1) one 18-point
// butterfly (256 of the 288 threads).  Loads and stores in HBM take 16 consecutive columns, so a
// warp touches two 128-byte segments per access; the shared-memory tile [n2][k1][16 columns] is
// read and written in 128-byte half-warp rows (no bank conflicts).  One shared-memory round trip
// per transform, against three for the radix plan 8, 4, 3, 3.
#include "fft288_2s.cuh"
#include "fft_smem.cuh"
#include "grid_common.cuh"
#include "kb_unit.cuh"
#include "sgw_internal.cuh"

namespace sgw {
namespace {

constexpr int L2N = 288;                 // line length
constexpr int L2T = 16;                  // columns per tile
constexpr int L2NT = L2T * 18;           // threads per tile (stage A butterflies)

}  // namespace

// The y lines of a tile of 16 x-columns of one z plane, in place (dir -1 forward, +1 inverse).
template <int DIR>
__global__ void __launch_bounds__(L2NT, 3) k_ylines288_2s(float2* __restrict__ W, const float2* __restrict__ tw) {
    extern __shared__ __align__(16) float2 sm[];
    float2* tws = sm + L2N * L2T;
    for (int i = threadIdx.x; i < L2N; i += L2NT) tws[i] = __ldg(tw + i);
    const int l = threadIdx.x % L2T, j = threadIdx.x / L2T;
    const int xt = blockIdx.x % (L2N / L2T), z = blockIdx.x / (L2N / L2T);
    float2* base = W + (size_t)blockIdx.y * L2N * L2N * L2N + (size_t)z * L2N * L2N + xt * L2T + l;
    float2 v[18];
    // stage A, n2 = j: x[18 n1 + j] -> DFT16 over n1 -> times W288^(j k1) -> tile[j][k1]
#pragma unroll
    for (int n1 = 0; n1 < 16; ++n1) v[n1] = __ldg(base + (size_t)(18 * n1 + j) * L2N);
    dft16<DIR>(v);
    __syncthreads();                                      // the twiddle table
#pragma unroll
    for (int k1 = 1; k1 < 16; ++k1) v[k1] = cmul(v[k1], tw288<DIR>(tws, j * k1));
#pragma unroll
    for (int k1 = 0; k1 < 16; ++k1) sm[(j * 16 + k1) * L2T + l] = v[k1];
    __syncthreads();
    // stage B, k1 = j: tile[n2][j] -> DFT18 over n2 -> X[j + 16 k2]
    if (j < 16) {
#pragma unroll
        for (int n2 = 0; n2 < 18; ++n2) v[n2] = sm[(n2 * 16 + j) * L2T + l];
        dft18<DIR>(v);
#pragma unroll
        for (int k2 = 0; k2 < 18; ++k2) base[(size_t)(j + 16 * k2) * L2N] = v[k2];
    }
}

// The z lines of a tile of 16 kx-columns at one ky, in place: forward transform along z, the
// k-space factor (KIND 0 kinetic, 1 Coulomb; / n^3), inverse transform.
template <int KIND>
__global__ void __launch_bounds__(L2NT, 3) k_zlines288_2s(float2* __restrict__ W, float kscale, float ecut,
                                                          const float2* __restrict__ tw) {
    extern __shared__ __align__(16) float2 sm[];
    float2* tws = sm + L2N * L2T;
    for (int i = threadIdx.x; i < L2N; i += L2NT) tws[i] = __ldg(tw + i);
    const int l = threadIdx.x % L2T, j = threadIdx.x / L2T;
    const int xt = blockIdx.x % (L2N / L2T), ky = blockIdx.x / (L2N / L2T);
    constexpr size_t ZS = (size_t)L2N * L2N;              // stride between z planes
    float2* base = W + (size_t)blockIdx.y * L2N * ZS + (size_t)ky * L2N + xt * L2T + l;
    float2 v[18];
    // forward stage A, n2 = j
#pragma unroll
    for (int n1 = 0; n1 < 16; ++n1) v[n1] = __ldg(base + (18 * n1 + j) * ZS);
    dft16<-1>(v);
    __syncthreads();
#pragma unroll
    for (int k1 = 1; k1 < 16; ++k1) v[k1] = cmul(v[k1], tw288<-1>(tws, j * k1));
#pragma unroll
    for (int k1 = 0; k1 < 16; ++k1) sm[(j * 16 + k1) * L2T + l] = v[k1];
    __syncthreads();
    // forward stage B (k1 = j), the factor at kz = j + 16 k2, inverse stage B over k2, times
    // W288^(+n2 j), back to the tile at [n2][j]
    if (j < 16) {
#pragma unroll
        for (int n2 = 0; n2 < 18; ++n2) v[n2] = sm[(n2 * 16 + j) * L2T + l];
        dft18<-1>(v);
#pragma unroll
        for (int k2 = 0; k2 < 18; ++k2)
            v[k2] = cscale(v[k2], kspace_factor<L2N, KIND>(xt * L2T + l, ky, j + 16 * k2, kscale, ecut));
        dft18<+1>(v);
#pragma unroll
        for (int n2 = 1; n2 < 18; ++n2) v[n2] = cmul(v[n2], tw288<+1>(tws, n2 * j));
#pragma unroll
        for (int n2 = 0; n2 < 18; ++n2) sm[(n2 * 16 + j) * L2T + l] = v[n2];
    }
    __syncthreads();
    // inverse stage A, n2 = j: tile[j][k1] -> DFT16 over k1 -> x[18 n1 + j]
#pragma unroll
    for (int k1 = 0; k1 < 16; ++k1) v[k1] = sm[(j * 16 + k1) * L2T + l];
    dft16<+1>(v);
#pragma unroll
    for (int n1 = 0; n1 < 16; ++n1) base[(18 * n1 + j) * ZS] = v[n1];
}

// ------------------------------------------------------------------ the 36-row step, two-stage rows
// k_rows36_step with the rows transformed by the 16 x 18 factorisation instead of warp FFTs: one CTA
// per 36-row unit u of vector b (vectors fastest in launch order), 12 warps.
//   inverse along x: stage A for (row, n2) loads x[18 n1 + n2] from HBM, DFT16, times
//     W288^(+n2 k1), into the row's group k1 at slot n2 (a row is 16 groups of 19 slots);
//     stage B for (row, k1) transforms its own group (DFT18 over n2) in place, which leaves
//     column x = k1 + 16 k2 at slot 19 k1 + k2: the unit layout of kb_unit.cuh's LAYOUT 1;
//   KB apply, the pointwise step and the KB partials on that layout;
//   forward along x by the transposed factorisation x = 16 m1 + m2: stage A' for (row, m2)
//     transforms its own group (DFT18 over m1), times W288^(-m2 k1'), in place; stage B' for
//     (row, k1') takes slot k1' of the 16 groups (DFT16 over m2) and stores X[k1' + 18 k2'] to HBM.
// Every shared-memory access is a half-warp over 16 consecutive slots or 16 groups at stride 19
// (no bank conflicts); no stage needs a barrier between its reads and its writes.
constexpr int R2N = 288, R2S = 36, R2P = 304, R2W = 12;

template <int NW>
__global__ void __launch_bounds__(NW * 32, 2) k_rows36_2s(StepArgs a, const float2* __restrict__ tw) {
    constexpr int CNT = NW * 32;
    constexpr size_t NG = (size_t)R2N * R2N * R2N;
    constexpr unsigned UB = R2S * R2N * sizeof(float2), VB = R2S * R2N * sizeof(float);
    extern __shared__ __align__(16) float2 sm[];
    float2* rowb = sm;
    float2* tws = rowb + R2S * R2P;
    float2* kcs = tws + R2N;
    const int b = blockIdx.x, u = blockIdx.y;
    const size_t uoff = (size_t)u * R2S * R2N;
    const size_t off = (size_t)b * NG + uoff;
    const VecInfo inf = a.info[b];
    if ((a.pf_operands & 1) && threadIdx.x == 0) {
        l2_prefetch(a.b1 + off, UB);
        if (a.psi != nullptr) l2_prefetch(a.psi + off, UB);
        if (a.b2 != nullptr) l2_prefetch(a.b2 + off, UB);
        l2_prefetch(a.vpot + (size_t)inf.vrow * NG + uoff, VB);
        if (a.dvpot != nullptr && inf.dvrow >= 0) {
            l2_prefetch(a.dvpot + (size_t)inf.dvrow * NG + uoff, VB);
            l2_prefetch(a.b1 + (size_t)inf.partner * NG + uoff, UB);
        }
    }
    for (int i = threadIdx.x; i < R2N; i += CNT) tws[i] = __ldg(tw + i);
    const float2* kc = a.kbc != nullptr ? a.kbc + (size_t)b * a.n_proj : nullptr;
    if (kc != nullptr) kb_stage_coeffs<CNT>(a, kc, u, kcs);
    __syncthreads();
    float2 v[18];
    {
        const float2* src = a.W + off;
        for (int w = threadIdx.x; w < R2S * 18; w += CNT) {
            const int r = w / 18, n2 = w - 18 * r;
#pragma unroll
            for (int n1 = 0; n1 < 16; ++n1) v[n1] = __ldg(src + r * R2N + 18 * n1 + n2);
            dft16<+1>(v);
#pragma unroll
            for (int k1 = 1; k1 < 16; ++k1) v[k1] = cmul(v[k1], tw288<+1>(tws, n2 * k1));
#pragma unroll
            for (int k1 = 0; k1 < 16; ++k1) rowb[r * R2P + 19 * k1 + n2] = v[k1];
        }
    }
    __syncthreads();
    for (int w = threadIdx.x; w < R2S * 16; w += CNT) {
        float2* g = rowb + (w >> 4) * R2P + 19 * (w & 15);
#pragma unroll
        for (int n2 = 0; n2 < 18; ++n2) v[n2] = g[n2];
        dft18<+1>(v);
#pragma unroll
        for (int k2 = 0; k2 < 18; ++k2) g[k2] = v[k2];
    }
    __syncthreads();
    if (kc != nullptr) kb_apply_unit<R2N, R2P, CNT, 1>(a, u, kcs, rowb);
    const bool stream = (a.pf_operands & 2) != 0;
    if (stream)
        step_pointwise<R2N, R2S, R2P, CNT, 4, 1, true>(a, inf, off, uoff, rowb);
    else
        step_pointwise<R2N, R2S, R2P, CNT, 4, 1>(a, inf, off, uoff, rowb);
    if (a.Wout == nullptr) return;
    __syncthreads();
    if (a.kbp != nullptr) kb_project_unit<R2N, R2P, CNT, 1>(a, u, b, rowb);
    __syncthreads();
    for (int w = threadIdx.x; w < R2S * 16; w += CNT) {
        const int m2 = w & 15;
        float2* g = rowb + (w >> 4) * R2P + 19 * m2;
#pragma unroll
        for (int m1 = 0; m1 < 18; ++m1) v[m1] = g[m1];
        dft18<-1>(v);
#pragma unroll
        for (int k1 = 1; k1 < 18; ++k1) v[k1] = cmul(v[k1], tw288<-1>(tws, m2 * k1));
#pragma unroll
        for (int k1 = 0; k1 < 18; ++k1) g[k1] = v[k1];
    }
    __syncthreads();
    {
        float2* dst = a.Wout + off;
        for (int w = threadIdx.x; w < R2S * 18; w += CNT) {
            const int r = w / 18, k1 = w - 18 * r;
            const float2* g = rowb + r * R2P + k1;
#pragma unroll
            for (int m2 = 0; m2 < 16; ++m2) v[m2] = g[19 * m2];
            dft16<-1>(v);
            if (stream) {
#pragma unroll
                for (int k2 = 0; k2 < 16; ++k2) __stcs(dst + r * R2N + k1 + 18 * k2, v[k2]);
            } else {
#pragma unroll
                for (int k2 = 0; k2 < 16; ++k2) dst[r * R2N + k1 + 18 * k2] = v[k2];
            }
        }
    }
}

static size_t rows36_2s_smem(int max_unit_slots) {
    return sizeof(float2) * ((size_t)R2S * R2P + R2N + 4 * (size_t)max_unit_slots);
}

cudaError_t rows36_2s_init_attributes(int max_unit_slots) {
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(k_rows36_2s<R2W>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                  (int)cudaSharedmemCarveoutMaxShared)))
        return e;
    return cudaFuncSetAttribute(k_rows36_2s<R2W>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)rows36_2s_smem(max_unit_slots));
}

int rows36_2s_blocks_per_sm(int max_unit_slots) {
    int r = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&r, k_rows36_2s<R2W>, R2W * 32, rows36_2s_smem(max_unit_slots));
    return r;
}

void rows36_2s_step(const StepArgs& a, int batch, const float2* tw, cudaStream_t st) {
    if (batch == 0) return;
    const int slots = a.kbc != nullptr ? a.max_plane_slots : 0;
    k_rows36_2s<R2W><<<dim3(batch, R2N * (R2N / R2S)), R2W * 32, rows36_2s_smem(slots), st>>>(a, tw);
}

static size_t lines2s_smem() { return sizeof(float2) * ((size_t)L2N * L2T + L2N); }

cudaError_t lines288_2s_init_attributes() {
    cudaError_t e;
    const int b = (int)lines2s_smem();
    if ((e = cudaFuncSetAttribute(k_ylines288_2s<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, b))) return e;
    if ((e = cudaFuncSetAttribute(k_ylines288_2s<-1>, cudaFuncAttributeMaxDynamicSharedMemorySize, b))) return e;
    if ((e = cudaFuncSetAttribute(k_zlines288_2s<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, b))) return e;
    return cudaFuncSetAttribute(k_zlines288_2s<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
}

int lines288_2s_blocks_per_sm() {
    int r = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&r, k_zlines288_2s<0>, L2NT, lines2s_smem());
    return r;
}

void ylines288_2s(float2* W, int batch, int dir, const float2* tw, cudaStream_t st) {
    if (batch == 0) return;
    const dim3 grid((L2N / L2T) * L2N, batch);
    if (dir > 0)
        k_ylines288_2s<1><<<grid, L2NT, lines2s_smem(), st>>>(W, tw);
    else
        k_ylines288_2s<-1><<<grid, L2NT, lines2s_smem(), st>>>(W, tw);
}

void zlines288_2s(float2* W, int batch, int kind, float kscale, float ecut, const float2* tw, cudaStream_t st) {
    if (batch == 0) return;
    const dim3 grid((L2N / L2T) * L2N, batch);
    if (kind == 0)
        k_zlines288_2s<0><<<grid, L2NT, lines2s_smem(), st>>>(W, kscale, ecut, tw);
    else
        k_zlines288_2s<1><<<grid, L2NT, lines2s_smem(), st>>>(W, kscale, ecut, tw);
}

}  // namespace sgw
