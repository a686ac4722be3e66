// The 288^3 grid in two HBM passes per Chebyshev term.
//
// A 288^2 complex plane (663 KB) is more than one CTA's shared memory, so the row path splits its
// 2D transform into separate passes over x rows and y lines (four HBM passes per term).  Here a
// thread-block cluster of 8 CTAs holds one plane instead: CTA c owns 36 of the 288 columns while
// the plane is transformed along y and 36 of the rows while it is transformed along x, and the
// two layouts are exchanged through distributed shared memory (plain loads and stores of a peer
// CTA's shared memory inside the cluster; no TMA multicast).  Every 288-point line transform is
// done by one warp in registers and shuffles (warp_fft.cuh), and the exchanges cost no extra pass:
// the warp transforming row y along x loads its 288 points straight from the columns of the 8
// CTAs, and the forward transform along x stores its outputs straight into them.  So one term is
//   [z lines: FFT z, * T(k) / n^3, inverse FFT z]  ->  [cluster plane: inverse FFT y, inverse FFT x
//   (inputs from the cluster), + V b + V_NL b, Chebyshev combine, write, per-slot KB partials,
//   FFT x (outputs into the cluster), FFT y]
// i.e. the two passes of the plane path (Sec. 2.2: the cost of an H application is dominated by
// the FFTs; the potential multiply and the KB apply are fused into them).  The KB tables are per
// unit of 36 rows (a CTA's rows of a plane).
#include <cooperative_groups.h>

#include "fft_smem.cuh"
#include "grid_common.cuh"
#include "kb_unit.cuh"
#include "sgw_internal.cuh"
#include "warp_fft.cuh"

namespace cg = cooperative_groups;

namespace sgw {

constexpr int CN = 288;                 // grid side
constexpr int CL = 8;                   // CTAs per cluster: one xy plane
constexpr int CS = CN / CL;             // 36 columns (y phase) or rows (x phase) per CTA
constexpr int PC = CS + 1;              // shared-memory pitch of the columns [y][36]
constexpr int PR = CN + 1;              // shared-memory pitch of the rows [36][x]
constexpr int SLAB = CN * PC + CS * PR; // float2 elements of the column and row buffers

bool cluster_plane(int n) { return n == CN; }
int cluster_unit_rows() { return CS; }
size_t cplane_smem(int max_unit_slots) { return sizeof(float2) * (SLAB + CN + 4 * (size_t)max_unit_slots); }

// 32-bit shared::cluster address of the same offset as local pointer p in the shared memory of
// cluster CTA `rank`, and loads / stores through it
__device__ __forceinline__ uint32_t dsm_addr(const void* p, uint32_t rank) {
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
    return r;
}
__device__ __forceinline__ float2 ld_dsm(uint32_t addr) {
    float2 v;
    asm volatile("ld.shared::cluster.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(addr) : "memory");
    return v;
}
__device__ __forceinline__ void st_dsm(uint32_t addr, float2 v) {
    asm volatile("st.shared::cluster.v2.f32 [%0], {%1, %2};" ::"r"(addr), "f"(v.x), "f"(v.y) : "memory");
}

// The two compiled forms of the cluster step (a launch choice; results are identical): 32 warps
// per CTA (the default) or 18; one CTA per SM either way (its column and row buffers take 176 KB).
template <int V> struct CPlaneCfg;
template <> struct CPlaneCfg<0> { static constexpr int W = 32; };
template <> struct CPlaneCfg<1> { static constexpr int W = 18; };

// ------------------------------------------------------------------ fused Chebyshev step
// Cluster (8 CTAs) per plane z of vector b: grid (8 * batch, 288), vectors fastest in launch order.  CTA c keeps the plane's columns
// 36c .. 36c + 35 in `colb` [y][36] and its rows 36c .. 36c + 35 in `rowb` [36][x].  Each transform
// along x or y is a 288-point warp FFT of one line (warp_fft.cuh); warp w takes the lines
// w, w + W, ... of the 36, loads a line, transforms it and stores it, so no transform waits at a
// barrier and no warp holds data across one.  Barriers: the CTA's after the column load, after the
// row transforms, per KB colour and before the store; the cluster's (1) after the column transforms
// (the columns may be read), (2) after the pointwise step (every CTA has read the columns it needed,
// so they may be overwritten, and a CTA may leave), (3) after the exchange back (the columns are
// complete).  Every CTA of a cluster takes the same branches (the arguments are uniform), so each
// reaches the same cluster barriers.
template <int V>
__global__ void __cluster_dims__(CL, 1, 1) __launch_bounds__(CPlaneCfg<V>::W * 32, 1)
    k_cplane_step(StepArgs a, const float2* __restrict__ tw) {
    constexpr int NW = CPlaneCfg<V>::W, CNT = NW * 32;
    extern __shared__ __align__(16) float2 sm[];
    constexpr size_t NG = (size_t)CN * CN * CN;
    float2* colb = sm;
    float2* rowb = colb + CN * PC;
    float2* tws = rowb + CS * PR;
    float2* kcs = tws + CN;
    cg::cluster_group cl = cg::this_cluster();
    const int c = (int)cl.block_rank();
    const int b = blockIdx.x / CL, z = blockIdx.y;        // vectors fastest in launch order
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int n1 = wfft_n1(lane), k1 = wfft_k1(lane);
    const int u = z * CL + c;                              // KB unit: rows 36c .. 36c + 35 of plane z
    const size_t plane = (size_t)b * NG + (size_t)z * CN * CN;
    const size_t uoff = (size_t)u * CS * CN;
    const size_t off = (size_t)b * NG + uoff;
    for (int i = threadIdx.x; i < CN; i += CNT) tws[i] = __ldg(tw + i);
    const VecInfo inf = a.info[b];
    const float2* kc = a.kbc != nullptr ? a.kbc + (size_t)b * a.n_proj : nullptr;
    if (kc != nullptr) kb_stage_coeffs<CNT>(a, kc, u, kcs);
    // columns 36c .. 36c + 35 of the plane from HBM (rows of 288 bytes)
    {
        const float2* src = a.W + plane + c * CS;
        for (int q = threadIdx.x; q < CN * CS / 2; q += CNT) {
            const int y = q / (CS / 2), x = 2 * (q % (CS / 2));
            const float4 v = ld4(src + (size_t)y * CN + x);
            colb[y * PC + x] = make_float2(v.x, v.y);
            colb[y * PC + x + 1] = make_float2(v.z, v.w);
        }
    }
    __syncthreads();
    // inverse FFT along y, a warp per column, in place
    for (int l = warp; l < CS; l += NW) {
        float2 v[9];
#pragma unroll
        for (int n = 0; n < 9; ++n) v[n] = colb[(n1 + 32 * n) * PC + l];
        warp_fft288<+1>(v, lane, tws);
#pragma unroll
        for (int k = 0; k < 9; ++k) colb[(k + 9 * k1) * PC + l] = v[k];
    }
    cl.sync();                                             // (1) the plane's columns are transformed
    // inverse FFT along x of rows 36c + l: point x of a row is column x mod 36 of CTA x / 36
    for (int l = warp; l < CS; l += NW) {
        const int row = c * CS + l;
        float2 v[9];
#pragma unroll
        for (int n = 0; n < 9; ++n) {
            const int x = n1 + 32 * n, r = x / CS;
            v[n] = ld_dsm(dsm_addr(colb, r) + (uint32_t)sizeof(float2) * (row * PC + x - r * CS));
        }
        warp_fft288<+1>(v, lane, tws);
#pragma unroll
        for (int k = 0; k < 9; ++k) rowb[l * PR + k + 9 * k1] = v[k];
    }
    __syncthreads();
    if (kc != nullptr) kb_apply_unit<CN, PR, CNT>(a, u, kcs, rowb);
    step_pointwise<CN, CS, PR, CNT>(a, inf, off, uoff, rowb);
    cl.sync();                                             // (2) no CTA reads another's columns any more
    if (a.Wout == nullptr) return;
    if (a.kbp != nullptr) kb_project_unit<CN, PR, CNT>(a, u, b, rowb);
    // forward FFT along x, a warp per row; point x goes to column x mod 36 of CTA x / 36
    for (int l = warp; l < CS; l += NW) {
        const int row = c * CS + l;
        float2 v[9];
#pragma unroll
        for (int n = 0; n < 9; ++n) v[n] = rowb[l * PR + n1 + 32 * n];
        warp_fft288<-1>(v, lane, tws);
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            const int x = k + 9 * k1, r = x / CS;
            st_dsm(dsm_addr(colb, r) + (uint32_t)sizeof(float2) * (row * PC + x - r * CS), v[k]);
        }
    }
    cl.sync();                                             // (3) the plane's columns are complete
    // forward FFT along y, a warp per column, in place; then the columns to HBM
    for (int l = warp; l < CS; l += NW) {
        float2 v[9];
#pragma unroll
        for (int n = 0; n < 9; ++n) v[n] = colb[(n1 + 32 * n) * PC + l];
        warp_fft288<-1>(v, lane, tws);
#pragma unroll
        for (int k = 0; k < 9; ++k) colb[(k + 9 * k1) * PC + l] = v[k];
    }
    __syncthreads();
    {
        float2* dst = a.Wout + plane + c * CS;
        for (int q = threadIdx.x; q < CN * CS / 2; q += CNT) {
            const int y = q / (CS / 2), x = 2 * (q % (CS / 2));
            st4(dst + (size_t)y * CN + x, colb[y * PC + x], colb[y * PC + x + 1]);
        }
    }
}

// ------------------------------------------------------------------ the row form of the step
// The same 36-row units without a cluster: the y transforms are separate passes over tiles of 16
// x-columns (k_ylines288, in place on W), and k_rows36_step transforms its 36 rows along x, applies
// the potential and KB parts and the Chebyshev combine, and transforms back.  Four HBM passes per
// term (with the z lines) instead of two, but every CTA is independent and two fit on an SM.
constexpr int YT = 16;                  // x columns per y-line tile
constexpr int YP = YT + 1;              // the shared-memory pitch of a warp-FFT tile
constexpr int ZT_NT = 192;              // threads of a Stockham line tile of 16 columns
constexpr int ROWS36_W = 12;            // warps of the row step (3 rows each)

// The y lines: tiles of 16 x-columns of one z plane, in place; radix plan 8, 4, 3, 3 with the first
// stage loaded from HBM into registers and the last stage stored from registers (as the z lines).
template <int DIR>
__global__ void __launch_bounds__(ZT_NT, 4) k_ylines288(float2* __restrict__ W, const float2* __restrict__ tw) {
    constexpr int TX = YT, NT = ZT_NT;
    extern __shared__ __align__(16) float2 sm[];
    for (int i = threadIdx.x; i < CN; i += NT) sm[TX * CN + i] = __ldg(tw + i);
    const TwShared tws{sm + TX * CN};
    const int xt = blockIdx.x % (CN / TX), z = blockIdx.x / (CN / TX);
    float2* base = W + (size_t)blockIdx.y * CN * CN * CN + (size_t)z * CN * CN + xt * TX;
    {
        constexpr int R = 8, NB = CN / R, TOT = TX * NB, PER = (TOT + NT - 1) / NT;
        float2 v[PER][R];
#pragma unroll
        for (int p = 0; p < PER; ++p) {
            const int q = threadIdx.x + p * NT;
            if (q < TOT) {
                const int l = q % TX, j = q / TX;
#pragma unroll
                for (int r = 0; r < R; ++r) v[p][r] = __ldg(base + (size_t)(j + r * NB) * CN + l);
            }
        }
        stage_r2s<CN, R, 1, TX, 1, TX, NT, DIR>(v, sm, tws);
    }
    fft_stage<CN, 4, 8, TX, 1, TX, NT, DIR>(sm, tws);
    fft_stage<CN, 3, 32, TX, 1, TX, NT, DIR>(sm, tws);
    {
        constexpr int R = 3, NS = 96, TOT = TX * NS, PER = (TOT + NT - 1) / NT;
        float2 v[PER][R];
        stage_s2r<CN, R, NS, TX, 1, TX, NT, DIR>(sm, v, tws);
#pragma unroll
        for (int p = 0; p < PER; ++p) {
            const int q = threadIdx.x + p * NT;
            if (q < TOT) {
                const int l = q % TX, j = q / TX;
#pragma unroll
                for (int r = 0; r < R; ++r) base[(size_t)(j + r * NS) * CN + l] = v[p][r];
            }
        }
    }
}

// One CTA per 36-row unit u of vector b (after the inverse y lines), vectors fastest in launch order:
// the CTAs of one unit for all vectors run together, so the unit's potential rows and KB entries
// come from DRAM once and from L2 for the other vectors (at 288^3 neither fits in L2 whole).  The
// unit's rows are copied into shared memory by 16-byte cp.async copies (all in flight at once, no
// registers held), each row is transformed along x by a warp FFT in place, then the KB apply, the
// pointwise step and the KB partials, then a warp transforms each row forward and the rows are
// written out.  With bit 0 of a.pf_operands thread 0 first asks L2 for the unit's pointwise operands (b1, psi,
// b2, potential rows) so that they arrive while the transforms run (a launch hint).
constexpr int PR36 = CN + 2;            // row pitch of the 36-row step: rows start on 16-byte boundaries

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem) : "memory");
}

template <int NW>
__global__ void __launch_bounds__(NW * 32, 2) k_rows36_step(StepArgs a, const float2* __restrict__ tw) {
    constexpr int CNT = NW * 32;
    constexpr size_t NG = (size_t)CN * CN * CN;
    constexpr unsigned UB = CS * CN * sizeof(float2), VB = CS * CN * sizeof(float);
    extern __shared__ __align__(16) float2 sm[];
    float2* rowb = sm;
    float2* tws = rowb + CS * PR36;
    float2* kcs = tws + CN;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int n1 = wfft_n1(lane), k1 = wfft_k1(lane);
    const int b = blockIdx.x, u = blockIdx.y;
    const size_t uoff = (size_t)u * CS * CN;
    const size_t off = (size_t)b * NG + uoff;
    const VecInfo inf = a.info[b];
    {
        const float2* src = a.W + off;
        for (int q = threadIdx.x; q < CS * CN / 2; q += CNT) {
            const int y = q / (CN / 2), x = 2 * (q % (CN / 2));
            cp_async16(rowb + y * PR36 + x, src + y * CN + x);
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    }
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
    for (int i = threadIdx.x; i < CN; i += CNT) tws[i] = __ldg(tw + i);
    const float2* kc = a.kbc != nullptr ? a.kbc + (size_t)b * a.n_proj : nullptr;
    if (kc != nullptr) kb_stage_coeffs<CNT>(a, kc, u, kcs);
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    __syncthreads();
    for (int l = warp; l < CS; l += NW) {
        float2 v[9];
#pragma unroll
        for (int n = 0; n < 9; ++n) v[n] = rowb[l * PR36 + n1 + 32 * n];
        warp_fft288<+1>(v, lane, tws);
        __syncwarp();
#pragma unroll
        for (int k = 0; k < 9; ++k) rowb[l * PR36 + k + 9 * k1] = v[k];
    }
    __syncthreads();
    if (kc != nullptr) kb_apply_unit<CN, PR36, CNT>(a, u, kcs, rowb);
    const bool stream = (a.pf_operands & 2) != 0;
    if (stream)
        step_pointwise<CN, CS, PR36, CNT, 4, 0, true>(a, inf, off, uoff, rowb);
    else
        step_pointwise<CN, CS, PR36, CNT, 4>(a, inf, off, uoff, rowb);
    if (a.Wout == nullptr) return;
    __syncthreads();
    if (a.kbp != nullptr) kb_project_unit<CN, PR36, CNT>(a, u, b, rowb);
    __syncthreads();
    for (int l = warp; l < CS; l += NW) {
        float2 v[9];
#pragma unroll
        for (int n = 0; n < 9; ++n) v[n] = rowb[l * PR36 + n1 + 32 * n];
        warp_fft288<-1>(v, lane, tws);
        __syncwarp();
#pragma unroll
        for (int k = 0; k < 9; ++k) rowb[l * PR36 + k + 9 * k1] = v[k];
    }
    __syncthreads();
    {
        float2* dst = a.Wout + off;
#pragma unroll 4
        for (int q = threadIdx.x; q < CS * CN / 2; q += CNT) {
            const int y = q / (CN / 2), x = 2 * (q % (CN / 2));
            if (stream)
                stcs4(dst + y * CN + x, rowb[y * PR36 + x], rowb[y * PR36 + x + 1]);
            else
                st4(dst + y * CN + x, rowb[y * PR36 + x], rowb[y * PR36 + x + 1]);
        }
    }
}

// ------------------------------------------------------------------ z lines, register-ended
// One CTA per (TX kx-columns, ky) of a vector whose planes are xy-transformed: FFT along z (plan
// 8, 4, 3, 3; first stage from HBM), the diagonal k-space factor (KIND 0 kinetic, 1 Coulomb; / n^3)
// on the last stage's outputs in registers, the inverse with the reversed plan 3, 3, 4, 8 (first
// stage from those registers, last stage stored to HBM).  Three shared-memory round trips fewer
// than transforming a loaded tile in shared memory both ways.
template <int TX> struct ZCfg {
    static constexpr int NT = TX == 16 ? 192 : 384;        // stages of 8, 4, 3 fill every thread
    static constexpr int MINB = TX == 16 ? 4 : 2;          // 85 registers a thread: no spills
};

template <int TX>
__device__ __forceinline__ void zl_forward(const float2* __restrict__ base, float2* sm, float2 (&c)[(TX * 96 + ZCfg<TX>::NT - 1) / ZCfg<TX>::NT][3],
                                           TwShared tws) {
    constexpr int NT = ZCfg<TX>::NT;
    constexpr int R = 8, NB = CN / R, TOT = TX * NB, PER = (TOT + NT - 1) / NT;
    float2 v[PER][R];
#pragma unroll
    for (int p = 0; p < PER; ++p) {
        const int q = threadIdx.x + p * NT;
        if (q < TOT) {
            const int l = q % TX, j = q / TX;
#pragma unroll
            for (int r = 0; r < R; ++r) v[p][r] = __ldg(base + (size_t)(j + r * NB) * CN * CN + l);
        }
    }
    stage_r2s<CN, R, 1, TX, 1, TX, NT, -1>(v, sm, tws);
    fft_stage<CN, 4, 8, TX, 1, TX, NT, -1>(sm, tws);
    fft_stage<CN, 3, 32, TX, 1, TX, NT, -1>(sm, tws);
    stage_s2r<CN, 3, 96, TX, 1, TX, NT, -1>(sm, c, tws);
}

template <int TX, int KIND>
__global__ void __launch_bounds__(ZCfg<TX>::NT, ZCfg<TX>::MINB) k_zlines_reg(float2* __restrict__ W, float kscale,
                                                                           float ecut, const float2* __restrict__ tw) {
    extern __shared__ __align__(16) float2 sm[];
    constexpr int NT = ZCfg<TX>::NT, NXT = CN / TX;
    constexpr int TOT3 = TX * 96, P3 = (TOT3 + NT - 1) / NT;
    for (int i = threadIdx.x; i < CN; i += NT) sm[TX * CN + i] = __ldg(tw + i);
    const TwShared tws{sm + TX * CN};
    const int xt = blockIdx.x % NXT, ky = blockIdx.x / NXT;
    float2* base = W + (size_t)blockIdx.y * CN * CN * CN + (size_t)ky * CN + xt * TX;
    float2 c[P3][3];
    zl_forward<TX>(base, sm, c, tws);
    // X[l][kz = j + 96 q] in registers: the k-space factor
#pragma unroll
    for (int p = 0; p < P3; ++p) {
        const int q = threadIdx.x + p * NT;
        if (q < TOT3) {
            const int l = q % TX, j = q / TX;
#pragma unroll
            for (int r = 0; r < 3; ++r) c[p][r] = cscale(c[p][r], kspace_factor<CN, KIND>(xt * TX + l, ky, j + 96 * r,
                                                                                          kscale, ecut));
        }
    }
    // inverse with the reversed plan: its first radix-3 stage takes x[j + 96 r] = the registers
    stage_r2s<CN, 3, 1, TX, 1, TX, NT, +1>(c, sm, tws);
    fft_stage<CN, 3, 3, TX, 1, TX, NT, +1>(sm, tws);
    fft_stage<CN, 4, 9, TX, 1, TX, NT, +1>(sm, tws);
    {
        constexpr int R = 8, NS = CN / R, TOT = TX * NS, PER = (TOT + NT - 1) / NT;
        float2 v[PER][R];
        stage_s2r<CN, R, NS, TX, 1, TX, NT, +1>(sm, v, tws);
#pragma unroll
        for (int p = 0; p < PER; ++p) {
            const int q = threadIdx.x + p * NT;
            if (q < TOT) {
                const int l = q % TX, j = q / TX;
#pragma unroll
                for (int r = 0; r < R; ++r) base[(size_t)(j + r * NS) * CN * CN + l] = v[p][r];
            }
        }
    }
}

// The z lines with warp FFTs: tiles of 16 kx-columns at one ky, a warp per column: FFT along z,
// the k-space factor on the outputs, back through shared memory (the warp's own column) into the
// input order, the inverse FFT.  Two CTA barriers per tile.
template <int KIND>
__global__ void __launch_bounds__(YT * 32, 2) k_zlines_warp(float2* __restrict__ W, float kscale, float ecut,
                                                            const float2* __restrict__ tw) {
    constexpr int CNT = YT * 32;
    extern __shared__ __align__(16) float2 sm[];
    float2* tws = sm + CN * YP;
    for (int i = threadIdx.x; i < CN; i += CNT) tws[i] = __ldg(tw + i);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int xt = blockIdx.x % (CN / YT), ky = blockIdx.x / (CN / YT);
    float2* base = W + (size_t)blockIdx.y * CN * CN * CN + (size_t)ky * CN + xt * YT;
    for (int q = threadIdx.x; q < CN * YT / 2; q += CNT) {
        const int z = q / (YT / 2), x = 2 * (q % (YT / 2));
        const float4 v = ld4(base + (size_t)z * CN * CN + x);
        sm[z * YP + x] = make_float2(v.x, v.y);
        sm[z * YP + x + 1] = make_float2(v.z, v.w);
    }
    __syncthreads();
    {
        const int n1 = wfft_n1(lane), k1 = wfft_k1(lane);
        float2 v[9];
#pragma unroll
        for (int n = 0; n < 9; ++n) v[n] = sm[(n1 + 32 * n) * YP + warp];
        warp_fft288<-1>(v, lane, tws);
#pragma unroll
        for (int k = 0; k < 9; ++k)
            v[k] = cscale(v[k], kspace_factor<CN, KIND>(xt * YT + warp, ky, k + 9 * k1, kscale, ecut));
        __syncwarp();
#pragma unroll
        for (int k = 0; k < 9; ++k) sm[(k + 9 * k1) * YP + warp] = v[k];
        __syncwarp();
#pragma unroll
        for (int n = 0; n < 9; ++n) v[n] = sm[(n1 + 32 * n) * YP + warp];
        warp_fft288<+1>(v, lane, tws);
        __syncwarp();
#pragma unroll
        for (int k = 0; k < 9; ++k) sm[(k + 9 * k1) * YP + warp] = v[k];
    }
    __syncthreads();
    for (int q = threadIdx.x; q < CN * YT / 2; q += CNT) {
        const int z = q / (YT / 2), x = 2 * (q % (YT / 2));
        st4(base + (size_t)z * CN * CN + x, sm[z * YP + x], sm[z * YP + x + 1]);
    }
}

// ------------------------------------------------------------------ launchers
template <int TX> static size_t zreg_smem() { return sizeof(float2) * ((size_t)TX * CN + CN); }

static size_t rows36_smem(int max_unit_slots) { return sizeof(float2) * ((size_t)CS * PR36 + CN + 4 * (size_t)max_unit_slots); }
static size_t ylines288_smem() { return sizeof(float2) * ((size_t)CN * YT + CN); }
static size_t zwarp_smem() { return sizeof(float2) * ((size_t)CN * YP + CN); }

template <class K> static cudaError_t big_smem(K kern, size_t bytes) {
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                                  (int)cudaSharedmemCarveoutMaxShared)))
        return e;
    return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

cudaError_t cluster_init_attributes(int max_unit_slots) {
    cudaError_t e;
    if ((e = big_smem(k_cplane_step<0>, cplane_smem(max_unit_slots)))) return e;
    if ((e = big_smem(k_cplane_step<1>, cplane_smem(max_unit_slots)))) return e;
    if ((e = big_smem(k_rows36_step<ROWS36_W>, rows36_smem(max_unit_slots)))) return e;
    if ((e = big_smem(k_ylines288<1>, ylines288_smem()))) return e;
    if ((e = big_smem(k_ylines288<-1>, ylines288_smem()))) return e;
    if ((e = big_smem(k_zlines_warp<0>, zwarp_smem()))) return e;
    if ((e = big_smem(k_zlines_warp<1>, zwarp_smem()))) return e;
    if ((e = cudaFuncSetAttribute(k_zlines_reg<16, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)zreg_smem<16>())))
        return e;
    if ((e = cudaFuncSetAttribute(k_zlines_reg<16, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)zreg_smem<16>())))
        return e;
    if ((e = cudaFuncSetAttribute(k_zlines_reg<32, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)zreg_smem<32>())))
        return e;
    if ((e = cudaFuncSetAttribute(k_zlines_reg<32, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)zreg_smem<32>())))
        return e;
    if ((e = rows36_2s_init_attributes(max_unit_slots))) return e;
    return lines288_2s_init_attributes();
}

// variant 0: the row form; 1, 2: the cluster form with 32 / 18 warps
int cplane_blocks_per_sm(int variant, int max_unit_slots) {
    int r = 0;
    if (variant == 1)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&r, k_cplane_step<0>, CPlaneCfg<0>::W * 32,
                                                      cplane_smem(max_unit_slots));
    else if (variant == 2)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&r, k_cplane_step<1>, CPlaneCfg<1>::W * 32,
                                                      cplane_smem(max_unit_slots));
    else
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&r, k_rows36_step<ROWS36_W>, ROWS36_W * 32,
                                                      rows36_smem(max_unit_slots));
    return r;
}

int zlines_reg_blocks_per_sm(int form) {
    int r = 0;
    if (form >= 3) return lines288_2s_blocks_per_sm();
    if (form == 2)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&r, k_zlines_warp<0>, YT * 32, zwarp_smem());
    else if (form == 1)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&r, k_zlines_reg<32, 0>, ZCfg<32>::NT, zreg_smem<32>());
    else
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&r, k_zlines_reg<16, 0>, ZCfg<16>::NT, zreg_smem<16>());
    return r;
}

void cplane_step(const StepArgs& a, int batch, const float2* tw, cudaStream_t st, int variant, int line_form) {
    if (batch == 0) return;
    const int slots = a.kbc != nullptr ? a.max_plane_slots : 0;
    if (variant == 1) {
        k_cplane_step<0><<<dim3(CL * batch, CN), CPlaneCfg<0>::W * 32, cplane_smem(slots), st>>>(a, tw);
    } else if (variant == 2) {
        k_cplane_step<1><<<dim3(CL * batch, CN), CPlaneCfg<1>::W * 32, cplane_smem(slots), st>>>(a, tw);
    } else {
        lines288(const_cast<float2*>(a.W), batch, +1, line_form, tw, st);
        rows36_step(a, batch, tw, st, line_form);
        if (a.Wout != nullptr) lines288(a.Wout, batch, -1, line_form, tw, st);
    }
}

void lines288(float2* W, int batch, int dir, int form, const float2* tw, cudaStream_t st) {
    if (batch == 0) return;
    if (form >= 3) return ylines288_2s(W, batch, dir, tw, st);
    const dim3 yg((CN / YT) * CN, batch);
    if (dir > 0)
        k_ylines288<1><<<yg, ZT_NT, ylines288_smem(), st>>>(W, tw);
    else
        k_ylines288<-1><<<yg, ZT_NT, ylines288_smem(), st>>>(W, tw);
}

void rows36_step(const StepArgs& a, int batch, const float2* tw, cudaStream_t st, int form) {
    if (batch == 0) return;
    if (form == 4) return rows36_2s_step(a, batch, tw, st);
    const int slots = a.kbc != nullptr ? a.max_plane_slots : 0;
    k_rows36_step<ROWS36_W><<<dim3(batch, CN * CL), ROWS36_W * 32, rows36_smem(slots), st>>>(a, tw);
}

// form 0: register-ended Stockham tiles of 16 columns, 1: of 32 columns, 2: warp-FFT tiles of 16,
// 3, 4: two-stage 16 x 18 tiles of 16
void zlines_reg(float2* W, int batch, int kind, int form, float kscale, float ecut, const float2* tw, cudaStream_t st) {
    if (batch == 0) return;
    if (form >= 3) {
        zlines288_2s(W, batch, kind, kscale, ecut, tw, st);
    } else if (form == 2) {
        const dim3 grid((CN / YT) * CN, batch);
        if (kind == 0)
            k_zlines_warp<0><<<grid, YT * 32, zwarp_smem(), st>>>(W, kscale, ecut, tw);
        else
            k_zlines_warp<1><<<grid, YT * 32, zwarp_smem(), st>>>(W, kscale, ecut, tw);
    } else if (form == 1) {
        const dim3 grid((CN / 32) * CN, batch);
        if (kind == 0)
            k_zlines_reg<32, 0><<<grid, ZCfg<32>::NT, zreg_smem<32>(), st>>>(W, kscale, ecut, tw);
        else
            k_zlines_reg<32, 1><<<grid, ZCfg<32>::NT, zreg_smem<32>(), st>>>(W, kscale, ecut, tw);
    } else {
        const dim3 grid((CN / 16) * CN, batch);
        if (kind == 0)
            k_zlines_reg<16, 0><<<grid, ZCfg<16>::NT, zreg_smem<16>(), st>>>(W, kscale, ecut, tw);
        else
            k_zlines_reg<16, 1><<<grid, ZCfg<16>::NT, zreg_smem<16>(), st>>>(W, kscale, ecut, tw);
    }
}

}  // namespace sgw
