// Grid kernels of the H.psi path: a periodic n^3 complex grid function is transformed
// in two passes that each keep their working set on chip:
//   plane pass  (one CTA per xy plane):  2D FFT of the plane through shared memory;
//   pencil pass (one CTA per 16 kx-columns x all kz at one ky): FFT along z, the
//               diagonal k-space multiply, inverse FFT along z.
// H b = IFFT3(T(k) FFT3(b)) + V b + V_NL b is then
//   [plane fwd of b] -> [pencil: z fwd, *T/N^3, z inv] -> [plane: xy inv, + V b + V_NL b,
//   Chebyshev recurrence combine, write; xy fwd of the result for the next term].
// so one Chebyshev term costs two HBM passes over the batch (Sec. 2.2: the cost of each
// H application is dominated by the FFTs; the potential multiply is fused into them).
#include "fft_smem.cuh"
#include "grid_common.cuh"
#include "sgw_internal.cuh"

namespace sgw {

template <int N> struct Cfg {
    static constexpr int PLANE_NT = N == 16 ? 64 : (N == 32 ? 128 : (N == 64 ? 256 : 512));
    static constexpr int P = N + 1;   // smem row pitch of a plane (float2), breaks bank conflicts
    static constexpr int TX = 16;     // pencil tile width along kx (16 x 8 B = 128 B rows)
    static constexpr int PENCIL_NT = (TX * N / 8) < 64 ? 64 : (TX * N / 8);
    static constexpr size_t PLANE_SMEM = sizeof(float2) * N * (N + 1);
    // CTAs per SM the plane kernels are compiled for (register budget 65536 / (NT * MINB))
    static constexpr int PLANE_MINB = N == 128 ? 1 : (N == 64 ? 4 : 6);
    static constexpr size_t PENCIL_SMEM = sizeof(float2) * N * TX;
    // alternative thread count of the fused plane step (one butterfly per thread per stage at 64^2)
    static constexpr int PLANE_NT2 = 2 * PLANE_NT;
};

// CTAs per SM the fused plane step is compiled for, by thread count: registers 65536 / (NT MINB).
// The 512-thread 64^2 variant runs at 40 registers, 3 blocks (48 warps) per SM.
template <int N, int NT> struct PlaneMinB {
    static constexpr int v = (N == 64 && NT == 512) ? 3 : 1024 / NT;
    static constexpr int value = N == 128 ? 1 : (v > 6 ? 6 : (v < 1 ? 1 : v));
};

// ------------------------------------------------------------------ plane <-> smem
template <int N, int NT>
__device__ __forceinline__ void load_plane(float2* sm, const float2* __restrict__ src) {
    constexpr int P = N + 1;
#pragma unroll 8
    for (int q = threadIdx.x; q < N * N / 2; q += NT) {
        const int y = q / (N / 2), x = 2 * (q % (N / 2));
        const float4 v = ld4(src + y * N + x);
        sm[y * P + x] = make_float2(v.x, v.y);
        sm[y * P + x + 1] = make_float2(v.z, v.w);
    }
}

template <int N, int NT>
__device__ __forceinline__ void store_plane(float2* __restrict__ dst, const float2* sm) {
    constexpr int P = N + 1;
#pragma unroll 8
    for (int q = threadIdx.x; q < N * N / 2; q += NT) {
        const int y = q / (N / 2), x = 2 * (q % (N / 2));
        st4(dst + y * N + x, sm[y * P + x], sm[y * P + x + 1]);
    }
}

template <int N, int NT, int DIR, class TW>
__device__ __forceinline__ void fft2_plane(float2* sm, TW tw) {
    constexpr int P = N + 1;
    fft_lines<N, N, 1, P, NT, DIR>(sm, tw);   // along y: line = x, element stride = pitch
    fft_lines<N, N, P, 1, NT, DIR>(sm, tw);   // along x: line = y, element stride = 1
}

// Radix of the last stage of an n-point transform (same plan as NextRadix)
constexpr int last_radix(int n) {
    int ns = 1, r = 1;
    while (ns < n) {
        const int rem = n / ns;
        r = rem == 16 ? 4 : (rem % 8 == 0 ? 8 : (rem % 4 == 0 ? 4 : (rem % 2 == 0 ? 2 : 3)));
        ns *= r;
    }
    return r;
}

// Inverse xy transform of a plane read from global memory: the first stage along y takes its
// inputs straight from global (consecutive threads on consecutive x: coalesced rows), the
// remaining stages run in shared memory; the result is left in sm (pitch N + 1).
template <int N, int NT, class TW>
__device__ __forceinline__ void inv_plane_from_global(float2* sm, const float2* __restrict__ src, TW tw) {
    constexpr int P = N + 1, R1 = NextRadix<N>::value, NB = N / R1, TOT = N * NB, PER = (TOT + NT - 1) / NT;
    float2 v[PER][R1];
#pragma unroll
    for (int p = 0; p < PER; ++p) {
        const int b = threadIdx.x + p * NT;
        if (TOT % NT == 0 || b < TOT) {
            const int l = b % N, j = b / N;
#pragma unroll
            for (int r = 0; r < R1; ++r) v[p][r] = __ldg(src + (j + r * NB) * N + l);
        }
    }
    stage_r2s<N, R1, 1, N, 1, P, NT, +1>(v, sm, tw);
    fft_rec<N, R1, N, 1, P, NT, +1>(sm, tw);            // the other stages along y
    fft_lines<N, N, P, 1, NT, +1>(sm, tw);              // along x
}

// Forward xy transform of the plane in sm, written to global memory: along x, then along y
// with the last stage's outputs stored straight from registers (coalesced rows).
template <int N, int NT, class TW>
__device__ __forceinline__ void fwd_plane_to_global(float2* sm, float2* __restrict__ dst, TW tw) {
    constexpr int P = N + 1, RL = last_radix(N), NS = N / RL, TOT = N * NS, PER = (TOT + NT - 1) / NT;
    fft_lines<N, N, P, 1, NT, -1>(sm, tw);              // along x
    fft_rec_until<N, 1, NS, N, 1, P, NT, -1>(sm, tw);   // along y but the last stage
    float2 c[PER][RL];
    stage_s2r<N, RL, NS, N, 1, P, NT, -1>(sm, c, tw);
#pragma unroll
    for (int p = 0; p < PER; ++p) {
        const int b = threadIdx.x + p * NT;
        if (TOT % NT == 0 || b < TOT) {
            const int l = b % N, j = b / N;
#pragma unroll
            for (int q = 0; q < RL; ++q) dst[(j + q * NS) * N + l] = c[p][q];
        }
    }
}

// ------------------------------------------------------------------ forward plane pass
template <int N>
__global__ void __launch_bounds__(Cfg<N>::PLANE_NT, Cfg<N>::PLANE_MINB)
k_plane_fwd(const float2* __restrict__ in, float2* __restrict__ W, const float2* __restrict__ tw) {
    extern __shared__ float2 sm[];
    constexpr int NT = Cfg<N>::PLANE_NT;
    const size_t plane = ((size_t)blockIdx.y * N + blockIdx.x) * N * N;
    load_plane<N, NT>(sm, in + plane);
    __syncthreads();
    fwd_plane_to_global<N, NT>(sm, W + plane, tw);
}

// ------------------------------------------------------------------ pencil pass
// Radix plans along z (forward order; the inverse uses the reversed plan so that the
// forward's last stage, the k-space multiply and the inverse's first stage stay in registers).
template <int N> struct ZPlan;
template <> struct ZPlan<16> { static constexpr int R1 = 4, R2 = 4, R3 = 0; };
template <> struct ZPlan<32> { static constexpr int R1 = 8, R2 = 4, R3 = 0; };
template <> struct ZPlan<64> { static constexpr int R1 = 8, R2 = 8, R3 = 0; };
template <> struct ZPlan<128> { static constexpr int R1 = 8, R2 = 4, R3 = 4; };

// Forward z transform of a tile (TX kx-columns at one ky): global -> registers -> ... ->
// registers holding X[l][kz = j + q NS_last] (butterfly layout of the last stage).
template <int N, int NT, int PL, int RL>
__device__ __forceinline__ void pencil_forward(const float2* __restrict__ base, float2* sm, float2 (&c)[PL][RL],
                                               const float2* __restrict__ tw) {
    constexpr int TX = Cfg<N>::TX, R1 = ZPlan<N>::R1, R2 = ZPlan<N>::R2, R3 = ZPlan<N>::R3;
    constexpr int P1 = (TX * (N / R1) + NT - 1) / NT;
    float2 a[P1][R1];
#pragma unroll
    for (int p = 0; p < P1; ++p) {
        const int bb = threadIdx.x + p * NT;
        if ((TX * (N / R1)) % NT == 0 || bb < TX * (N / R1)) {
            const int l = bb % TX, j = bb / TX;
#pragma unroll
            for (int r = 0; r < R1; ++r) a[p][r] = __ldg(base + (size_t)(j + r * (N / R1)) * N * N + l);
        }
    }
    stage_r2s<N, R1, 1, TX, 1, TX, NT, -1>(a, sm, tw);
    if constexpr (R3 == 0) {
        stage_s2r<N, R2, R1, TX, 1, TX, NT, -1>(sm, c, tw);
    } else {
        fft_stage<N, R2, R1, TX, 1, TX, NT, -1>(sm, tw);
        stage_s2r<N, R3, R1 * R2, TX, 1, TX, NT, -1>(sm, c, tw);
    }
}

template <int N, int KIND>
__global__ void __launch_bounds__(Cfg<N>::PENCIL_NT)
k_pencil(float2* __restrict__ W, float kscale, float ecut, const float2* __restrict__ tw, int pf_ahead,
         const VecInfo* __restrict__ info, float dt) {
    extern __shared__ float2 sm[];
    constexpr int NT = Cfg<N>::PENCIL_NT, TX = Cfg<N>::TX, NXT = N / TX;
    constexpr int R1 = ZPlan<N>::R1, R2 = ZPlan<N>::R2, R3 = ZPlan<N>::R3;
    constexpr int RL = R3 == 0 ? R2 : R3;          // last forward radix = first inverse radix
    constexpr int NBL = N / RL;                    // butterflies per line of that stage
    constexpr int PL = (TX * NBL + NT - 1) / NT;
    const int xt = blockIdx.x % NXT, ky = blockIdx.x / NXT;
    float2* base = W + (size_t)blockIdx.y * N * N * N + (size_t)ky * N + xt * TX;
    if (pf_ahead > 0) {
        // the N rows (TX points each) of the block pf_ahead later in launch order, into L2
        const long nxt = (long)blockIdx.y * gridDim.x + blockIdx.x + pf_ahead;
        if (nxt < (long)gridDim.y * gridDim.x && threadIdx.x < N) {
            const int bx = (int)(nxt % gridDim.x), by = (int)(nxt / gridDim.x);
            const float2* nb = W + (size_t)by * N * N * N + (size_t)(bx / NXT) * N + (bx % NXT) * TX;
            l2_prefetch(nb + (size_t)threadIdx.x * N * N, TX * sizeof(float2));
        }
    }
    float2 c[PL][RL];
    pencil_forward<N, NT, PL, RL>(base, sm, c, tw);
    // k-space multiply on X[l][kz = j + q NBL]
    if constexpr (KIND == 2) {
        // split-operator kinetic factor e^{-i s T(k) dt} / N^3, s = +1 or -1 per vector
        const float sdt = (info[blockIdx.y].cset == 0 ? dt : -dt);
        constexpr float inv = 1.0f / ((float)N * N * N);
#pragma unroll
        for (int p = 0; p < PL; ++p) {
            const int bb = threadIdx.x + p * NT;
            if ((TX * NBL) % NT == 0 || bb < TX * NBL) {
                const int l = bb % TX, j = bb / TX;
#pragma unroll
                for (int q = 0; q < RL; ++q) {
                    const int mx = sfreq(xt * TX + l, N), my = sfreq(ky, N), mz = sfreq(j + q * NBL, N);
                    float tk = 0.5f * kscale * (float)(mx * mx + my * my + mz * mz);
                    if (ecut > 0.f) tk = fminf(tk, ecut);
                    float sn, cs;
                    sincosf(tk * sdt, &sn, &cs);
                    c[p][q] = cmul(c[p][q], make_float2(cs * inv, -sn * inv));
                }
            }
        }
    } else {
#pragma unroll
        for (int p = 0; p < PL; ++p) {
            const int bb = threadIdx.x + p * NT;
            if ((TX * NBL) % NT == 0 || bb < TX * NBL) {
                const int l = bb % TX, j = bb / TX;
#pragma unroll
                for (int q = 0; q < RL; ++q)
                    c[p][q] = cscale(c[p][q], kspace_factor<N, KIND>(xt * TX + l, ky, j + q * NBL, kscale, ecut));
            }
        }
    }
    // inverse along z with the reversed plan, first stage from registers
    stage_r2s<N, RL, 1, TX, 1, TX, NT, +1>(c, sm, tw);
    constexpr int P1 = (TX * (N / R1) + NT - 1) / NT;
    float2 a[P1][R1];
    if constexpr (R3 == 0) {
        stage_s2r<N, R1, N / R1, TX, 1, TX, NT, +1>(sm, a, tw);
    } else {
        fft_stage<N, R2, R3, TX, 1, TX, NT, +1>(sm, tw);
        stage_s2r<N, R1, N / R1, TX, 1, TX, NT, +1>(sm, a, tw);
    }
#pragma unroll
    for (int p = 0; p < P1; ++p) {
        const int bb = threadIdx.x + p * NT;
        if ((TX * (N / R1)) % NT == 0 || bb < TX * (N / R1)) {
            const int l = bb % TX, j = bb / TX;
#pragma unroll
            for (int q = 0; q < R1; ++q) base[(size_t)(j + q * (N / R1)) * N * N + l] = a[p][q];
        }
    }
}

// Coulomb energy of the xy-transformed planes: after the z transform F(k) is complete;
// acc[b / per] += dvn * sum_k 4 pi / k^2 |F(k)|^2 (FP64).
template <int N>
__global__ void __launch_bounds__(Cfg<N>::PENCIL_NT)
k_pencil_energy(const float2* __restrict__ W, float kscale, const float2* __restrict__ tw, double* __restrict__ part) {
    extern __shared__ float2 sm[];
    __shared__ double red[32];
    constexpr int NT = Cfg<N>::PENCIL_NT, TX = Cfg<N>::TX, NXT = N / TX;
    constexpr int R2 = ZPlan<N>::R2, R3 = ZPlan<N>::R3;
    constexpr int RL = R3 == 0 ? R2 : R3;
    constexpr int NBL = N / RL;
    constexpr int PL = (TX * NBL + NT - 1) / NT;
    const int xt = blockIdx.x % NXT, ky = blockIdx.x / NXT;
    const float2* base = W + (size_t)blockIdx.y * N * N * N + (size_t)ky * N + xt * TX;
    float2 c[PL][RL];
    pencil_forward<N, NT, PL, RL>(base, sm, c, tw);
    const int my = sfreq(ky, N);
    double s = 0.0;
#pragma unroll
    for (int p = 0; p < PL; ++p) {
        const int bb = threadIdx.x + p * NT;
        if ((TX * NBL) % NT == 0 || bb < TX * NBL) {
            const int l = bb % TX, j = bb / TX;
            const int mx = sfreq(xt * TX + l, N);
#pragma unroll
            for (int q = 0; q < RL; ++q) {
                const int mz = sfreq(j + q * NBL, N);
                const double k2 = (double)kscale * (double)(mx * mx + my * my + mz * mz);
                if (k2 > 0.0) s += 12.566370614359172 / k2 * ((double)c[p][q].x * c[p][q].x + (double)c[p][q].y * c[p][q].y);
            }
        }
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        double t = threadIdx.x < NT / 32 ? red[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (threadIdx.x == 0) part[(size_t)blockIdx.y * gridDim.x + blockIdx.x] = t;
    }
}

// acc[s] = dvn * sum of the partials of vectors s*per .. s*per+per-1 (fixed order: one block per
// sample, a strided pass then a shuffle tree)
__global__ void __launch_bounds__(256)
k_energy_reduce(const double* __restrict__ part, int per, int nblk, double dvn, double* __restrict__ acc) {
    __shared__ double red[8];
    const int s = blockIdx.x;
    const int64_t total = (int64_t)per * nblk;
    const double* p = part + (size_t)s * total;
    double t = 0.0;
    for (int64_t i = threadIdx.x; i < total; i += blockDim.x) t += p[i];
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = t;
    __syncthreads();
    if (threadIdx.x < 32) {
        double u = threadIdx.x < 8 ? red[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) u += __shfl_xor_sync(0xffffffffu, u, o);
        if (threadIdx.x == 0) acc[s] = u * dvn;
    }
}

// ------------------------------------------------------------------ fused Chebyshev step
// L2 prefetch of the pointwise operands of plane z of vector b (one thread)
template <int N>
__device__ __forceinline__ void prefetch_operands(const StepArgs& a, int z, int b) {
    constexpr size_t NG = (size_t)N * N * N;
    constexpr unsigned PB = N * N * sizeof(float2), VB = N * N * sizeof(float);
    const size_t plane = ((size_t)b * N + z) * N * N;
    const VecInfo inf = a.info[b];
    l2_prefetch(a.b1 + plane, PB);
    if (a.psi != nullptr) l2_prefetch(a.psi + plane, PB);
    if (a.b2 != nullptr) l2_prefetch(a.b2 + plane, PB);
    l2_prefetch(a.vpot + (size_t)inf.vrow * NG + (size_t)z * N * N, VB);
    if (a.dvpot != nullptr && inf.dvrow >= 0) {
        l2_prefetch(a.dvpot + (size_t)inf.dvrow * NG + (size_t)z * N * N, VB);
        l2_prefetch(a.b1 + ((size_t)inf.partner * N + z) * N * N, PB);
    }
}

// The fused Chebyshev step on plane z of vector b (see k_plane_step).  IN_SMEM: the plane's input
// W is already in sm (pitch N + 1), else the first inverse stage reads it from global memory.
template <int N, int NT, bool IN_SMEM>
__device__ __forceinline__ void plane_step_body(const StepArgs& a, float2* sm, float2* kcs, TwShared tws, int z,
                                                int b) {
    constexpr int P = N + 1;
    constexpr size_t NG = (size_t)N * N * N;
    const size_t plane = ((size_t)b * N + z) * N * N;
    const VecInfo inf = a.info[b];
    const float* V = a.vpot + (size_t)inf.vrow * NG + (size_t)z * N * N;
    const float* dV = (a.dvpot != nullptr && inf.dvrow >= 0) ? a.dvpot + (size_t)inf.dvrow * NG + (size_t)z * N * N
                                                                 : nullptr;
    const float2* bp = (dV != nullptr) ? a.b1 + ((size_t)inf.partner * N + z) * N * N : nullptr;
    const float2* kc = a.kbc != nullptr ? a.kbc + (size_t)b * a.n_proj : nullptr;
    const int s0 = kc != nullptr ? __ldg(a.plane_off + z) : 0;
    if (kc != nullptr) {
        const int ns = __ldg(a.plane_off + z + 1) - s0;
        for (int i = threadIdx.x; i < 4 * ns; i += NT) kcs[i] = kc[__ldg(a.slot_atom + s0 + i / 4) * 4 + (i & 3)];
    }
    if constexpr (IN_SMEM) {
        fft2_plane<N, NT, +1>(sm, tws);                // the plane is already in shared memory
    } else {
        inv_plane_from_global<N, NT>(sm, a.W + plane, tws);
    }
    if (kc != nullptr) {
        // KB apply, colour by colour: within a colour every point occurs once, so the adds need no
        // atomics and their order at a point (colour order) is fixed
        const int* col = a.kbe_col + z * (a.max_colors + 1);
        for (int c = 0; c < a.max_colors; ++c) {
            const int e0 = __ldg(col + c), e1 = __ldg(col + c + 1);
            if (e0 == e1) break;                  // a plane's colours are used from 0 upwards
#pragma unroll 4
            for (int e = e0 + threadIdx.x; e < e1; e += NT) {
                const unsigned os = __ldg(a.kbe_os + e);
                const float4 be = __ldg(a.kbe_beta + e);
                const int o = (int)(os & 0xffffu), sl = (int)(os >> 16);
                const float4 c01 = *reinterpret_cast<const float4*>(kcs + 4 * sl);
                const float4 c23 = *reinterpret_cast<const float4*>(kcs + 4 * sl + 2);
                float2& hv = sm[(o / N) * P + (o % N)];
                hv.x += be.x * c01.x + be.y * c01.z + be.z * c23.x + be.w * c23.z;
                hv.y += be.x * c01.y + be.y * c01.w + be.z * c23.y + be.w * c23.w;
            }
            __syncthreads();
        }
    }

    const float2 cpsi = a.coef.cpsi[inf.cset], ch = a.coef.ch[inf.cset], c2 = a.coef.c2[inf.cset];
    const float ebar = a.ebar, alpha = a.alpha;
    const bool want_kbp = a.kbp != nullptr;
#pragma unroll 2
    for (int q = threadIdx.x; q < N * N / 2; q += NT) {
        const int y = q / (N / 2), x = 2 * (q % (N / 2));
        const int o = y * N + x;
        float2 h0 = sm[y * P + x], h1 = sm[y * P + x + 1];
        const float4 bb = ld4(a.b1 + plane + o);
        const float2 v = __ldg(reinterpret_cast<const float2*>(V + o));
        h0.x += (v.x - ebar) * bb.x;
        h0.y += (v.x - ebar) * bb.y;
        h1.x += (v.y - ebar) * bb.z;
        h1.y += (v.y - ebar) * bb.w;
        if (dV != nullptr) {
            const float2 d = __ldg(reinterpret_cast<const float2*>(dV + o));
            const float4 pb = ld4(bp + o);
            h0.x += d.x * pb.x;
            h0.y += d.x * pb.y;
            h1.x += d.y * pb.z;
            h1.y += d.y * pb.w;
        }
        float2 o0 = cmul(ch, cscale(h0, alpha)), o1 = cmul(ch, cscale(h1, alpha));
        if (a.psi != nullptr) {
            const float4 pp = ld4(a.psi + plane + o);
            o0 = cadd(o0, cmul(cpsi, make_float2(pp.x, pp.y)));
            o1 = cadd(o1, cmul(cpsi, make_float2(pp.z, pp.w)));
        }
        if (a.b2 != nullptr) {
            const float4 b2 = ld4(a.b2 + plane + o);
            o0 = cadd(o0, cmul(c2, make_float2(b2.x, b2.y)));
            o1 = cadd(o1, cmul(c2, make_float2(b2.z, b2.w)));
        }
        st4(a.out + plane + o, o0, o1);
        sm[y * P + x] = o0;
        sm[y * P + x + 1] = o1;
    }
    if (a.Wout == nullptr) return;
    __syncthreads();
    if (want_kbp) {
        // partial projections of `out` on this plane: one warp per (plane, atom) slot sums the
        // atom's support points in the plane from shared memory, in a fixed order
        const int sb = __ldg(a.plane_off + z), s1 = __ldg(a.plane_off + z + 1);
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        for (int k = sb + warp; k < s1; k += NT / 32) {
            float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            const int e1 = __ldg(a.kbe_slot_end + k);
#pragma unroll 4
            for (int e = __ldg(a.kbe_slot_beg + k) + lane; e < e1; e += 32) {
                const int o = (int)(__ldg(a.kbe_os + e) & 0xffffu);
                const float2 v = sm[(o / N) * P + (o % N)];
                const float4 be = __ldg(a.kbe_beta + e);
                acc[0] += be.x * v.x; acc[1] += be.x * v.y;
                acc[2] += be.y * v.x; acc[3] += be.y * v.y;
                acc[4] += be.z * v.x; acc[5] += be.z * v.y;
                acc[6] += be.w * v.x; acc[7] += be.w * v.y;
            }
            // butterfly reduce-scatter of the 8 sums over the warp (9 shuffles, fixed order): after
            // it, lane l holds the total of accumulator 4 bit4(l) + 2 bit3(l) + bit2(l)
            const float r = warp_reduce_scatter8(acc, lane);
            if ((lane & 3) == 0)
                reinterpret_cast<float*>(a.kbp + ((size_t)b * a.total_slots + k) * 4)[lane >> 2] = r;
        }
    }
    fwd_plane_to_global<N, NT>(sm, a.Wout + plane, tws);
}



template <int N, int NT>
__global__ void __launch_bounds__(NT, (PlaneMinB<N, NT>::value))
k_plane_step(StepArgs a, const float2* __restrict__ tw) {
    extern __shared__ float2 sm[];
    constexpr int P = N + 1;
    const int z = blockIdx.x, b = blockIdx.y;
    // the pointwise operands stream into L2 while the inverse transform runs
    if (threadIdx.x == 0 && (a.pf_operands & 1)) prefetch_operands<N>(a, z, b);
    if (threadIdx.x == 0 && a.pf_ahead > 0) {
        const long nxt = (long)b * N + z + a.pf_ahead;         // linear id of a later block
        if (nxt < (long)gridDim.y * N) l2_prefetch(a.W + (size_t)nxt * N * N, N * N * sizeof(float2));
    }
    // twiddles and the E-weighted projections of b_{k+1} for the atoms of this plane's slots
    // (kcs[slot][4]) next to the plane in shared memory
    float2* stw = sm + N * P;
    float2* kcs = stw + N;
    for (int i = threadIdx.x; i < N; i += NT) stw[i] = __ldg(tw + i);
    plane_step_body<N, NT, false>(a, sm, kcs, TwShared{stw}, z, b);
}

// cp.async of 8 bytes (global -> shared, through L1) and its group controls
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int K> __device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(K) : "memory");
}

// plane (N x N complex, row-major in global memory) -> shared memory with pitch N + 1
template <int N, int NT>
__device__ __forceinline__ void copy_plane_async(float2* dst, const float2* __restrict__ src) {
    constexpr int P = N + 1;
#pragma unroll 4
    for (int q = threadIdx.x; q < N * N; q += NT) cp_async8(dst + (q / N) * P + (q % N), src + q);
}

// Persistent form of the fused step: block i takes the planes t = i, i + gridDim.x, ... (t = b N + z,
// t < total) and double-buffers their W input in shared memory with cp.async, so the next plane's
// input is in flight while the current one is transformed.  Same arithmetic as k_plane_step.
template <int N, int NT>
__global__ void __launch_bounds__(NT, 3)
k_plane_step_pipe(StepArgs a, const float2* __restrict__ tw, int total) {
    extern __shared__ float2 sm[];
    constexpr int P = N + 1;
    float2* stw = sm + 2 * N * P;
    float2* kcs = stw + N;
    for (int i = threadIdx.x; i < N; i += NT) stw[i] = __ldg(tw + i);
    int t = blockIdx.x;
    if (t < total) {
        copy_plane_async<N, NT>(sm, a.W + (size_t)t * N * N);
        if (threadIdx.x == 0 && (a.pf_operands & 1)) prefetch_operands<N>(a, t % N, t / N);
    }
    cp_async_commit();
    for (int it = 0; t < total; ++it, t += gridDim.x) {
        float2* cur = sm + (size_t)(it & 1) * N * P;
        const int tn = t + gridDim.x;
        if (tn < total) {
            copy_plane_async<N, NT>(sm + (size_t)((it + 1) & 1) * N * P, a.W + (size_t)tn * N * N);
            if (threadIdx.x == 0 && (a.pf_operands & 1)) prefetch_operands<N>(a, tn % N, tn / N);
        }
        cp_async_commit();
        cp_async_wait<1>();                 // this plane's group has landed (the newest may be in flight)
        __syncthreads();
        plane_step_body<N, NT, true>(a, cur, kcs, TwShared{stw}, t % N, t / N);
        __syncthreads();                    // cur is refilled two iterations later
    }
    cp_async_wait<0>();
}

// ------------------------------------------------------------------ inverse plane pass
template <int N>
__global__ void __launch_bounds__(Cfg<N>::PLANE_NT, Cfg<N>::PLANE_MINB)
k_plane_inv(const float2* __restrict__ W, const float2* __restrict__ tw, int mode, float2* out_c,
            const float* __restrict__ vloc, float* vtot, float* dv, float* uR, int64_t uR_stride, float* out_re) {
    extern __shared__ float2 sm[];
    constexpr int NT = Cfg<N>::PLANE_NT, P = N + 1;
    constexpr size_t NG = (size_t)N * N * N;
    const int z = blockIdx.x, b = blockIdx.y;
    const size_t plane = ((size_t)b * N + z) * N * N;
    inv_plane_from_global<N, NT>(sm, W + plane, tw);
    if (mode == 0) {
        store_plane<N, NT>(out_c + plane, sm);
        return;
    }
    for (int q = threadIdx.x; q < N * N; q += NT) {
        const int y = q / N, x = q % N;
        const size_t g = (size_t)z * N * N + q;
        const float2 c = sm[y * P + x];
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
// Sample s owns batch vectors [s*2*n_eta, (s+1)*2*n_eta): eta_l then d eta_l.
template <int N>
__global__ void __launch_bounds__(Cfg<N>::PLANE_NT, Cfg<N>::PLANE_MINB)
k_density_fwd(const float2* __restrict__ psi, int n_eta, float weight, float* rho0, int store_rho0,
              float2* __restrict__ Wp, const float2* __restrict__ tw) {
    extern __shared__ float2 sm[];
    constexpr int NT = Cfg<N>::PLANE_NT, P = N + 1;
    constexpr size_t NG = (size_t)N * N * N;
    const int z = blockIdx.x, s = blockIdx.y;
    const size_t zoff = (size_t)z * N * N;
    for (int q = threadIdx.x; q < N * N / 2; q += NT) {
        const int y = q / (N / 2), x = 2 * (q % (N / 2));
        const size_t g = zoff + y * N + x;
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
        sm[y * P + x] = make_float2(r0 - rz[0], d0);
        sm[y * P + x + 1] = make_float2(r1 - rz[1], d1);
    }
    __syncthreads();
    fwd_plane_to_global<N, NT>(sm, Wp + ((size_t)s * N + z) * N * N, tw);
}

// ------------------------------------------------------------------ split-operator passes
// out plane = forward xy transform of e^{-i s V dt/2} x (s = +1 or -1 per vector), V = the vector's
// row of vpot; for a tangent vector (dvpot given, dvrow >= 0) x = psi - i s (dt/2) dv psi_partner,
// the derivative of the half-step along V -> V + lam dv (V and dv are diagonal and commute).
template <int N>
__global__ void __launch_bounds__(Cfg<N>::PLANE_NT, Cfg<N>::PLANE_MINB)
k_plane_fwd_phase(const float2* __restrict__ psi, const float* __restrict__ vpot, const float* __restrict__ dvpot,
                  const VecInfo* __restrict__ info, float dt, float2* __restrict__ W, const float2* __restrict__ tw) {
    extern __shared__ float2 sm[];
    constexpr int NT = Cfg<N>::PLANE_NT, P = N + 1;
    constexpr size_t NG = (size_t)N * N * N;
    const int z = blockIdx.x, b = blockIdx.y;
    const size_t plane = ((size_t)b * N + z) * N * N;
    const VecInfo inf = info[b];
    const float hdt = 0.5f * (inf.cset == 0 ? dt : -dt);
    const float* V = vpot + (size_t)inf.vrow * NG + (size_t)z * N * N;
    const bool tan = dvpot != nullptr && inf.dvrow >= 0;
    const float* dV = tan ? dvpot + (size_t)inf.dvrow * NG + (size_t)z * N * N : nullptr;
    const float2* pp = tan ? psi + ((size_t)inf.partner * N + z) * N * N : nullptr;
#pragma unroll 4
    for (int q = threadIdx.x; q < N * N / 2; q += NT) {
        const int y = q / (N / 2), x = 2 * (q % (N / 2));
        const int o = y * N + x;
        const float4 v = ld4(psi + plane + o);
        float2 a0 = make_float2(v.x, v.y), a1 = make_float2(v.z, v.w);
        if (tan) {
            const float4 pa = ld4(pp + o);
            const float2 d = __ldg(reinterpret_cast<const float2*>(dV + o));
            // a -= i hdt dv p
            a0.x += hdt * d.x * pa.y;
            a0.y -= hdt * d.x * pa.x;
            a1.x += hdt * d.y * pa.w;
            a1.y -= hdt * d.y * pa.z;
        }
        const float2 pv = __ldg(reinterpret_cast<const float2*>(V + o));
        float s0, c0, s1, c1;
        sincosf(pv.x * hdt, &s0, &c0);
        sincosf(pv.y * hdt, &s1, &c1);
        sm[y * P + x] = cmul(a0, make_float2(c0, -s0));
        sm[y * P + x + 1] = cmul(a1, make_float2(c1, -s1));
    }
    __syncthreads();
    fwd_plane_to_global<N, NT>(sm, W + plane, tw);
}

// psi plane = e^{-i s V dt/2} (inverse xy transform of W), V = the vector's row of vpot
template <int N>
__global__ void __launch_bounds__(Cfg<N>::PLANE_NT, Cfg<N>::PLANE_MINB)
k_plane_inv_phase(const float2* __restrict__ W, const float* __restrict__ vpot, const VecInfo* __restrict__ info,
                  float dt, float2* __restrict__ psi, const float2* __restrict__ tw) {
    extern __shared__ float2 sm[];
    constexpr int NT = Cfg<N>::PLANE_NT, P = N + 1;
    constexpr size_t NG = (size_t)N * N * N;
    const int z = blockIdx.x, b = blockIdx.y;
    const size_t plane = ((size_t)b * N + z) * N * N;
    const VecInfo inf = info[b];
    const float hdt = 0.5f * (inf.cset == 0 ? dt : -dt);
    const float* V = vpot + (size_t)inf.vrow * NG + (size_t)z * N * N;
    inv_plane_from_global<N, NT>(sm, W + plane, tw);
#pragma unroll 4
    for (int q = threadIdx.x; q < N * N / 2; q += NT) {
        const int y = q / (N / 2), x = 2 * (q % (N / 2));
        const float2 pv = __ldg(reinterpret_cast<const float2*>(V + y * N + x));
        float s0, c0, s1, c1;
        sincosf(pv.x * hdt, &s0, &c0);
        sincosf(pv.y * hdt, &s1, &c1);
        st4(psi + plane + y * N + x, cmul(sm[y * P + x], make_float2(c0, -s0)),
            cmul(sm[y * P + x + 1], make_float2(c1, -s1)));
    }
}

// Tangent source of the second local half-step: for each tangent vector b (dvrow >= 0),
// psi_b -= i s (dt/2) dv psi_partner, after k_plane_inv_phase has written both vectors.
__global__ void __launch_bounds__(256)
k_split_tangent(float2* __restrict__ psi, const float* __restrict__ dvpot, const VecInfo* __restrict__ info, float dt,
                int64_t ng) {
    const VecInfo inf = info[blockIdx.y];
    if (inf.dvrow < 0) return;
    const float hdt = 0.5f * (inf.cset == 0 ? dt : -dt);
    float4* x = reinterpret_cast<float4*>(psi + (size_t)blockIdx.y * ng);
    const float4* p = reinterpret_cast<const float4*>(psi + (size_t)inf.partner * ng);
    const float2* d = reinterpret_cast<const float2*>(dvpot + (size_t)inf.dvrow * ng);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < ng / 2; i += (int64_t)gridDim.x * blockDim.x) {
        float4 a = x[i];
        const float4 pa = p[i];
        const float2 dv = d[i];
        a.x += hdt * dv.x * pa.y;
        a.y -= hdt * dv.x * pa.x;
        a.z += hdt * dv.y * pa.w;
        a.w -= hdt * dv.y * pa.z;
        x[i] = a;
    }
}

// One colour of the split KB factor: block (i, b) applies e^{-i tau V_a} = 1 + Q_a F_a Q_a^T to
// vector b for atom a = atoms[i]: c = Q_a^T x over the atom's support (fixed-order block sum),
// d = F c with F the 4 x 4 complex factor of the vector's direction, x += Q_a d.  Atoms of one
// colour have disjoint supports, so the blocks of a launch touch disjoint points.
__global__ void __launch_bounds__(256)
k_kb_split(const int* __restrict__ atoms, const int64_t* __restrict__ atom_off, const int* __restrict__ sup_idx,
           const float4* __restrict__ q4, const float2* __restrict__ F /*[n_atoms][2][16]*/,
           const VecInfo* __restrict__ info, float2* __restrict__ x, size_t ng) {
    __shared__ float red[8][8];
    __shared__ float2 d[4];
    const int a = __ldg(atoms + blockIdx.x), b = blockIdx.y;
    const int64_t s0 = __ldg(atom_off + a), s1 = __ldg(atom_off + a + 1);
    float2* v = x + (size_t)b * ng;
    float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    for (int64_t s = s0 + threadIdx.x; s < s1; s += blockDim.x) {
        const float2 p = v[__ldg(sup_idx + s)];
        const float4 q = __ldg(q4 + s);
        acc[0] += q.x * p.x; acc[1] += q.x * p.y;
        acc[2] += q.y * p.x; acc[3] += q.y * p.y;
        acc[4] += q.z * p.x; acc[5] += q.z * p.y;
        acc[6] += q.w * p.x; acc[7] += q.w * p.y;
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        for (int o = 16; o > 0; o >>= 1) acc[i] += __shfl_xor_sync(0xffffffffu, acc[i], o);
        if (lane == 0) red[w][i] = acc[i];
    }
    __syncthreads();
    if (threadIdx.x < 4) {
        const int p = threadIdx.x;
        const float2* f = F + ((size_t)a * 2 + (info[b].cset == 0 ? 0 : 1)) * 16 + p * 4;
        float2 c[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            float re = 0.f, im = 0.f;
            for (int ww = 0; ww < 8; ++ww) {
                re += red[ww][2 * k];
                im += red[ww][2 * k + 1];
            }
            c[k] = make_float2(re, im);
        }
        float2 o = make_float2(0.f, 0.f);
#pragma unroll
        for (int k = 0; k < 4; ++k) o = cadd(o, cmul(__ldg(f + k), c[k]));
        d[p] = o;
    }
    __syncthreads();
    const float2 d0 = d[0], d1 = d[1], d2 = d[2], d3 = d[3];
    for (int64_t s = s0 + threadIdx.x; s < s1; s += blockDim.x) {
        const int g = __ldg(sup_idx + s);
        const float4 q = __ldg(q4 + s);
        float2 p = v[g];
        p.x += q.x * d0.x + q.y * d1.x + q.z * d2.x + q.w * d3.x;
        p.y += q.x * d0.y + q.y * d1.y + q.z * d2.y + q.w * d3.y;
        v[g] = p;
    }
}

// ------------------------------------------------------------------ KB projection
// kbc[b][4a + p] = E_ap * dV * sum_{r in support(a)} beta_ap(r) b1_b(r)
__global__ void __launch_bounds__(256)
k_kb_project(const int64_t* __restrict__ atom_off, const int* __restrict__ sup_idx, const float4* __restrict__ sup_beta,
             const float4* __restrict__ atom_e, const float2* __restrict__ b1, size_t ng, int n_proj, float dV,
             float2* __restrict__ kbc) {
    __shared__ float red[8][8];
    const int at = blockIdx.x, b = blockIdx.y;
    const int64_t s0 = atom_off[at], s1 = atom_off[at + 1];
    const float2* v = b1 + (size_t)b * ng;
    float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    for (int64_t s = s0 + threadIdx.x; s < s1; s += blockDim.x) {
        const float2 p = __ldg(v + __ldg(sup_idx + s));
        const float4 be = __ldg(sup_beta + s);
        acc[0] += be.x * p.x; acc[1] += be.x * p.y;
        acc[2] += be.y * p.x; acc[3] += be.y * p.y;
        acc[4] += be.z * p.x; acc[5] += be.z * p.y;
        acc[6] += be.w * p.x; acc[7] += be.w * p.y;
    }
#pragma unroll
    for (int i = 0; i < 8; ++i)
        for (int o = 16; o > 0; o >>= 1) acc[i] += __shfl_xor_sync(0xffffffffu, acc[i], o);
    const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if ((threadIdx.x & 31) == 0)
        for (int i = 0; i < 8; ++i) red[w][i] = acc[i];
    __syncthreads();
    if (threadIdx.x < 8) {
        float t = 0.f;
        for (int k = 0; k < nw; ++k) t += red[k][threadIdx.x];
        const float4 e = __ldg(atom_e + at);
        const int p = threadIdx.x >> 1;
        const float ep = p == 0 ? e.x : (p == 1 ? e.y : (p == 2 ? e.z : e.w));
        reinterpret_cast<float*>(kbc + (size_t)b * n_proj + at * 4)[threadIdx.x] = ep * dV * t;
    }
}

// kbc[b][4a + p] = E_ap dV sum_{slots of a} kbp[b][slot][p].  One warp per (b, a): lane l takes
// projector p = l % 4 of the atom's slots l / 4, l / 4 + 8, ... (in increasing plane), then the
// eight lanes of each p are summed by a fixed shuffle tree.
__global__ void __launch_bounds__(256)
k_kb_reduce(const int* __restrict__ atom_pos_off, const int* __restrict__ atom_pos, const float4* __restrict__ atom_e,
            const float2* __restrict__ kbp, int n_atoms, int batch, int total_slots, int n_proj, float dV,
            float2* __restrict__ kbc) {
    const int w = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
    if (w >= batch * n_atoms) return;                     // whole warps leave together
    const int a = w % n_atoms, b = w / n_atoms, p = lane & 3;
    const int q0 = __ldg(atom_pos_off + a), q1 = __ldg(atom_pos_off + a + 1);
    const float2* kb = kbp + (size_t)b * total_slots * 4;
    float2 acc = make_float2(0.f, 0.f);
    for (int q = q0 + (lane >> 2); q < q1; q += 8) {
        const float2 v = __ldg(kb + (size_t)__ldg(atom_pos + q) * 4 + p);
        acc.x += v.x;
        acc.y += v.y;
    }
#pragma unroll
    for (int off = 4; off < 32; off <<= 1) {
        acc.x += __shfl_xor_sync(0xffffffffu, acc.x, off);
        acc.y += __shfl_xor_sync(0xffffffffu, acc.y, off);
    }
    if (lane < 4) {
        const float4 e = __ldg(atom_e + a);
        const float ep = (p == 0 ? e.x : (p == 1 ? e.y : (p == 2 ? e.z : e.w))) * dV;
        kbc[(size_t)b * n_proj + a * 4 + p] = make_float2(ep * acc.x, ep * acc.y);
    }
}

void launch_kb_reduce(const KBDev& kb, const float2* kbp, int batch, float dV, float2* kbc, cudaStream_t st) {
    const long warps = (long)batch * kb.n_atoms;
    if (warps == 0) return;
    k_kb_reduce<<<(unsigned)((warps * 32 + 255) / 256), 256, 0, st>>>(kb.atom_pos_off, kb.atom_pos, kb.atom_e, kbp,
                                                                     kb.n_atoms, batch, kb.total_slots, kb.n_proj, dV,
                                                                     kbc);
}

// ------------------------------------------------------------------ launchers
bool grid_supported(int n) { return n == 16 || n == 32 || n == 64 || n == 128 || rows_path(n); }

// SMs of the current device (cached per device)
static int sm_count() {
    static int cache[64] = {0};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) return 1;
    if (cache[dev] == 0) cudaDeviceGetAttribute(&cache[dev], cudaDevAttrMultiProcessorCount, dev);
    return cache[dev] > 0 ? cache[dev] : 1;
}

// Dynamic shared memory of the fused plane step: the plane, the twiddle table and 4
// projections per KB slot
size_t plane_step_smem(int n, int max_plane_slots) {
    if (rows_path(n)) return rows_step_smem(n, max_plane_slots);
    return sizeof(float2) * ((size_t)n * (n + 2) + 4 * (size_t)max_plane_slots);
}

// ... and of its persistent double-buffered form (two planes)
size_t plane_pipe_smem(int n, int max_plane_slots) {
    return sizeof(float2) * (2 * (size_t)n * (n + 1) + n + 4 * (size_t)max_plane_slots);
}

// the persistent form exists up to 64^2 planes (two 128^2 planes do not fit in shared memory)
bool plane_pipe_supported(int n) { return n <= 64 && !rows_path(n); }

template <int N> static cudaError_t set_attrs() {
    cudaError_t e = cudaSuccess;
    const int ps = (int)Cfg<N>::PLANE_SMEM;
    const int mx = (int)cudaSharedmemCarveoutMaxShared;
    if ((e = cudaFuncSetAttribute(k_plane_fwd<N>, cudaFuncAttributePreferredSharedMemoryCarveout, mx))) return e;
    if ((e = cudaFuncSetAttribute(k_plane_step<N, Cfg<N>::PLANE_NT>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                  mx)))
        return e;
    if ((e = cudaFuncSetAttribute(k_plane_step<N, Cfg<N>::PLANE_NT2>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                  mx)))
        return e;
    if ((e = cudaFuncSetAttribute(k_plane_inv<N>, cudaFuncAttributePreferredSharedMemoryCarveout, mx))) return e;
    if ((e = cudaFuncSetAttribute(k_density_fwd<N>, cudaFuncAttributePreferredSharedMemoryCarveout, mx))) return e;
    if ((e = cudaFuncSetAttribute(k_pencil<N, 0>, cudaFuncAttributePreferredSharedMemoryCarveout, mx))) return e;
    if ((e = cudaFuncSetAttribute(k_pencil<N, 1>, cudaFuncAttributePreferredSharedMemoryCarveout, mx))) return e;
    if ((e = cudaFuncSetAttribute(k_pencil<N, 2>, cudaFuncAttributePreferredSharedMemoryCarveout, mx))) return e;
    if ((e = cudaFuncSetAttribute(k_plane_fwd<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, ps))) return e;
    if constexpr (N <= 64) {
        if ((e = cudaFuncSetAttribute(k_plane_step_pipe<N, Cfg<N>::PLANE_NT>,
                                      cudaFuncAttributePreferredSharedMemoryCarveout, mx)))
            return e;
        if ((e = cudaFuncSetAttribute(k_plane_step_pipe<N, Cfg<N>::PLANE_NT>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)plane_pipe_smem(N, 0))))
            return e;
    }
    const int pss = (int)plane_step_smem(N, 0);
    if ((e = cudaFuncSetAttribute(k_plane_step<N, Cfg<N>::PLANE_NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, pss)))
        return e;
    if ((e = cudaFuncSetAttribute(k_plane_step<N, Cfg<N>::PLANE_NT2>, cudaFuncAttributeMaxDynamicSharedMemorySize, pss)))
        return e;
    if ((e = cudaFuncSetAttribute(k_plane_inv<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, ps))) return e;
    if ((e = cudaFuncSetAttribute(k_plane_fwd_phase<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, ps))) return e;
    if ((e = cudaFuncSetAttribute(k_plane_inv_phase<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, ps))) return e;
    if ((e = cudaFuncSetAttribute(k_density_fwd<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, ps))) return e;
    return e;
}

cudaError_t grid_init_attributes(int n) {
    if (rows_path(n)) return rows_init_attributes(n);
    switch (n) {
        case 16: return set_attrs<16>();
        case 32: return set_attrs<32>();
        case 64: return set_attrs<64>();
        case 128: return set_attrs<128>();
    }
    return cudaErrorInvalidValue;
}

#define SGW_DISPATCH_N(n, ...)                          \
    switch (n) {                                        \
        case 16: { constexpr int N = 16; __VA_ARGS__; } break; \
        case 32: { constexpr int N = 32; __VA_ARGS__; } break; \
        case 64: { constexpr int N = 64; __VA_ARGS__; } break; \
        case 128: { constexpr int N = 128; __VA_ARGS__; } break; \
        default: break;                                 \
    }

// Resident CTAs per SM of the two passes of a Chebyshev term (for the launch-order lookahead)
cudaError_t plane_step_reserve_smem(int n, int max_plane_slots) {
    if (rows_path(n)) return rows_step_reserve_smem(n, max_plane_slots);
    cudaError_t e = cudaSuccess;
    const int bytes = (int)plane_step_smem(n, max_plane_slots);
    SGW_DISPATCH_N(n, {
        e = cudaFuncSetAttribute(k_plane_step<N, Cfg<N>::PLANE_NT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 bytes);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_plane_step<N, Cfg<N>::PLANE_NT2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     bytes);
        if constexpr (N <= 64) {
            if (e == cudaSuccess)
                e = cudaFuncSetAttribute(k_plane_step_pipe<N, Cfg<N>::PLANE_NT>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)plane_pipe_smem(N, max_plane_slots));
        }
    });
    return e;
}

int plane_step_blocks_per_sm(int n, int variant, int max_plane_slots) {
    if (rows_path(n)) return rows_step_blocks_per_sm(n, variant, max_plane_slots);
    int r = 0;
    const size_t sm = plane_step_smem(n, max_plane_slots);
    if (variant == 2 && !plane_pipe_supported(n)) variant = 0;
    SGW_DISPATCH_N(n, {
        if (variant == 0)
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&r, k_plane_step<N, Cfg<N>::PLANE_NT>, Cfg<N>::PLANE_NT, sm);
        else if (variant == 1)
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&r, k_plane_step<N, Cfg<N>::PLANE_NT2>, Cfg<N>::PLANE_NT2, sm);
        else if constexpr (N <= 64)
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&r, k_plane_step_pipe<N, Cfg<N>::PLANE_NT>, Cfg<N>::PLANE_NT,
                                                          plane_pipe_smem(N, max_plane_slots));
    });
    return r;
}

int pencil_blocks_per_sm(int n) {
    if (rows_path(n)) return zlines_blocks_per_sm(n);
    int r = 0;
    SGW_DISPATCH_N(n, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&r, k_pencil<N, 0>, Cfg<N>::PENCIL_NT,
                                                                    Cfg<N>::PENCIL_SMEM));
    return r;
}

void launch_plane_fwd(int n, const float2* in, float2* W, int batch, const float2* tw, cudaStream_t st) {
    if (rows_path(n)) return rows_plane_fwd(n, in, W, batch, tw, st);
    SGW_DISPATCH_N(n, k_plane_fwd<N><<<dim3(N, batch), Cfg<N>::PLANE_NT, Cfg<N>::PLANE_SMEM, st>>>(in, W, tw));
}

void launch_pencil(int n, float2* W, int batch, int kind, float kscale, float ecut, const float2* tw, cudaStream_t st,
                   int pf_ahead, const VecInfo* info, float dt, int line_form) {
    if (rows_path(n)) return rows_pencil(n, W, batch, kind, kscale, ecut, tw, st, line_form);
    SGW_DISPATCH_N(n, {
        const dim3 grid((N / Cfg<N>::TX) * N, batch);
        if (kind == 0)
            k_pencil<N, 0><<<grid, Cfg<N>::PENCIL_NT, Cfg<N>::PENCIL_SMEM, st>>>(W, kscale, ecut, tw, pf_ahead, info, dt);
        else if (kind == 1)
            k_pencil<N, 1><<<grid, Cfg<N>::PENCIL_NT, Cfg<N>::PENCIL_SMEM, st>>>(W, kscale, ecut, tw, pf_ahead, info, dt);
        else
            k_pencil<N, 2><<<grid, Cfg<N>::PENCIL_NT, Cfg<N>::PENCIL_SMEM, st>>>(W, kscale, ecut, tw, pf_ahead, info, dt);
    });
}

int pencil_blocks(int n) { return (n / 16) * n; }

void launch_pencil_coulomb_energy(int n, const float2* W, int batch, int per, float kscale, double dvn,
                                  const float2* tw, double* part, double* acc, cudaStream_t st) {
    if (rows_path(n)) {
        rows_zlines_energy(n, W, batch, kscale, tw, part, st);
        if (batch > 0) k_energy_reduce<<<batch / per, 256, 0, st>>>(part, per, pencil_blocks(n), dvn, acc);
        return;
    }
    SGW_DISPATCH_N(n, {
        static_assert(Cfg<N>::TX == 16, "pencil_blocks assumes 16-column tiles");
        const dim3 grid((N / Cfg<N>::TX) * N, batch);
        k_pencil_energy<N><<<grid, Cfg<N>::PENCIL_NT, Cfg<N>::PENCIL_SMEM, st>>>(W, kscale, tw, part);
        k_energy_reduce<<<batch / per, 256, 0, st>>>(part, per, (int)grid.x, dvn, acc);
    });
}

void launch_plane_step(int n, const StepArgs& a, int batch, const float2* tw, cudaStream_t st, int variant,
                       int line_form) {
    if (rows_path(n)) return rows_plane_step(n, a, batch, tw, st, variant, line_form);
    const int slots = a.kbc != nullptr ? a.max_plane_slots : 0;
    const size_t sm = plane_step_smem(n, slots);
    if (variant == 2 && !plane_pipe_supported(n)) variant = 0;
    SGW_DISPATCH_N(n, {
        if (variant == 0) {
            k_plane_step<N, Cfg<N>::PLANE_NT><<<dim3(N, batch), Cfg<N>::PLANE_NT, sm, st>>>(a, tw);
        } else if (variant == 1) {
            k_plane_step<N, Cfg<N>::PLANE_NT2><<<dim3(N, batch), Cfg<N>::PLANE_NT2, sm, st>>>(a, tw);
        } else if constexpr (N <= 64) {
            // one wave of resident blocks, each walking its planes
            const int total = N * batch;
            const int grid = std::min(total, std::max(1, plane_step_blocks_per_sm(n, 2, slots)) * sm_count());
            k_plane_step_pipe<N, Cfg<N>::PLANE_NT><<<grid, Cfg<N>::PLANE_NT, plane_pipe_smem(N, slots), st>>>(a, tw,
                                                                                                            total);
        }
    });
}

void launch_plane_inv(int n, const float2* W, int batch, const float2* tw, int mode, float2* out_c,
                      const float* vloc, float* vtot, float* dv, float* uR, int64_t uR_stride, float* out_re,
                      cudaStream_t st) {
    if (rows_path(n)) return rows_plane_inv(n, W, batch, tw, mode, out_c, vloc, vtot, dv, uR, uR_stride, out_re, st);
    SGW_DISPATCH_N(n, k_plane_inv<N><<<dim3(N, batch), Cfg<N>::PLANE_NT, Cfg<N>::PLANE_SMEM, st>>>(
                              W, tw, mode, out_c, vloc, vtot, dv, uR, uR_stride, out_re));
}

void launch_density_fwd(int n, const float2* psi, int n_samples, int n_eta, float weight, float* rho0,
                        int store_rho0, float2* Wp, const float2* tw, cudaStream_t st) {
    if (rows_path(n)) return rows_density_fwd(n, psi, n_samples, n_eta, weight, rho0, store_rho0, Wp, tw, st);
    SGW_DISPATCH_N(n, k_density_fwd<N><<<dim3(N, n_samples), Cfg<N>::PLANE_NT, Cfg<N>::PLANE_SMEM, st>>>(
                              psi, n_eta, weight, rho0, store_rho0, Wp, tw));
}

void launch_plane_fwd_phase(int n, const float2* psi, const float* vpot, const float* dvpot, const VecInfo* info,
                            float dt, float2* W, int batch, const float2* tw, cudaStream_t st) {
    SGW_DISPATCH_N(n, k_plane_fwd_phase<N><<<dim3(N, batch), Cfg<N>::PLANE_NT, Cfg<N>::PLANE_SMEM, st>>>(
                              psi, vpot, dvpot, info, dt, W, tw));
}

void launch_plane_inv_phase(int n, const float2* W, const float* vpot, const VecInfo* info, float dt, float2* psi,
                            int batch, const float2* tw, cudaStream_t st) {
    SGW_DISPATCH_N(n, k_plane_inv_phase<N><<<dim3(N, batch), Cfg<N>::PLANE_NT, Cfg<N>::PLANE_SMEM, st>>>(
                              W, vpot, info, dt, psi, tw));
}

void launch_split_tangent(float2* psi, const float* dvpot, const VecInfo* info, float dt, int batch, int64_t ng,
                          cudaStream_t st) {
    const unsigned bx = (unsigned)std::min<int64_t>((ng / 2 + 255) / 256, 256);
    k_split_tangent<<<dim3(bx, batch), 256, 0, st>>>(psi, dvpot, info, dt, ng);
}

void launch_kb_split(const int* atoms, int n_atoms_colour, const KBDev& kb, const float4* q4, const float2* F,
                     const VecInfo* info, float2* x, int batch, size_t ng, cudaStream_t st) {
    if (n_atoms_colour == 0 || batch == 0) return;
    k_kb_split<<<dim3(n_atoms_colour, batch), 256, 0, st>>>(atoms, kb.atom_off, kb.sup_idx, q4, F, info, x, ng);
}

void launch_kb_project(int n, const KBDev& kb, const float2* b1, int batch, float dV, float2* kbc, cudaStream_t st) {
    if (kb.n_atoms == 0 || batch == 0) return;
    const size_t ng = (size_t)n * n * n;
    k_kb_project<<<dim3(kb.n_atoms, batch), 256, 0, st>>>(kb.atom_off, kb.sup_idx, kb.sup_beta, kb.atom_e, b1, ng,
                                                         kb.n_proj, dV, kbc);
}

}  // namespace sgw
