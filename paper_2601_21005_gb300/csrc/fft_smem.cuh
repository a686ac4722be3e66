// Shared-memory FFT building blocks for sm_103a.
//
// Batched complex FFTs of lines held in shared memory, by Stockham mixed-radix stages
// (radix 8, 4, 3 and 2; Govindaraju et al., "High performance discrete Fourier transforms
// on graphics processors", SC'08).  Each stage reads its butterflies' inputs into
// registers, synchronises, and writes the outputs back to the same buffer, so the
// transform runs in place without a ping-pong buffer.
//
// Stage (radix R, current sub-length Ns) for butterfly j in [0, N/R):
//   k = j mod Ns; v_r = x[j + r N/R] * w^(r k), w = exp(dir 2 pi i / (Ns R));
//   V = DFT_R(v); y[(j div Ns) Ns R + k + q Ns] = V_q.
// dir = -1 is the forward transform (e^{-2 pi i jk/N}), +1 the unnormalised inverse.
#pragma once
#include <cuda_runtime.h>

namespace sgw {

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
// multiply by dir * i  (dir = +-1)
template <int DIR> __device__ __forceinline__ float2 mul_i(float2 a) {
    return DIR > 0 ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}

template <int R, int DIR> struct Dft;

template <int DIR> struct Dft<2, DIR> {
    __device__ __forceinline__ static void run(float2* v) {
        float2 a = v[0], b = v[1];
        v[0] = cadd(a, b);
        v[1] = csub(a, b);
    }
};

template <int DIR> struct Dft<4, DIR> {
    __device__ __forceinline__ static void run(float2* v) {
        float2 s02 = cadd(v[0], v[2]), d02 = csub(v[0], v[2]);
        float2 s13 = cadd(v[1], v[3]), d13 = mul_i<DIR>(csub(v[1], v[3]));
        v[0] = cadd(s02, s13);
        v[2] = csub(s02, s13);
        v[1] = cadd(d02, d13);
        v[3] = csub(d02, d13);
    }
};

template <int DIR> struct Dft<8, DIR> {
    __device__ __forceinline__ static void run(float2* v) {
        // split into even / odd radix-4 transforms, combine with w8^q = exp(dir 2 pi i q / 8)
        float2 e[4] = {v[0], v[2], v[4], v[6]};
        float2 o[4] = {v[1], v[3], v[5], v[7]};
        Dft<4, DIR>::run(e);
        Dft<4, DIR>::run(o);
        const float r = 0.70710678118654752440f;  // 1/sqrt(2)
        // w8^1 = (1 + dir i)/sqrt2, w8^2 = dir i, w8^3 = (-1 + dir i)/sqrt2
        float2 o1 = make_float2(r * (o[1].x - DIR * o[1].y), r * (o[1].y + DIR * o[1].x));
        float2 o2 = mul_i<DIR>(o[2]);
        float2 o3 = make_float2(r * (-o[3].x - DIR * o[3].y), r * (-o[3].y + DIR * o[3].x));
        v[0] = cadd(e[0], o[0]);
        v[4] = csub(e[0], o[0]);
        v[1] = cadd(e[1], o1);
        v[5] = csub(e[1], o1);
        v[2] = cadd(e[2], o2);
        v[6] = csub(e[2], o2);
        v[3] = cadd(e[3], o3);
        v[7] = csub(e[3], o3);
    }
};

template <int DIR> struct Dft<3, DIR> {
    __device__ __forceinline__ static void run(float2* v) {
        // X_q = sum_r v_r w^(r q), w = exp(dir 2 pi i / 3) = -1/2 + dir i sqrt(3)/2:
        // X_0 = v0 + s, X_1,2 = v0 - s/2 +- dir i (sqrt(3)/2) d with s = v1 + v2, d = v1 - v2
        const float h = 0.86602540378443864676f;  // sqrt(3)/2
        const float2 s = cadd(v[1], v[2]);
        const float2 d = cscale(mul_i<DIR>(csub(v[1], v[2])), h);
        const float2 t = make_float2(v[0].x - 0.5f * s.x, v[0].y - 0.5f * s.y);
        v[0] = cadd(v[0], s);
        v[1] = cadd(t, d);
        v[2] = csub(t, d);
    }
};

// Twiddle table access: a plain pointer is a global table read through the read-only path;
// TwShared wraps a copy of the table in shared memory.
struct TwShared {
    const float2* p;
};
__device__ __forceinline__ float2 tw_at(const float2* __restrict__ t, int i) { return __ldg(t + i); }
__device__ __forceinline__ float2 tw_at(TwShared t, int i) { return t.p[i]; }

// Radix of the next stage given the remaining length: 8 while possible, except that
// 16 splits as 4 x 4 (fewer registers, same passes); then 4, 2, and 3 for the odd factors.
template <int REM> struct NextRadix {
    static constexpr int value =
        (REM == 16) ? 4 : (REM % 8 == 0 ? 8 : (REM % 4 == 0 ? 4 : (REM % 2 == 0 ? 2 : 3)));
    static_assert(REM % value == 0, "lengths must be of the form 2^a 3^b");
};

// One Stockham stage over NL lines.  Element e of line l is at s[l*LS + e*ES].
// Consecutive threads take consecutive lines (conflict-free for the layouts used here).
// tw: table exp(-2 pi i m / N), m < N (read through the read-only cache).
template <int N, int R, int NS, int NL, int LS, int ES, int NT, int DIR, class TW>
__device__ __forceinline__ void fft_stage(float2* s, TW tw) {
    constexpr int NB = N / R;
    constexpr int TOT = NL * NB;
    constexpr int PER = (TOT + NT - 1) / NT;
    constexpr int TWS = N / (NS * R);
    float2 v[PER][R];
#pragma unroll
    for (int p = 0; p < PER; ++p) {
        const int b = threadIdx.x + p * NT;
        if (TOT % NT == 0 || b < TOT) {
            const int l = b % NL, j = b / NL;
#pragma unroll
            for (int r = 0; r < R; ++r) v[p][r] = s[l * LS + (j + r * NB) * ES];
        }
    }
    __syncthreads();
#pragma unroll
    for (int p = 0; p < PER; ++p) {
        const int b = threadIdx.x + p * NT;
        if (TOT % NT == 0 || b < TOT) {
            const int l = b % NL, j = b / NL;
            const int k = j % NS;
            if (NS > 1) {
#pragma unroll
                for (int r = 1; r < R; ++r) {
                    float2 w = tw_at(tw, r * k * TWS);
                    if (DIR > 0) w.y = -w.y;
                    v[p][r] = cmul(v[p][r], w);
                }
            }
            Dft<R, DIR>::run(v[p]);
            const int base = (j / NS) * NS * R + k;
#pragma unroll
            for (int q = 0; q < R; ++q) s[l * LS + (base + q * NS) * ES] = v[p][q];
        }
    }
    __syncthreads();
}

template <int N, int NS, int NL, int LS, int ES, int NT, int DIR, class TW>
__device__ __forceinline__ void fft_rec(float2* s, TW tw) {
    if constexpr (NS < N) {
        constexpr int R = NextRadix<N / NS>::value;
        fft_stage<N, R, NS, NL, LS, ES, NT, DIR>(s, tw);
        fft_rec<N, NS * R, NL, LS, ES, NT, DIR>(s, tw);
    }
}

// Stages with sub-length NS in [NS, NSTOP)
template <int N, int NS, int NSTOP, int NL, int LS, int ES, int NT, int DIR, class TW>
__device__ __forceinline__ void fft_rec_until(float2* s, TW tw) {
    if constexpr (NS < NSTOP) {
        constexpr int R = NextRadix<N / NS>::value;
        fft_stage<N, R, NS, NL, LS, ES, NT, DIR>(s, tw);
        fft_rec_until<N, NS * R, NSTOP, NL, LS, ES, NT, DIR, TW>(s, tw);
    }
}

// NL independent N-point FFTs (N = 2^a 3^b, 2..4096) in shared memory.  Twiddle index
// r k TWS < N in every stage (r < R, k < NS, TWS = N / (NS R)).
// Caller must __syncthreads() before (data ready); returns after a barrier.
template <int N, int NL, int LS, int ES, int NT, int DIR, class TW>
__device__ __forceinline__ void fft_lines(float2* s, TW tw) {
    fft_rec<N, 1, NL, LS, ES, NT, DIR>(s, tw);
}

// ---------------------------------------------------------------- register-ended stages
// The first Stockham stage (NS = 1) of butterfly j reads elements j + r N/R, and the last
// stage (NS = N/R) of butterfly j writes elements j + q N/R.  So the inputs of the first stage
// can be loaded straight from global memory into registers, the outputs of the last stage can
// be stored straight from registers, and a forward transform whose last radix equals the first
// radix of the inverse (reversed plan) can hand its outputs to the inverse in registers.
// Butterfly b = threadIdx.x + p NT of a stage maps to line l = b % NL, index j = b / NL.

// Stage with inputs in registers v[p][r] (= x[l][j + r N/R] before twiddles), outputs to smem.
template <int N, int R, int NS, int NL, int LS, int ES, int NT, int DIR, int PER, class TW>
__device__ __forceinline__ void stage_r2s(float2 (&v)[PER][R], float2* s, TW tw) {
    constexpr int NB = N / R;
    constexpr int TOT = NL * NB;
    constexpr int TWS = N / (NS * R);
    static_assert(PER * NT >= TOT, "register array too small");
#pragma unroll
    for (int p = 0; p < PER; ++p) {
        const int b = threadIdx.x + p * NT;
        if (TOT % NT == 0 || b < TOT) {
            const int l = b % NL, j = b / NL;
            const int k = j % NS;
            if (NS > 1) {
#pragma unroll
                for (int r = 1; r < R; ++r) {
                    float2 w = tw_at(tw, r * k * TWS);
                    if (DIR > 0) w.y = -w.y;
                    v[p][r] = cmul(v[p][r], w);
                }
            }
            Dft<R, DIR>::run(v[p]);
            const int base = (j / NS) * NS * R + k;
#pragma unroll
            for (int q = 0; q < R; ++q) s[l * LS + (base + q * NS) * ES] = v[p][q];
        }
    }
    __syncthreads();
}

// Last stage (NS * R == N) with inputs from smem and outputs kept in registers:
// v[p][q] = y[l][j + q NS].  Ends with a barrier so that smem may be overwritten.
template <int N, int R, int NS, int NL, int LS, int ES, int NT, int DIR, int PER, class TW>
__device__ __forceinline__ void stage_s2r(const float2* s, float2 (&v)[PER][R], TW tw) {
    constexpr int NB = N / R;
    constexpr int TOT = NL * NB;
    constexpr int TWS = N / (NS * R);
    static_assert(NS * R == N, "stage_s2r is the last stage");
    static_assert(PER * NT >= TOT, "register array too small");
#pragma unroll
    for (int p = 0; p < PER; ++p) {
        const int b = threadIdx.x + p * NT;
        if (TOT % NT == 0 || b < TOT) {
            const int l = b % NL, j = b / NL;
            const int k = j;   // j < NS
#pragma unroll
            for (int r = 0; r < R; ++r) v[p][r] = s[l * LS + (j + r * NB) * ES];
            if (NS > 1) {
#pragma unroll
                for (int r = 1; r < R; ++r) {
                    float2 w = tw_at(tw, r * k * TWS);
                    if (DIR > 0) w.y = -w.y;
                    v[p][r] = cmul(v[p][r], w);
                }
            }
            Dft<R, DIR>::run(v[p]);
        }
    }
    __syncthreads();
}

}  // namespace sgw
