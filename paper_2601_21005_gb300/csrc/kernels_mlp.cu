// Learned control variate: features of a sample's random vector, a 4-layer MLP trained and
// evaluated on the GPU (BF16 operands on the tensor cores, FP32 accumulate, FP32 master
// weights and Adam state), and the FP64 standardisation / control-variate rows.
//
// Network: h1 = tanh(x W1 + b1), h2 = tanh(h1 W2 + b2), h3 = tanh(h2 W3 + b3), y = h3 W4 + b4.
// Loss: mean over samples and outputs of (y - t)^2.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/sgw.h"
#include "fft_smem.cuh"
#include "sgw_internal.cuh"

namespace sgw {

// ------------------------------------------------------------------ BF16 tensor-core GEMM
// C[m][n] = sum_k A(m, k) B(k, n),  A(m, k) = TA ? A[k lda + m] : A[m lda + k],
//                                   B(k, n) = TB ? B[n ldb + k] : B[k ldb + n].
// CTA tile 64 x 64, K step 32, 4 warps of 32 x 32 (2 x 4 tiles of mma.m16n8k16).
enum { EPI_STORE = 0, EPI_BIAS_TANH = 1, EPI_BIAS = 2, EPI_DTANH = 3 };

struct GemmEpi {
    int mode;
    const float* bias;      // [N] (EPI_BIAS*)
    float* out;             // [M][ldo] fp32 result (pre-activation for EPI_BIAS_TANH; dZ for EPI_DTANH)
    int ldo;
    __nv_bfloat16* out_bf;  // [M][ldo] bf16 copy of tanh(z) (BIAS_TANH) or of dZ (DTANH); may be null
    const float* zprev;     // [M][ldo] pre-activation whose tanh' multiplies (EPI_DTANH)
};

constexpr int GT = 64, GK = 32, GPAD = 8;

__device__ __forceinline__ uint32_t ld_bf2(const __nv_bfloat16* p) { return *reinterpret_cast<const uint32_t*>(p); }

template <int TA, int TB>
__global__ void __launch_bounds__(128)
k_gemm_bf16(int M, int N, int K, const __nv_bfloat16* __restrict__ A, int lda, const __nv_bfloat16* __restrict__ B,
            int ldb, GemmEpi ep) {
    __shared__ __align__(16) __nv_bfloat16 sA[GT][GK + GPAD];    // [m][k]
    __shared__ __align__(16) __nv_bfloat16 sB[GT][GK + GPAD];    // [n][k] (B transposed)
    const int m0 = blockIdx.y * GT, n0 = blockIdx.x * GT;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
    const int g = lane >> 2, t = lane & 3;
    float acc[2][4][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int jn = 0; jn < 4; ++jn)
#pragma unroll
            for (int r = 0; r < 4; ++r) acc[i][jn][r] = 0.f;
    const __nv_bfloat16 zero = __float2bfloat16(0.f);
    for (int k0 = 0; k0 < K; k0 += GK) {
        for (int e = threadIdx.x; e < GT * GK; e += 128) {
            int mm, kk;
            if (TA) { mm = e % GT; kk = e / GT; } else { kk = e % GK; mm = e / GK; }
            const int gm = m0 + mm, gk = k0 + kk;
            sA[mm][kk] = (gm < M && gk < K) ? (TA ? A[(size_t)gk * lda + gm] : A[(size_t)gm * lda + gk]) : zero;
            int nn, kb;
            if (TB) { kb = e % GK; nn = e / GK; } else { nn = e % GT; kb = e / GT; }
            const int gn = n0 + nn, gk2 = k0 + kb;
            sB[nn][kb] = (gn < N && gk2 < K) ? (TB ? B[(size_t)gn * ldb + gk2] : B[(size_t)gk2 * ldb + gn]) : zero;
        }
        __syncthreads();
#pragma unroll
        for (int ks = 0; ks < GK; ks += 16) {
            uint32_t af[2][4], bfr[4][2];
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                const int r0 = wm + 16 * i + g;
                af[i][0] = ld_bf2(&sA[r0][ks + 2 * t]);
                af[i][1] = ld_bf2(&sA[r0 + 8][ks + 2 * t]);
                af[i][2] = ld_bf2(&sA[r0][ks + 2 * t + 8]);
                af[i][3] = ld_bf2(&sA[r0 + 8][ks + 2 * t + 8]);
            }
#pragma unroll
            for (int jn = 0; jn < 4; ++jn) {
                const int c0 = wn + 8 * jn + g;
                bfr[jn][0] = ld_bf2(&sB[c0][ks + 2 * t]);
                bfr[jn][1] = ld_bf2(&sB[c0][ks + 2 * t + 8]);
            }
#pragma unroll
            for (int i = 0; i < 2; ++i)
#pragma unroll
                for (int jn = 0; jn < 4; ++jn) {
                    float* c = acc[i][jn];
                    asm volatile(
                        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
                        "{%8,%9}, {%0,%1,%2,%3};\n"
                        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
                        : "r"(af[i][0]), "r"(af[i][1]), "r"(af[i][2]), "r"(af[i][3]), "r"(bfr[jn][0]),
                          "r"(bfr[jn][1]));
                }
        }
        __syncthreads();
    }
    // epilogue: c0,c1 at (row g, cols 2t, 2t+1), c2,c3 at (row g + 8, same cols)
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int jn = 0; jn < 4; ++jn)
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const int row = m0 + wm + 16 * i + g + (r >= 2 ? 8 : 0);
                const int col = n0 + wn + 8 * jn + 2 * t + (r & 1);
                if (row >= M || col >= N) continue;
                float v = acc[i][jn][r];
                const size_t o = (size_t)row * ep.ldo + col;
                if (ep.mode == EPI_BIAS_TANH) {
                    v += ep.bias[col];
                    ep.out[o] = v;
                    if (ep.out_bf) ep.out_bf[o] = __float2bfloat16(tanhf(v));
                } else if (ep.mode == EPI_BIAS) {
                    ep.out[o] = v + ep.bias[col];
                } else if (ep.mode == EPI_DTANH) {
                    const float th = tanhf(ep.zprev[o]);
                    v *= 1.f - th * th;
                    ep.out[o] = v;
                    if (ep.out_bf) ep.out_bf[o] = __float2bfloat16(v);
                } else {
                    ep.out[o] = v;
                }
            }
}

static void gemm(int M, int N, int K, int TA, int TB, const __nv_bfloat16* A, int lda, const __nv_bfloat16* B, int ldb,
                 const GemmEpi& ep, cudaStream_t st) {
    const dim3 grid((N + GT - 1) / GT, (M + GT - 1) / GT);
    if (!TA && !TB) k_gemm_bf16<0, 0><<<grid, 128, 0, st>>>(M, N, K, A, lda, B, ldb, ep);
    else if (TA && !TB) k_gemm_bf16<1, 0><<<grid, 128, 0, st>>>(M, N, K, A, lda, B, ldb, ep);
    else if (!TA && TB) k_gemm_bf16<0, 1><<<grid, 128, 0, st>>>(M, N, K, A, lda, B, ldb, ep);
    else k_gemm_bf16<1, 1><<<grid, 128, 0, st>>>(M, N, K, A, lda, B, ldb, ep);
}

// ------------------------------------------------------------------ small MLP kernels
__global__ void k_to_bf16(int64_t n, const float* __restrict__ x, __nv_bfloat16* __restrict__ y) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] = __float2bfloat16(x[i]);
}

// Weighted loss sum_o w_o (y - t)^2 / (M O): dY = 2 w_o (y - t) / (M O) (fp32 and bf16); the loss
// sum is accumulated in FP64.  w == nullptr means all weights 1.
__global__ void k_loss_grad(int64_t n, int O, const float* __restrict__ y, const float* __restrict__ t,
                            const float* __restrict__ w, float scale, float* __restrict__ d,
                            __nv_bfloat16* __restrict__ dbf, double* loss) {
    __shared__ double sh[32];
    double a = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float e = y[i] - t[i];
        const float wo = w ? w[i % O] : 1.f;
        a += (double)wo * e * e;
        d[i] = scale * wo * e;
        dbf[i] = __float2bfloat16(scale * wo * e);
    }
    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = a;
    __syncthreads();
    if (threadIdx.x < 32) {
        double s = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (threadIdx.x == 0) loss[1 + blockIdx.x] = s;      // per-block partial, summed by k_loss_sum
    }
}

// loss[0] = sum of the nb per-block partials loss[1 .. nb] in a fixed order (one warp)
__global__ void k_loss_sum(int nb, double* loss) {
    double s = 0.0;
    for (int i = threadIdx.x; i < nb; i += 32) s += loss[1 + i];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) loss[0] = s;
}

// db[n] = sum_m d[m][n]   (one thread per column, fixed order)
__global__ void k_colsum(int M, int N, const float* __restrict__ d, float* __restrict__ db) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    float s = 0.f;
    for (int m = 0; m < M; ++m) s += d[(size_t)m * N + n];
    db[n] = s;
}

// Adam (Kingma & Ba) on FP32 master weights; writes the BF16 copies of the matrices.
__global__ void k_adam(int64_t n, float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, __nv_bfloat16* __restrict__ wbf, float lr, float b1, float b2, float c1,
                       float c2, float eps) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        const float wi = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
        w[i] = wi;
        if (wbf) wbf[i] = __float2bfloat16(wi);
    }
}

// ------------------------------------------------------------------ features
// feat[s][f]: for wave vector f = (mx, my, mz) of the list, sqrt(4 pi)/|k| dV sum_z W[s][z][my][mx] e^{-2 pi i mz z/n}
// (W = forward xy transform of zeta-bar * phi); real parts, then imaginary parts, then F(0) real.
__global__ void k_cv_gather(int n, const float2* __restrict__ W, int nk, const int4* __restrict__ ks, float kscale,
                            float dV, const float2* __restrict__ tw, float* __restrict__ feat) {
    const int s = blockIdx.x;
    const int nf = 2 * nk + 1;
    const size_t ng = (size_t)n * n * n;
    for (int f = threadIdx.x; f <= nk; f += blockDim.x) {
        const int4 m = f < nk ? ks[f] : make_int4(0, 0, 0, 0);
        const int ix = (m.x % n + n) % n, iy = (m.y % n + n) % n, iz = (m.z % n + n) % n;
        float re = 0.f, im = 0.f;
        for (int z = 0; z < n; ++z) {
            const float2 v = W[(size_t)s * ng + ((size_t)z * n + iy) * n + ix];
            const float2 w = tw[(iz * z) % n];          // e^{-2 pi i mz z / n}
            re += v.x * w.x - v.y * w.y;
            im += v.x * w.y + v.y * w.x;
        }
        if (f < nk) {
            const float k2 = kscale * (float)(m.x * m.x + m.y * m.y + m.z * m.z);
            const float wgt = dV * 3.5449077018110318f / sqrtf(k2);    // sqrt(4 pi)/|k|
            feat[(size_t)s * nf + f] = re * wgt;
            feat[(size_t)s * nf + nk + f] = im * wgt;
        } else {
            feat[(size_t)s * nf + 2 * nk] = re * dV;
        }
    }
}

// feat[s] = [|F_{s,0}(k)|^2 (nk), F_{s,0}(0)^2, sum_{v>=1} |F_{s,v}(k)|^2 (nk), sum_{v>=1} F_{s,v}(0)^2]
// from the per-vector coefficients raw[s][v] = [Re F(k) (nk), Im F(k) (nk), F(0)].
__global__ void k_cv_combine(int n_samples, int nv, int nk, const float* __restrict__ raw, float* __restrict__ feat) {
    const int s = blockIdx.x;
    const int nr = 2 * nk + 1, nf = 2 * (nk + 1);
    for (int f = threadIdx.x; f <= nk; f += blockDim.x) {
        float z = 0.f, e = 0.f;
        for (int v = 0; v < nv; ++v) {
            const float* r = raw + ((size_t)s * nv + v) * nr;
            const float q = f < nk ? r[f] * r[f] + r[nk + f] * r[nk + f] : r[2 * nk] * r[2 * nk];
            if (v == 0) z = q;
            else e += q;
        }
        feat[(size_t)s * nf + f] = z;
        feat[(size_t)s * nf + nk + 1 + f] = e;
    }
}

// float columns standardised in place with FP64 statistics (computed when compute != 0)
__global__ void k_cv_stats_f32(int n, int O, const float* __restrict__ y, double* __restrict__ mu,
                               double* __restrict__ sd) {
    const int o = blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= O) return;
    double m = 0.0;
    for (int i = 0; i < n; ++i) m += y[(size_t)i * O + o];
    m /= n;
    double v = 0.0;
    for (int i = 0; i < n; ++i) {
        const double d = y[(size_t)i * O + o] - m;
        v += d * d;
    }
    v = n > 1 ? v / (n - 1) : 0.0;
    mu[o] = m;
    sd[o] = v > 0.0 ? sqrt(v) : 1.0;
}

__global__ void k_cv_apply_f32(int64_t total, int O, float* __restrict__ y, const double* __restrict__ mu,
                               const double* __restrict__ sd) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int o = (int)(i % O);
        y[i] = (float)(((double)y[i] - mu[o]) / sd[o]);
    }
}

// source s = Re(zeta-bar) * phi as c64, zeta-bar taken with a sample stride
__global__ void k_cv_source(int64_t ng, const float2* __restrict__ zb, int64_t stride, const float* __restrict__ phi,
                            int n_samples, float2* __restrict__ out) {
    const int64_t total = ng * n_samples;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t s = i / ng, g = i % ng;
        out[i] = make_float2(zb[s * stride + g].x * phi[g], 0.f);
    }
}

// ------------------------------------------------------------------ FP64 standardisation and CV rows
// mu[o], sd[o] over n rows of y (double [n][O]); t = (y - mu)/sd in float.
__global__ void k_cv_stats(int n, int O, const double* __restrict__ y, double* __restrict__ mu, double* __restrict__ sd) {
    const int o = blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= O) return;
    double m = 0.0;
    for (int i = 0; i < n; ++i) m += y[(size_t)i * O + o];
    m /= n;
    double v = 0.0;
    for (int i = 0; i < n; ++i) {
        const double d = y[(size_t)i * O + o] - m;
        v += d * d;
    }
    v = n > 1 ? v / (n - 1) : 0.0;
    mu[o] = m;
    sd[o] = v > 0.0 ? sqrt(v) : 1.0;
}

__global__ void k_cv_standardize(int64_t total, int O, const double* __restrict__ y, const double* __restrict__ mu,
                                 const double* __restrict__ sd, float* __restrict__ t) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int o = (int)(i % O);
        t[i] = (float)((y[i] - mu[o]) / sd[o]);
    }
}

// rows[i][o] = mean_j f_c[j][o] + y[i][o] - f_p[i][o], with f = mu + sd * net (FP64).
__global__ void k_cv_rows(int Mc, int n, int O, const float* __restrict__ fc, const float* __restrict__ fp,
                          const double* __restrict__ y, const double* __restrict__ mu, const double* __restrict__ sd,
                          double* __restrict__ rows) {
    const int o = blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= O) return;
    double mc = 0.0;
    for (int j = 0; j < Mc; ++j) mc += mu[o] + sd[o] * (double)fc[(size_t)j * O + o];
    if (Mc > 0) mc /= Mc;
    for (int i = 0; i < n; ++i) {
        const double f = Mc > 0 ? mu[o] + sd[o] * (double)fp[(size_t)i * O + o] : 0.0;
        rows[(size_t)i * O + o] = (Mc > 0 ? mc : 0.0) + y[(size_t)i * O + o] - f;
    }
}

}  // namespace sgw

// ================================================================== host side
namespace sgw {
// ---------------------------------------------------------------- shell sums and the linear part
// out[i][c]: c < S: sum of the zeta-bar features of shell c, c = S: the zeta-bar k = 0 feature,
// then the same for the eta-bar block (S = n_shells); fixed k order, FP64 accumulation.
__global__ void k_cv_shells(int n, int nk, int n_shells, const int* __restrict__ shell_of_k,
                            const float* __restrict__ feat, float* __restrict__ out) {
    const int per = 2 * (n_shells + 1);
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n * per) return;
    const int i = t / per, c = t % per, half = c / (n_shells + 1), sh = c % (n_shells + 1);
    const float* f = feat + (size_t)i * 2 * (nk + 1) + (size_t)half * (nk + 1);
    double acc = 0.0;
    if (sh == n_shells) {
        acc = f[nk];
    } else {
        for (int k = 0; k < nk; ++k)
            if (__ldg(shell_of_k + k) == sh) acc += f[k];
    }
    out[t] = (float)acc;
}

__global__ void k_f32_to_f64(int64_t n, const float* __restrict__ a, double* __restrict__ b) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        b[i] = (double)a[i];
}

// G[a][b] = sum_r xs[r][a] xs[r][b], xs = (x - mu) / sd  (rows in increasing order)
__global__ void k_cv_gram(int n, int p, const double* __restrict__ x, const double* __restrict__ mu,
                          const double* __restrict__ sd, double* __restrict__ G) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= p * p) return;
    const int a = t / p, b = t % p;
    double acc = 0.0;
    for (int r = 0; r < n; ++r)
        acc += ((x[(size_t)r * p + a] - mu[a]) / sd[a]) * ((x[(size_t)r * p + b] - mu[b]) / sd[b]);
    G[t] = acc;
}

// C[a][j] = sum_r xs[r][a] (y[r][j] - ybar[j])
__global__ void k_cv_xty(int n, int p, int o, const double* __restrict__ x, const double* __restrict__ mu,
                         const double* __restrict__ sd, const double* __restrict__ y, const double* __restrict__ ybar,
                         double* __restrict__ C) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= (int64_t)p * o) return;
    const int a = (int)(t / o), j = (int)(t % o);
    double acc = 0.0;
    for (int r = 0; r < n; ++r) acc += ((x[(size_t)r * p + a] - mu[a]) / sd[a]) * (y[(size_t)r * o + j] - ybar[j]);
    C[t] = acc;
}

// Linear model m = [mu p][sd p][ybar o][B p x o]; f(x)_j = ybar_j + sum_a ((x_a - mu_a) / sd_a) B_aj
__device__ __forceinline__ double lin_eval(const double* __restrict__ m, int p, int o, const float* x, int j) {
    const double* mu = m;
    const double* sd = m + p;
    const double* ybar = m + 2 * p;
    const double* B = m + 2 * p + o;
    double acc = ybar[j];
    for (int a = 0; a < p; ++a) acc += (((double)x[a] - mu[a]) / sd[a]) * B[(size_t)a * o + j];
    return acc;
}

// out = f(x), or y - f(x) when y is given
__global__ void k_cv_lin_apply(int n, int p, int o, const double* __restrict__ m, const float* __restrict__ x,
                               const double* __restrict__ y, double* __restrict__ out) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= (int64_t)n * o) return;
    const int i = (int)(t / o), j = (int)(t % o);
    const double f = lin_eval(m, p, o, x + (size_t)i * p, j);
    out[t] = y != nullptr ? y[t] - f : f;
}

// xbar[a] = mean over the m cheap samples of x[.][a] (fixed order)
__global__ void k_cv_lin_mean(int mc, int p, const float* __restrict__ x, double* __restrict__ xbar) {
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= p) return;
    double acc = 0.0;
    for (int r = 0; r < mc; ++r) acc += (double)x[(size_t)r * p + a];
    xbar[a] = acc / mc;
}

// yout[i][j] = y[i][j] - f(x_i)_j + f(xbar)_j  (the mean of a linear f over the cheap samples)
__global__ void k_cv_lin_rows(int n, int p, int o, const double* __restrict__ m, const double* __restrict__ xbar,
                              const float* __restrict__ xp, const double* __restrict__ y, double* __restrict__ yout) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= (int64_t)n * o) return;
    const int i = (int)(t / o), j = (int)(t % o);
    const double* mu = m;
    const double* sd = m + p;
    const double* B = m + 2 * p + o;
    double d = 0.0;     // f(x_i) - f(xbar) = sum_a (x_ia - xbar_a) / sd_a B_aj
    for (int a = 0; a < p; ++a) d += (((double)xp[(size_t)i * p + a] - mu[a]) / sd[a] - (xbar[a] - mu[a]) / sd[a]) *
                                     B[(size_t)a * o + j];
    yout[t] = y[t] - d;
}

void launch_cv_source(int64_t ng, const float2* zb, int64_t stride, const float* phi, int n_samples, float2* out,
                      cudaStream_t st) {
    const int64_t total = ng * n_samples;
    if (total == 0) return;
    const int64_t blocks = std::min<int64_t>((total + 255) / 256, 152 * 32);
    k_cv_source<<<(unsigned)blocks, 256, 0, st>>>(ng, zb, stride, phi, n_samples, out);
}
void launch_cv_gather(int n, const float2* W, int n_samples, int nk, const int4* ks, float kscale, float dV,
                      const float2* tw, float* feat, cudaStream_t st) {
    if (n_samples == 0) return;
    k_cv_gather<<<n_samples, 128, 0, st>>>(n, W, nk, ks, kscale, dV, tw, feat);
}
void launch_cv_combine(int n_samples, int nv, int nk, const float* raw, float* feat, cudaStream_t st) {
    if (n_samples == 0) return;
    k_cv_combine<<<n_samples, 128, 0, st>>>(n_samples, nv, nk, raw, feat);
}
void launch_cv_standardize_f32(int n, int O, float* y, double* mu, double* sd, int compute, cudaStream_t st) {
    if (compute) k_cv_stats_f32<<<(O + 127) / 128, 128, 0, st>>>(n, O, y, mu, sd);
    const int64_t total = (int64_t)n * O;
    if (total == 0) return;
    const int64_t blocks = std::min<int64_t>((total + 255) / 256, 152 * 32);
    k_cv_apply_f32<<<(unsigned)blocks, 256, 0, st>>>(total, O, y, mu, sd);
}
void launch_cv_stats(int n, int O, const double* y, double* mu, double* sd, cudaStream_t st) {
    k_cv_stats<<<(O + 127) / 128, 128, 0, st>>>(n, O, y, mu, sd);
}
void launch_cv_standardize(int64_t total, int O, const double* y, const double* mu, const double* sd, float* t,
                           cudaStream_t st) {
    if (total == 0) return;
    const int64_t blocks = std::min<int64_t>((total + 255) / 256, 152 * 32);
    k_cv_standardize<<<(unsigned)blocks, 256, 0, st>>>(total, O, y, mu, sd, t);
}
void launch_cv_rows(int Mc, int n, int O, const float* fc, const float* fp, const double* y, const double* mu,
                    const double* sd, double* rows, cudaStream_t st) {
    k_cv_rows<<<(O + 127) / 128, 128, 0, st>>>(Mc, n, O, fc, fp, y, mu, sd, rows);
}

void launch_cv_shells(int n, int nk, int n_shells, const int* shell_of_k, const float* feat, float* out, cudaStream_t st) {
    const int total = n * 2 * (n_shells + 1);
    if (total > 0) k_cv_shells<<<(total + 127) / 128, 128, 0, st>>>(n, nk, n_shells, shell_of_k, feat, out);
}

void launch_f32_to_f64(int64_t n, const float* a, double* b, cudaStream_t st) {
    if (n > 0) k_f32_to_f64<<<(unsigned)std::min<int64_t>((n + 255) / 256, 4096), 256, 0, st>>>(n, a, b);
}

void launch_cv_gram(int n, int p, const double* x, const double* mu, const double* sd, double* G, cudaStream_t st) {
    k_cv_gram<<<(p * p + 127) / 128, 128, 0, st>>>(n, p, x, mu, sd, G);
}

void launch_cv_xty(int n, int p, int o, const double* x, const double* mu, const double* sd, const double* y,
                   const double* ybar, double* C, cudaStream_t st) {
    const int64_t total = (int64_t)p * o;
    k_cv_xty<<<(unsigned)((total + 127) / 128), 128, 0, st>>>(n, p, o, x, mu, sd, y, ybar, C);
}

void launch_cv_lin_apply(int n, int p, int o, const double* m, const float* x, const double* y, double* out,
                         cudaStream_t st) {
    const int64_t total = (int64_t)n * o;
    if (total > 0) k_cv_lin_apply<<<(unsigned)((total + 127) / 128), 128, 0, st>>>(n, p, o, m, x, y, out);
}

void launch_cv_lin_rows(int mc, int n, int p, int o, const double* m, const float* xc, const float* xp,
                        const double* y, double* xbar, double* yout, cudaStream_t st) {
    k_cv_lin_mean<<<(p + 63) / 64, 64, 0, st>>>(mc, p, xc, xbar);
    const int64_t total = (int64_t)n * o;
    if (total > 0) k_cv_lin_rows<<<(unsigned)((total + 127) / 128), 128, 0, st>>>(n, p, o, m, xbar, xp, y, yout);
}

}  // namespace sgw

struct sgw_mlp {
    int n_in = 0, width = 0, n_out = 0, max_batch = 0, device = 0;
    cudaStream_t stream = nullptr;
    int dims[5] = {0};
    int64_t woff[4] = {0}, boff[4] = {0}, np = 0;
    float* P = nullptr;            // FP32 master parameters: W1, b1, W2, b2, W3, b3, W4, b4
    float* G = nullptr;            // gradients (same layout)
    float* Ma = nullptr;           // Adam first moments
    float* Va = nullptr;           // Adam second moments
    __nv_bfloat16* Pbf = nullptr;  // BF16 copies (weights used by the GEMMs)
    int step = 0;
    __nv_bfloat16 *Xbf = nullptr, *Abf[3] = {nullptr}, *dYbf = nullptr, *dZbf[2] = {nullptr};
    float *Z[3] = {nullptr}, *Y = nullptr, *dY = nullptr, *dZ[2] = {nullptr};
    double* loss = nullptr;
    float* lw = nullptr;           // per-output loss weights (nullptr: all 1)
    std::string err;
};

namespace {
sgw_status mfail(sgw_mlp* m, sgw_status s, const std::string& msg) {
    if (m) m->err = msg;
    else sgw::set_global_error(msg.c_str());
    return s;
}
#define MCK(call)                                                                                         \
    do {                                                                                                  \
        cudaError_t e_ = (call);                                                                          \
        if (e_ != cudaSuccess) return mfail(m, SGW_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

uint64_t splitmix64(uint64_t& s) {
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

unsigned grid1(int64_t n) { return (unsigned)std::min<int64_t>((n + 255) / 256, 152 * 16); }

sgw_status mlp_forward(sgw_mlp* m, const float* x, int M) {
    cudaStream_t st = m->stream;
    const int H = m->width, I = m->n_in, O = m->n_out;
    sgw::k_to_bf16<<<grid1((int64_t)M * I), 256, 0, st>>>((int64_t)M * I, x, m->Xbf);
    const __nv_bfloat16* in = m->Xbf;
    int K = I;
    for (int l = 0; l < 3; ++l) {
        sgw::GemmEpi ep{sgw::EPI_BIAS_TANH, m->P + m->boff[l], m->Z[l], H, m->Abf[l], nullptr};
        sgw::gemm(M, H, K, 0, 0, in, K, m->Pbf + m->woff[l], H, ep, st);
        in = m->Abf[l];
        K = H;
    }
    sgw::GemmEpi ep{sgw::EPI_BIAS, m->P + m->boff[3], m->Y, O, nullptr, nullptr};
    sgw::gemm(M, O, H, 0, 0, in, H, m->Pbf + m->woff[3], O, ep, st);
    MCK(cudaGetLastError());
    return SGW_OK;
}

sgw_status mlp_backward(sgw_mlp* m, const float* t, int M) {
    cudaStream_t st = m->stream;
    const int H = m->width, I = m->n_in, O = m->n_out;
    const int64_t ny = (int64_t)M * O;
    sgw::k_loss_grad<<<grid1(ny), 256, 0, st>>>(ny, O, m->Y, t, m->lw, 2.0f / (float)ny, m->dY, m->dYbf, m->loss);
    sgw::k_loss_sum<<<1, 32, 0, st>>>((int)grid1(ny), m->loss);
    // layer 4
    {
        sgw::GemmEpi ep{sgw::EPI_STORE, nullptr, m->G + m->woff[3], O, nullptr, nullptr};
        sgw::gemm(H, O, M, 1, 0, m->Abf[2], H, m->dYbf, O, ep, st);
        sgw::k_colsum<<<(O + 127) / 128, 128, 0, st>>>(M, O, m->dY, m->G + m->boff[3]);
        sgw::GemmEpi ed{sgw::EPI_DTANH, nullptr, m->dZ[0], H, m->dZbf[0], m->Z[2]};
        sgw::gemm(M, H, O, 0, 1, m->dYbf, O, m->Pbf + m->woff[3], O, ed, st);
    }
    int cur = 0;
    for (int l = 2; l >= 0; --l) {
        const __nv_bfloat16* a_in = l > 0 ? m->Abf[l - 1] : m->Xbf;
        const int K_in = l > 0 ? H : I;
        sgw::GemmEpi ep{sgw::EPI_STORE, nullptr, m->G + m->woff[l], H, nullptr, nullptr};
        sgw::gemm(K_in, H, M, 1, 0, a_in, K_in, m->dZbf[cur], H, ep, st);
        sgw::k_colsum<<<(H + 127) / 128, 128, 0, st>>>(M, H, m->dZ[cur], m->G + m->boff[l]);
        if (l > 0) {
            sgw::GemmEpi ed{sgw::EPI_DTANH, nullptr, m->dZ[1 - cur], H, m->dZbf[1 - cur], m->Z[l - 1]};
            sgw::gemm(M, H, H, 0, 1, m->dZbf[cur], H, m->Pbf + m->woff[l], H, ed, st);
            cur = 1 - cur;
        }
    }
    MCK(cudaGetLastError());
    return SGW_OK;
}

sgw_status mlp_check(sgw_mlp* m, int M) {
    if (!m) return mfail(nullptr, SGW_EINVAL, "null mlp");
    if (M < 1 || M > m->max_batch) return mfail(m, SGW_EINVAL, "batch out of range (1..max_batch)");
    MCK(cudaSetDevice(m->device));
    return SGW_OK;
}
}  // namespace

extern "C" {

sgw_status sgw_mlp_create(sgw_mlp** out, int n_in, int width, int n_out, int max_batch, uint64_t seed, int device,
                          void* stream) {
    sgw_mlp* m = nullptr;
    if (!out || n_in < 1 || width < 1 || n_out < 1 || max_batch < 1) return mfail(nullptr, SGW_EINVAL, "bad mlp sizes");
    *out = nullptr;
    if (cudaSetDevice(device) != cudaSuccess) return mfail(nullptr, SGW_ECUDA, "cudaSetDevice failed");
    m = new (std::nothrow) sgw_mlp();
    if (!m) return mfail(nullptr, SGW_ENOMEM, "host allocation failed");
    m->n_in = n_in; m->width = width; m->n_out = n_out; m->max_batch = max_batch;
    m->device = device; m->stream = (cudaStream_t)stream;
    const int d[5] = {n_in, width, width, width, n_out};
    int64_t off = 0;
    for (int l = 0; l < 4; ++l) {
        m->woff[l] = off; off += (int64_t)d[l] * d[l + 1];
        m->boff[l] = off; off += d[l + 1];
    }
    for (int l = 0; l < 5; ++l) m->dims[l] = d[l];
    m->np = off;
    const size_t B = max_batch;
    bool ok = cudaMalloc(&m->P, 4 * off) == cudaSuccess && cudaMalloc(&m->G, 4 * off) == cudaSuccess &&
              cudaMalloc(&m->Ma, 4 * off) == cudaSuccess && cudaMalloc(&m->Va, 4 * off) == cudaSuccess &&
              cudaMalloc(&m->Pbf, 2 * off) == cudaSuccess && cudaMalloc(&m->Xbf, 2 * B * n_in) == cudaSuccess &&
              cudaMalloc(&m->Y, 4 * B * n_out) == cudaSuccess && cudaMalloc(&m->dY, 4 * B * n_out) == cudaSuccess &&
              cudaMalloc(&m->dYbf, 2 * B * n_out) == cudaSuccess && cudaMalloc(&m->loss, sizeof(double) * (1 + 152 * 16)) == cudaSuccess;
    for (int l = 0; l < 3 && ok; ++l)
        ok = cudaMalloc(&m->Abf[l], 2 * B * width) == cudaSuccess && cudaMalloc(&m->Z[l], 4 * B * width) == cudaSuccess;
    for (int l = 0; l < 2 && ok; ++l)
        ok = cudaMalloc(&m->dZ[l], 4 * B * width) == cudaSuccess && cudaMalloc(&m->dZbf[l], 2 * B * width) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        sgw_mlp_destroy(m);
        return mfail(nullptr, SGW_ENOMEM, "mlp device allocation failed");
    }
    // uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) weights from splitmix64, zero biases
    std::vector<float> h(off, 0.f);
    uint64_t s = seed;
    for (int l = 0; l < 4; ++l) {
        const double a = 1.0 / std::sqrt((double)d[l]);
        for (int64_t i = 0; i < (int64_t)d[l] * d[l + 1]; ++i) {
            const double u = (double)(splitmix64(s) >> 11) * (1.0 / 9007199254740992.0);
            h[m->woff[l] + i] = (float)(a * (2.0 * u - 1.0));
        }
    }
    sgw_status st = sgw_mlp_set_params(m, h.data(), off);
    if (st != SGW_OK) {
        std::string e = m->err;
        sgw_mlp_destroy(m);
        return mfail(nullptr, st, e);
    }
    *out = m;
    return SGW_OK;
}

void sgw_mlp_destroy(sgw_mlp* m) {
    if (!m) return;
    cudaSetDevice(m->device);
    void* p[] = {m->P, m->G, m->Ma, m->Va, m->Pbf, m->Xbf, m->Y, m->dY, m->dYbf, m->loss, m->lw, m->Abf[0], m->Abf[1],
                 m->Abf[2], m->Z[0], m->Z[1], m->Z[2], m->dZ[0], m->dZ[1], m->dZbf[0], m->dZbf[1]};
    for (void* q : p)
        if (q) cudaFree(q);
    delete m;
}

const char* sgw_mlp_last_error(const sgw_mlp* m) { return m ? m->err.c_str() : sgw_last_error(nullptr); }

int64_t sgw_mlp_param_count(const sgw_mlp* m) { return m ? m->np : 0; }

sgw_status sgw_mlp_set_params(sgw_mlp* m, const float* params_host, int64_t n) {
    if (!m || !params_host || n != m->np) return mfail(m, SGW_EINVAL, "parameter count mismatch");
    MCK(cudaSetDevice(m->device));
    MCK(cudaMemcpy(m->P, params_host, 4 * n, cudaMemcpyHostToDevice));
    MCK(cudaMemset(m->Ma, 0, 4 * n));
    MCK(cudaMemset(m->Va, 0, 4 * n));
    m->step = 0;
    sgw::k_to_bf16<<<grid1(n), 256, 0, m->stream>>>(n, m->P, m->Pbf);
    MCK(cudaGetLastError());
    MCK(cudaStreamSynchronize(m->stream));
    return SGW_OK;
}

sgw_status sgw_mlp_get_params(sgw_mlp* m, float* params_host, int64_t n) {
    if (!m || !params_host || n != m->np) return mfail(m, SGW_EINVAL, "parameter count mismatch");
    MCK(cudaSetDevice(m->device));
    MCK(cudaStreamSynchronize(m->stream));
    MCK(cudaMemcpy(params_host, m->P, 4 * n, cudaMemcpyDeviceToHost));
    return SGW_OK;
}

sgw_status sgw_mlp_set_loss_weights(sgw_mlp* m, const float* w_host, int n_out) {
    if (!m || n_out != m->n_out) return mfail(m, SGW_EINVAL, "loss weights need n_out entries");
    MCK(cudaSetDevice(m->device));
    if (!w_host) {
        if (m->lw) cudaFree(m->lw);
        m->lw = nullptr;
        return SGW_OK;
    }
    if (!m->lw) MCK(cudaMalloc(&m->lw, sizeof(float) * n_out));
    MCK(cudaMemcpy(m->lw, w_host, sizeof(float) * n_out, cudaMemcpyHostToDevice));
    return SGW_OK;
}

sgw_status sgw_mlp_forward(sgw_mlp* m, const float* x_dev, int M, float* y_dev) {
    sgw_status s = mlp_check(m, M);
    if (s) return s;
    if (!x_dev || !y_dev) return mfail(m, SGW_EINVAL, "null pointers");
    if ((s = mlp_forward(m, x_dev, M))) return s;
    MCK(cudaMemcpyAsync(y_dev, m->Y, sizeof(float) * (size_t)M * m->n_out, cudaMemcpyDeviceToDevice, m->stream));
    return SGW_OK;
}

sgw_status sgw_mlp_gradients(sgw_mlp* m, const float* x_dev, const float* t_dev, int M, double* loss_host,
                             float* grads_host) {
    sgw_status s = mlp_check(m, M);
    if (s) return s;
    if (!x_dev || !t_dev) return mfail(m, SGW_EINVAL, "null pointers");
    if ((s = mlp_forward(m, x_dev, M))) return s;
    if ((s = mlp_backward(m, t_dev, M))) return s;
    if (loss_host) {
        double l;
        MCK(cudaMemcpyAsync(&l, m->loss, 8, cudaMemcpyDeviceToHost, m->stream));
        MCK(cudaStreamSynchronize(m->stream));
        *loss_host = l / ((double)M * m->n_out);
    }
    if (grads_host) {
        MCK(cudaStreamSynchronize(m->stream));
        MCK(cudaMemcpy(grads_host, m->G, 4 * m->np, cudaMemcpyDeviceToHost));
    }
    return SGW_OK;
}

sgw_status sgw_mlp_adam_step(sgw_mlp* m, float lr) {
    if (!m) return mfail(nullptr, SGW_EINVAL, "null mlp");
    MCK(cudaSetDevice(m->device));
    m->step += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - (float)std::pow(0.9, m->step), c2 = 1.f - (float)std::pow(0.999, m->step);
    sgw::k_adam<<<grid1(m->np), 256, 0, m->stream>>>(m->np, m->P, m->G, m->Ma, m->Va, m->Pbf, lr, b1, b2, c1, c2,
                                                     1e-8f);
    MCK(cudaGetLastError());
    return SGW_OK;
}

sgw_status sgw_mlp_train_epoch(sgw_mlp* m, const float* x_dev, const float* t_dev, int n_rows, int batch, float lr,
                               double* mean_loss_host) {
    if (!m || !x_dev || !t_dev || n_rows < 1 || batch < 1 || batch > m->max_batch)
        return mfail(m, SGW_EINVAL, "bad training arguments");
    double tot = 0.0;
    for (int r0 = 0; r0 < n_rows; r0 += batch) {
        const int M = std::min(batch, n_rows - r0);
        double l = 0.0;
        sgw_status s = sgw_mlp_gradients(m, x_dev + (size_t)r0 * m->n_in, t_dev + (size_t)r0 * m->n_out, M,
                                          mean_loss_host ? &l : nullptr, nullptr);
        if (s) return s;
        if ((s = sgw_mlp_adam_step(m, lr))) return s;
        tot += l * M;
    }
    if (mean_loss_host) *mean_loss_host = tot / n_rows;
    return SGW_OK;
}

}  // extern "C"
