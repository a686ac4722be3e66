// Non-FFT kernels of the sGW hot path: Philox white noise, the TDH kick, power-iteration
// reductions, the Sigma(t) reductions (Eq. 5), time ordering of u^R (FFT over t), the
// damped transform (Eq. 7) and the QP root (Eq. 6).
#include <cmath>
#include <mutex>
#include <string>

#include "../../include/sgw.h"
#include "fft_smem.cuh"
#include "sgw_internal.cuh"

namespace sgw {

// ------------------------------------------------------------------ Philox4x32-10
// Written from the published definition (Salmon et al., SC'11): per round
// (c0,c1,c2,c3) <- (hi(M1 c2) ^ c1 ^ k0, lo(M1 c2), hi(M0 c0) ^ c3 ^ k1, lo(M0 c0)),
// key bumped by the Weyl constants between rounds.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u, W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += W0;
            k1 += W1;
        }
        const uint32_t hi0 = __umulhi(M0, c.x), lo0 = M0 * c.x;
        const uint32_t hi1 = __umulhi(M1, c.z), lo1 = M1 * c.z;
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    }
    return c;
}

__global__ void k_noise(int64_t ng, int64_t nblk, uint32_t k0, uint32_t k1, uint32_t stream_id, int sample0, int n_vec,
                        int64_t total, float amp, float2* __restrict__ out) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t blk = t % nblk;
        const int64_t sv = t / nblk;
        const int v = (int)(sv % n_vec);
        const int s = (int)(sv / n_vec);
        const uint4 w = philox4x32_10(make_uint4((uint32_t)blk, (uint32_t)v, (uint32_t)(sample0 + s), stream_id), k0, k1);
        const uint32_t ws[4] = {w.x, w.y, w.z, w.w};
        float2* o = out + sv * ng;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int64_t g = blk * 4 + u;
            if (g < ng) o[g] = make_float2((ws[u] >> 31) ? -amp : amp, 0.f);
        }
    }
}

void launch_noise(int ng, uint64_t seed, uint32_t stream_id, int sample0, int n_samples, int n_vec, float amp,
                  float2* out, cudaStream_t st) {
    const int64_t nblk = (ng + 3) / 4;
    const int64_t total = nblk * n_samples * n_vec;
    if (total == 0) return;
    const int threads = 256;
    const int64_t blocks = std::min<int64_t>((total + threads - 1) / threads, 152 * 32);
    k_noise<<<(unsigned)blocks, threads, 0, st>>>(ng, nblk, (uint32_t)(seed & 0xFFFFFFFFu), (uint32_t)(seed >> 32),
                                                  stream_id, sample0, n_vec, total, amp, out);
}

// ------------------------------------------------------------------ small elementwise kernels
__global__ void k_real_to_c64(int64_t count, const float* __restrict__ in, float2* __restrict__ out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = make_float2(in[i], 0.f);
}

void launch_real_to_c64(int64_t count, const float* in, float2* out, cudaStream_t st) {
    if (count == 0) return;
    const int64_t blocks = std::min<int64_t>((count + 255) / 256, 152 * 32);
    k_real_to_c64<<<(unsigned)blocks, 256, 0, st>>>(count, in, out);
}

// psi[s][l] = eta[s][l];  psi[s][n_eta + l] = -i v_p[s] eta[s][l]   (derivative of e^{-i lam v_p} eta)
__global__ void k_kick(int64_t ng, const float2* __restrict__ eta, const float* __restrict__ vp, int n_samples, int n_eta,
                       float2* __restrict__ psi) {
    const int64_t total = ng * n_samples * n_eta;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t g = i % ng;
        const int64_t sl = i / ng;
        const int64_t s = sl / n_eta, l = sl % n_eta;
        const float2 e = eta[i];
        const float v = vp[s * ng + g];
        psi[(s * 2 * n_eta + l) * ng + g] = e;
        psi[(s * 2 * n_eta + n_eta + l) * ng + g] = make_float2(v * e.y, -v * e.x);
    }
}

void launch_kick(int ng, const float2* eta, const float* vp, int n_samples, int n_eta, float2* psi, cudaStream_t st) {
    const int64_t total = (int64_t)ng * n_samples * n_eta;
    if (total == 0) return;
    const int64_t blocks = std::min<int64_t>((total + 255) / 256, 152 * 32);
    k_kick<<<(unsigned)blocks, 256, 0, st>>>(ng, eta, vp, n_samples, n_eta, psi);
}

// out[i] = phi[i mod ng] * eta[i]
__global__ void k_scale_mul(int64_t count, const float* __restrict__ phi, int64_t ng, const float2* __restrict__ eta,
                            float2* __restrict__ out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
        const float f = phi[i % ng];
        const float2 e = eta[i];
        out[i] = make_float2(f * e.x, f * e.y);
    }
}

void launch_scale_mul(int64_t count, const float* phi, int ng, const float2* eta, float2* out, cudaStream_t st) {
    if (count == 0) return;
    const int64_t blocks = std::min<int64_t>((count + 255) / 256, 152 * 32);
    k_scale_mul<<<(unsigned)blocks, 256, 0, st>>>(count, phi, ng, eta, out);
}

// Split one filtered batch per sample (vector 0 = zeta, 1..n_eta = eta_l):
//   eta[s][l] = filt[s][1 + l]; zeta[s] = (zeta_occ = filt[s][0], zeta_unocc = noise[s][0] - filt[s][0]);
//   source[s] = Re noise[s][0] * phi   (the source zeta-bar phi of the TDH kick).
__global__ void k_prepare(int64_t ng, const float2* __restrict__ noise, const float2* __restrict__ filt,
                          const float* __restrict__ phi, int n_samples, int n_eta, float2* __restrict__ eta,
                          float2* __restrict__ zeta, float* __restrict__ source) {
    const int64_t per = (int64_t)(n_eta + 1) * ng;
    const int64_t total = per * n_samples;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t s = i / per, r = i % per;
        const int64_t v = r / ng, g = r % ng;
        const float2 f = filt[i];
        if (v == 0) {
            const float2 z = noise[i];
            zeta[(2 * s) * ng + g] = f;
            zeta[(2 * s + 1) * ng + g] = make_float2(z.x - f.x, z.y - f.y);
            source[s * ng + g] = z.x * phi[g];
        } else {
            eta[(s * n_eta + v - 1) * ng + g] = f;
        }
    }
}

void launch_prepare(int ng, const float2* noise, const float2* filt, const float* phi, int n_samples, int n_eta,
                    float2* eta, float2* zeta, float* source, cudaStream_t st) {
    const int64_t total = (int64_t)ng * (n_eta + 1) * n_samples;
    if (total == 0) return;
    const int64_t blocks = std::min<int64_t>((total + 255) / 256, 152 * 32);
    k_prepare<<<(unsigned)blocks, 256, 0, st>>>(ng, noise, filt, phi, n_samples, n_eta, eta, zeta, source);
}

// ------------------------------------------------------------------ block reductions
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV], double* sh /*[32*NV]*/) {
#pragma unroll
    for (int i = 0; i < NV; ++i)
        for (int o = 16; o > 0; o >>= 1) v[i] += __shfl_xor_sync(0xffffffffu, v[i], o);
    const int w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    if ((threadIdx.x & 31) == 0)
        for (int i = 0; i < NV; ++i) sh[w * NV + i] = v[i];
    __syncthreads();
    if (threadIdx.x < 32) {
        for (int i = 0; i < NV; ++i) {
            double t = threadIdx.x < nw ? sh[threadIdx.x * NV + i] : 0.0;
            for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
            v[i] = t;
        }
    }
}

template <int NV>
__device__ __forceinline__ void block_sumf(float (&v)[NV], float* sh /*[32*NV]*/) {
#pragma unroll
    for (int i = 0; i < NV; ++i)
        for (int o = 16; o > 0; o >>= 1) v[i] += __shfl_xor_sync(0xffffffffu, v[i], o);
    const int w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    if ((threadIdx.x & 31) == 0)
        for (int i = 0; i < NV; ++i) sh[w * NV + i] = v[i];
    __syncthreads();
    if (threadIdx.x < 32) {
        for (int i = 0; i < NV; ++i) {
            float t = threadIdx.x < nw ? sh[threadIdx.x * NV + i] : 0.f;
            for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
            v[i] = t;
        }
    }
}

// ------------------------------------------------------------------ power iteration (Sec. 2.1)
// scal[0] = Re <v|w>/dV, scal[1] = <w|w>/dV, scal[2] = <v|v>/dV  (the dV factors cancel).  One
// block, so that the sums have a fixed order (the iteration runs once per setup).
__global__ void __launch_bounds__(1024) k_dot2(int64_t ng, const float2* __restrict__ v, const float2* __restrict__ w,
                                               double* scal) {
    __shared__ double sh[32 * 3];
    double a[3] = {0.0, 0.0, 0.0};
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < ng; i += (int64_t)gridDim.x * blockDim.x) {
        const float2 x = v[i], y = w[i];
        a[0] += (double)x.x * y.x + (double)x.y * y.y;
        a[1] += (double)y.x * y.x + (double)y.y * y.y;
        a[2] += (double)x.x * x.x + (double)x.y * x.y;
    }
    block_sum<3>(a, sh);
    if (threadIdx.x == 0) {
        scal[0] = a[0];
        scal[1] = a[1];
        scal[2] = a[2];
    }
}

void launch_dot2(int ng, const float2* v, const float2* w, double* scal, cudaStream_t st) {
    k_dot2<<<1, 1024, 0, st>>>(ng, v, w, scal);
}

// With sigma = *shift (0 if null): est = (S0 - sigma S2)/S2 (Rayleigh quotient of A = H - sigma);
// v <- (w - sigma v) / |w - sigma v|.
__global__ void k_power_update(int64_t ng, const float2* __restrict__ w, float2* __restrict__ v,
                               const double* __restrict__ scal, double* est_out, const double* shift) {
    const double sig = shift ? *shift : 0.0;
    const double s0 = scal[0], s1 = scal[1], s2 = scal[2];
    const double nrm2 = s1 - 2.0 * sig * s0 + sig * sig * s2;
    const float inv = (float)(1.0 / sqrt(nrm2));
    const float sg = (float)sig;
    if (blockIdx.x == 0 && threadIdx.x == 0 && est_out) *est_out = (s0 - sig * s2) / s2;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < ng; i += (int64_t)gridDim.x * blockDim.x) {
        const float2 a = w[i], b = v[i];
        v[i] = make_float2((a.x - sg * b.x) * inv, (a.y - sg * b.y) * inv);
    }
}

void launch_power_update(int ng, const float2* w, float2* v, const double* scal, double* est_out, const double* shift,
                         float /*dV*/, cudaStream_t st) {
    const int blocks = std::min<int>((ng + 255) / 256, 152 * 4);
    k_power_update<<<blocks, 256, 0, st>>>(ng, w, v, scal, est_out, shift);
}

// ------------------------------------------------------------------ Sigma(t) accumulation (Eq. 5)
// zeta: [n_samples][2] (occ, unocc).  partial[((s*(n_steps+1) + j)*2 + pm) * nblk + blk]:
// pm = 0: sum phi zeta_unocc u ; pm = 1: sum phi zeta_occ u.
template <typename T>
__global__ void __launch_bounds__(256)
k_sigma_accum(int64_t ng, const float2* __restrict__ zeta, const float* __restrict__ phi, const float2* __restrict__ u,
              int64_t u_ss, int j, int n_steps, double2* __restrict__ partial) {
    __shared__ T sh[32 * 4];
    const int s = blockIdx.y;
    const float2* zo = zeta + (size_t)(2 * s) * ng;
    const float2* zu = zeta + (size_t)(2 * s + 1) * ng;
    const float2* uj = u + (size_t)s * u_ss + (size_t)j * ng;
    T a[4] = {0, 0, 0, 0};
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < ng; i += (int64_t)gridDim.x * blockDim.x) {
        const float f = phi[i];
        const float2 uu = uj[i];
        const float2 p = zu[i], m = zo[i];
        // f * zeta * u  (complex product, no conjugation)
        const T ur = (T)uu.x * f, ui = (T)uu.y * f;
        a[0] += (T)p.x * ur - (T)p.y * ui;
        a[1] += (T)p.x * ui + (T)p.y * ur;
        a[2] += (T)m.x * ur - (T)m.y * ui;
        a[3] += (T)m.x * ui + (T)m.y * ur;
    }
    if constexpr (sizeof(T) == 8) block_sum<4>(a, sh);
    else block_sumf<4>(a, sh);
    if (threadIdx.x == 0) {
        const size_t base = ((size_t)s * (n_steps + 1) + j) * 2;
        partial[(base + 0) * gridDim.x + blockIdx.x] = make_double2((double)a[0], (double)a[1]);
        partial[(base + 1) * gridDim.x + blockIdx.x] = make_double2((double)a[2], (double)a[3]);
    }
}

void launch_sigma_accum(int ng, const float2* zeta, const float* phi, const float2* u, int n_samples,
                        int64_t u_sample_stride, int j, int n_steps, float /*dV*/, int fp64, double2* partial, int nblk,
                        cudaStream_t st) {
    const dim3 grid(nblk, n_samples);
    if (fp64)
        k_sigma_accum<double><<<grid, 256, 0, st>>>(ng, zeta, phi, u, u_sample_stride, j, n_steps, partial);
    else
        k_sigma_accum<float><<<grid, 256, 0, st>>>(ng, zeta, phi, u, u_sample_stride, j, n_steps, partial);
}

// ------------------------------------------------------------------ xi compression (Sec. 2.3)
// Draw k of xi_m of sample `sample`: Philox counter (k, m, sample, stream): segment p = floor(w0
// n_seg / 2^32) (the L points from L p), sign of point l = bit l of w1 (set -> -1).
__device__ __forceinline__ void xi_draw(uint32_t k, uint32_t m, uint32_t sample, uint32_t stream, uint32_t k0,
                                        uint32_t k1, uint32_t n_seg, uint32_t* pos, uint32_t* signs) {
    const uint4 w = philox4x32_10(make_uint4(k, m, sample, stream), k0, k1);
    *pos = (uint32_t)(((uint64_t)w.x * n_seg) >> 32);
    *signs = w.y;
}

// U[s][m] (row stride u_ss per sample) = c dV sum_r xi_m(r) f_s(r) for real rows f_s (stride f_ss):
// one warp per (m, s), lane l < L on point l of each draw; warp sums in a fixed order.
__global__ void __launch_bounds__(256)
k_xi_project(const float* __restrict__ f, int64_t f_ss, int n_samples, int n_xi, int K, int L, uint32_t n_seg,
             uint32_t k0, uint32_t k1, uint32_t stream, int sample0, float cdv, float* __restrict__ U, int64_t u_ss) {
    const int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= (int64_t)n_xi * n_samples) return;
    const int m = (int)(w % n_xi), s = (int)(w / n_xi);
    const float* fs = f + (size_t)s * f_ss;
    float acc = 0.f;
    for (int kb = 0; kb < K; kb += 32) {
        // lane i draws segment kb + i once; the warp walks the draws in order through shuffles
        uint32_t pl = 0, sgl = 0;
        if (kb + lane < K) xi_draw((uint32_t)(kb + lane), (uint32_t)m, (uint32_t)(sample0 + s), stream, k0, k1, n_seg, &pl, &sgl);
        const int kn = min(32, K - kb);
        for (int i = 0; i < kn; ++i) {
            const uint32_t p = __shfl_sync(0xffffffffu, pl, i), sg = __shfl_sync(0xffffffffu, sgl, i);
            if (lane < L) {
                const float v = fs[(size_t)p * L + lane];
                acc += ((sg >> lane) & 1u) ? -v : v;
            }
        }
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) U[(size_t)s * u_ss + m] = cdv * acc;
}

void launch_xi_project(const float* f, int64_t f_ss, int n_samples, int n_xi, int K, int L, int64_t ng, uint64_t seed,
                       uint32_t stream, int sample0, float cdv, float* U, int64_t u_ss, cudaStream_t st) {
    const int64_t warps = (int64_t)n_xi * n_samples;
    if (warps == 0) return;
    k_xi_project<<<(unsigned)((warps * 32 + 255) / 256), 256, 0, st>>>(
        f, f_ss, n_samples, n_xi, K, L, (uint32_t)(ng / L), (uint32_t)(seed & 0xFFFFFFFFu), (uint32_t)(seed >> 32),
        stream, sample0, cdv, U, u_ss);
}

// Sigma accumulation in the xi basis: partial sums of sum_m U_m(j) c sum_r xi_m(r)... written as
// sum_m U_m(j) [c sum_k sum_l sign phi zeta] for zeta_unocc (pm 0) and zeta_occ (pm 1), same partial
// layout as k_sigma_accum (the dV and the signs of Sigma(-t) are applied by k_sigma_reduce).
// Block b of sample s takes xi functions m = warp index + b * warps_per_block, strided by the grid.
template <typename T>
__global__ void __launch_bounds__(256)
k_sigma_accum_xi(const float2* __restrict__ zeta, const float* __restrict__ phi, const float2* __restrict__ Uxi,
                 int64_t u_ss, int j, int n_steps, int n_xi, int K, int L, uint32_t n_seg, uint32_t k0, uint32_t k1,
                 uint32_t stream, int sample0, float c, int64_t ng, double2* __restrict__ partial) {
    __shared__ T sh[32 * 4];
    const int s = blockIdx.y;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, wpb = blockDim.x >> 5;
    const float2* zo = zeta + (size_t)(2 * s) * ng;
    const float2* zu = zeta + (size_t)(2 * s + 1) * ng;
    const float2* Uj = Uxi + (size_t)s * u_ss + (size_t)j * n_xi;
    T a[4] = {0, 0, 0, 0};
    for (int m = blockIdx.x * wpb + wib; m < n_xi; m += gridDim.x * wpb) {
        float b[4] = {0.f, 0.f, 0.f, 0.f};     // sum over the support of sign phi zeta_unocc / zeta_occ
        for (int kb = 0; kb < K; kb += 32) {
            uint32_t pl = 0, sgl = 0;
            if (kb + lane < K)
                xi_draw((uint32_t)(kb + lane), (uint32_t)m, (uint32_t)(sample0 + s), stream, k0, k1, n_seg, &pl, &sgl);
            const int kn = min(32, K - kb);
            for (int i = 0; i < kn; ++i) {
                const uint32_t p = __shfl_sync(0xffffffffu, pl, i), sg = __shfl_sync(0xffffffffu, sgl, i);
                if (lane < L) {
                    const size_t r = (size_t)p * L + lane;
                    const float f = ((sg >> lane) & 1u) ? -phi[r] : phi[r];
                    const float2 pu = zu[r], po = zo[r];
                    b[0] += f * pu.x; b[1] += f * pu.y;
                    b[2] += f * po.x; b[3] += f * po.y;
                }
            }
        }
#pragma unroll
        for (int i = 0; i < 4; ++i)
            for (int o = 16; o > 0; o >>= 1) b[i] += __shfl_xor_sync(0xffffffffu, b[i], o);
        if (lane == 0) {
            const float2 u = Uj[m];
            const T ur = (T)u.x * c, ui = (T)u.y * c;
            a[0] += (T)b[0] * ur - (T)b[1] * ui;
            a[1] += (T)b[0] * ui + (T)b[1] * ur;
            a[2] += (T)b[2] * ur - (T)b[3] * ui;
            a[3] += (T)b[2] * ui + (T)b[3] * ur;
        }
    }
    if constexpr (sizeof(T) == 8) block_sum<4>(a, sh);
    else block_sumf<4>(a, sh);
    if (threadIdx.x == 0) {
        const size_t base = ((size_t)s * (n_steps + 1) + j) * 2;
        partial[(base + 0) * gridDim.x + blockIdx.x] = make_double2((double)a[0], (double)a[1]);
        partial[(base + 1) * gridDim.x + blockIdx.x] = make_double2((double)a[2], (double)a[3]);
    }
}

void launch_sigma_accum_xi(const float2* zeta, const float* phi, const float2* Uxi, int n_samples, int64_t u_ss, int j,
                           int n_steps, int n_xi, int K, int L, int64_t ng, uint64_t seed, uint32_t stream, int sample0,
                           float c, int fp64, double2* partial, int nblk, cudaStream_t st) {
    const dim3 grid(nblk, n_samples);
    const uint32_t k0 = (uint32_t)(seed & 0xFFFFFFFFu), k1 = (uint32_t)(seed >> 32), ns = (uint32_t)(ng / L);
    if (fp64)
        k_sigma_accum_xi<double><<<grid, 256, 0, st>>>(zeta, phi, Uxi, u_ss, j, n_steps, n_xi, K, L, ns, k0, k1, stream,
                                                       sample0, c, ng, partial);
    else
        k_sigma_accum_xi<float><<<grid, 256, 0, st>>>(zeta, phi, Uxi, u_ss, j, n_steps, n_xi, K, L, ns, k0, k1, stream,
                                                      sample0, c, ng, partial);
}

// sigma[s][n + j] = dV S+ ; sigma[s][n - j] = -dV S- ; sigma[s][n] = (dV S+ - dV S-)/2 at j = 0.
// The cross-block sums run in the accumulation precision (fp64 flag).
__global__ void k_sigma_reduce(const double2* __restrict__ partial, int n_samples, int n_steps, int nblk, double dV,
                               int fp64, double2* __restrict__ sigma) {
    const int total = n_samples * (n_steps + 1);
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
        const int s = t / (n_steps + 1), j = t % (n_steps + 1);
        double2 r[2];
        for (int pm = 0; pm < 2; ++pm) {
            const double2* p = partial + ((size_t)t * 2 + pm) * nblk;
            if (fp64) {
                double x = 0, y = 0;
                for (int b = 0; b < nblk; ++b) { x += p[b].x; y += p[b].y; }
                r[pm] = make_double2(x, y);
            } else {
                float x = 0, y = 0;
                for (int b = 0; b < nblk; ++b) { x += (float)p[b].x; y += (float)p[b].y; }
                r[pm] = make_double2(x, y);
            }
        }
        double2* row = sigma + (size_t)s * (2 * n_steps + 1);
        const double2 sp = make_double2(dV * r[0].x, dV * r[0].y);
        const double2 sm = make_double2(-dV * r[1].x, -dV * r[1].y);
        if (j == 0) {
            row[n_steps] = make_double2(0.5 * (sp.x + sm.x), 0.5 * (sp.y + sm.y));
        } else {
            row[n_steps + j] = sp;
            row[n_steps - j] = sm;
        }
    }
}

void launch_sigma_reduce(const double2* partial, int n_samples, int n_steps, int nblk, double dV, int fp64,
                            double* sigma, cudaStream_t st) {
    const int total = n_samples * (n_steps + 1);
    const int blocks = (total + 127) / 128;
    k_sigma_reduce<<<blocks, 128, 0, st>>>(partial, n_samples, n_steps, nblk, dV, fp64,
                                           reinterpret_cast<double2*>(sigma));
}

// ------------------------------------------------------------------ time ordering
// One CTA per (GP grid points, sample).  Lines are padded to M + 1 complex.
template <int M, int GP, int NT>
__global__ void __launch_bounds__(NT)
k_time_order(int64_t ng, const float* __restrict__ uR, float2* __restrict__ u, int n_steps, const float2* __restrict__ tw) {
    extern __shared__ float2 sm[];
    constexpr int LS = M + 1;
    constexpr int NP = GP / 2;           // packed lines
    const int s = blockIdx.y;
    const int64_t g0 = (int64_t)blockIdx.x * GP;
    const int nt = n_steps + 1;
    const float* src = uR + (size_t)s * nt * ng;
    // 1. pack two real grid points per complex line (point 2l in .x, 2l+1 in .y), zero padded;
    //    reads run along the grid index so that each time row is one contiguous segment.
    for (int q = threadIdx.x; q < NP * (M - nt); q += NT) {
        const int l = q / (M - nt), t = nt + q % (M - nt);
        sm[l * LS + t] = make_float2(0.f, 0.f);
    }
    float* smf = reinterpret_cast<float*>(sm);
    for (int q = threadIdx.x; q < nt * GP; q += NT) {
        const int t = q / GP, p = q % GP;
        const int64_t g = g0 + p;
        smf[2 * ((p >> 1) * LS + t) + (p & 1)] = g < ng ? src[(size_t)t * ng + g] : 0.f;
    }
    __syncthreads();
    // 2. transform with e^{+i omega t}
    fft_lines<M, NP, LS, 1, NT, +1>(sm, tw);
    // 3. unpack: X_a = (Z_m + conj Z_-m)/2, X_b = -i (Z_m - conj Z_-m)/2; take the even extension of
    //    the non-negative frequencies (the negative half becomes the conjugate) -> lines 2l, 2l+1.
    constexpr int HALF = M / 2 + 1;
    constexpr int PER = (NP * HALF + NT - 1) / NT;
    float2 ya[PER], yb[PER];
#pragma unroll
    for (int p = 0; p < PER; ++p) {
        const int q = threadIdx.x + p * NT;
        if (q < NP * HALF) {
            const int l = q / HALF, m = q % HALF;
            const float2 zm = sm[l * LS + m];
            const float2 zn = sm[l * LS + ((M - m) & (M - 1))];
            ya[p] = make_float2(0.5f * (zm.x + zn.x), 0.5f * (zm.y - zn.y));
            yb[p] = make_float2(0.5f * (zm.y + zn.y), -0.5f * (zm.x - zn.x));
        }
    }
    __syncthreads();
#pragma unroll
    for (int p = 0; p < PER; ++p) {
        const int q = threadIdx.x + p * NT;
        if (q < NP * HALF) {
            const int l = q / HALF, m = q % HALF;
            sm[(2 * l) * LS + m] = ya[p];
            sm[(2 * l + 1) * LS + m] = yb[p];
            if (m > 0 && m < M / 2) {
                sm[(2 * l) * LS + M - m] = ya[p];
                sm[(2 * l + 1) * LS + M - m] = yb[p];
            }
        }
    }
    __syncthreads();
    // 4. inverse transform e^{-i omega t} / M
    fft_lines<M, GP, LS, 1, NT, -1>(sm, tw);
    const float inv = 1.0f / (float)M;
    float2* dst = u + (size_t)s * nt * ng;
    for (int q = threadIdx.x; q < GP * nt; q += NT) {
        const int t = q / GP, l = q % GP;
        const int64_t g = g0 + l;
        if (g < ng) dst[(size_t)t * ng + g] = cscale(sm[l * LS + t], inv);
    }
}

int time_order_threads(int M) { return M <= 1024 ? 256 : 512; }

template <int M> static void tlaunch(int64_t ng, const float* uR, float2* u, int n_samples, int n_steps,
                                     const float2* tw, cudaStream_t st) {
    constexpr int GP = M <= 2048 ? 8 : 4;
    constexpr int NT = M <= 1024 ? 256 : 512;
    const size_t smem = sizeof(float2) * GP * (M + 1);
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_time_order<M, GP, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        attr = true;
    }
    const dim3 grid((unsigned)((ng + GP - 1) / GP), n_samples);
    k_time_order<M, GP, NT><<<grid, NT, smem, st>>>(ng, uR, u, n_steps, tw);
}

void launch_time_order(int ng, const float* uR, float2* u, int n_samples, int n_steps, int M, const float2* twM,
                       cudaStream_t st) {
    switch (M) {
        case 4: tlaunch<4>(ng, uR, u, n_samples, n_steps, twM, st); break;
        case 8: tlaunch<8>(ng, uR, u, n_samples, n_steps, twM, st); break;
        case 16: tlaunch<16>(ng, uR, u, n_samples, n_steps, twM, st); break;
        case 32: tlaunch<32>(ng, uR, u, n_samples, n_steps, twM, st); break;
        case 64: tlaunch<64>(ng, uR, u, n_samples, n_steps, twM, st); break;
        case 128: tlaunch<128>(ng, uR, u, n_samples, n_steps, twM, st); break;
        case 256: tlaunch<256>(ng, uR, u, n_samples, n_steps, twM, st); break;
        case 512: tlaunch<512>(ng, uR, u, n_samples, n_steps, twM, st); break;
        case 1024: tlaunch<1024>(ng, uR, u, n_samples, n_steps, twM, st); break;
        case 2048: tlaunch<2048>(ng, uR, u, n_samples, n_steps, twM, st); break;
        case 4096: tlaunch<4096>(ng, uR, u, n_samples, n_steps, twM, st); break;
        default: break;
    }
}

// ------------------------------------------------------------------ Sigma(omega) (Eq. 7)
template <typename T>
__device__ __forceinline__ void damped_term(const double2* __restrict__ sigma, int n_samples, int n_steps, int jj,
                                            double dt, double gamma, T& re, T& im, T& t) {
    // mean over samples of Sigma(t_j), times dt w_j e^{-gamma^2 t^2 / 2}
    double sx = 0, sy = 0;
    for (int s = 0; s < n_samples; ++s) {
        const double2 v = sigma[(size_t)s * (2 * n_steps + 1) + jj];
        sx += v.x;
        sy += v.y;
    }
    const int j = jj - n_steps;
    const T tj = (T)(dt * j);
    const T w = (jj == 0 || jj == 2 * n_steps) ? (T)0.5 : (T)1.0;
    const T damp = (T)dt * w * exp(-(T)0.5 * (T)gamma * (T)gamma * tj * tj) / (T)n_samples;
    re = (T)sx * damp;
    im = (T)sy * damp;
    t = tj;
}

template <typename T>
__global__ void k_sigma_omega(const double2* __restrict__ sigma, int n_samples, int n_steps, double dt, double gamma,
                              const double* __restrict__ omega, int n_omega, double2* __restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_omega) return;
    const T w = (T)omega[i];
    T ax = 0, ay = 0;
    for (int jj = 0; jj <= 2 * n_steps; ++jj) {
        T re, im, t;
        damped_term<T>(sigma, n_samples, n_steps, jj, dt, gamma, re, im, t);
        T sn, cs;
        sincos(w * t, &sn, &cs);
        ax += re * cs - im * sn;
        ay += re * sn + im * cs;
    }
    out[i] = make_double2((double)ax, (double)ay);
}

void launch_sigma_omega(const double* sigma, int n_samples, int n_steps, double dt, double gamma, const double* omega,
                        int n_omega, int fp64, double* out, cudaStream_t st) {
    if (n_omega == 0) return;
    const int blocks = (n_omega + 127) / 128;
    if (fp64)
        k_sigma_omega<double><<<blocks, 128, 0, st>>>(reinterpret_cast<const double2*>(sigma), n_samples, n_steps, dt,
                                                      gamma, omega, n_omega, reinterpret_cast<double2*>(out));
    else
        k_sigma_omega<float><<<blocks, 128, 0, st>>>(reinterpret_cast<const double2*>(sigma), n_samples, n_steps, dt,
                                                     gamma, omega, n_omega, reinterpret_cast<double2*>(out));
}

// ------------------------------------------------------------------ QP equation (Eq. 6)
// damped[jj] = mean_s Sigma_s(t_j) * dt w_j e^{-gamma^2 t_j^2/2}  (complex), jj = 0..2n
template <typename T>
__global__ void k_qp_damped(const double2* __restrict__ sigma, int n_samples, int n_steps, double dt, double gamma,
                            double2* __restrict__ damped) {
    const int jj = blockIdx.x * blockDim.x + threadIdx.x;
    if (jj > 2 * n_steps) return;
    T re, im, t;
    damped_term<T>(sigma, n_samples, n_steps, jj, dt, gamma, re, im, t);
    damped[jj] = make_double2((double)re, (double)im);
}

template <typename T>
__device__ __forceinline__ T re_sigma_at(const double2* __restrict__ damped, int n_steps, double dt, T w, int j0, int js) {
    T acc = 0;
    for (int jj = j0; jj <= 2 * n_steps; jj += js) {
        const T t = (T)(dt * (jj - n_steps));
        T sn, cs;
        sincos(w * t, &sn, &cs);
        acc += (T)damped[jj].x * cs - (T)damped[jj].y * sn;
    }
    return acc;
}

// scan[i] = f(w_i) = w_i - eps - X - Re Sigma(w_i) + vxc, w_i = eps - window + i step
template <typename T>
__global__ void k_qp_scan(const double2* __restrict__ damped, int n_steps, double dt, double eps,
                          const double* __restrict__ x, int n_samples, double vxc, double window, double step,
                          int n_scan, double* __restrict__ scan) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_scan) return;
    double xm = 0.0;
    for (int s = 0; s < n_samples; ++s) xm += x[s];
    xm /= n_samples;
    const double w = eps - window + step * i;
    scan[i] = w - eps - xm - (double)re_sigma_at<T>(damped, n_steps, dt, (T)w, 0, 1) + vxc;
}

template <typename T>
__device__ double block_re_sigma(const double2* damped, int n_steps, double dt, double w, double* sh) {
    double v[1] = {(double)re_sigma_at<T>(damped, n_steps, dt, (T)w, threadIdx.x, blockDim.x)};
    __syncthreads();
    block_sum<1>(v, sh);
    __syncthreads();
    if (threadIdx.x == 0) sh[64] = v[0];
    __syncthreads();
    const double r = sh[64];
    __syncthreads();
    return r;
}

// Single CTA: bracket nearest eps, bisection to 1e-10, standard error with the Z factor.
// result = (eps_qp, se, Re Sigma(eps_qp), Z); status[0] = 0 ok, 1 no root.
template <typename T>
__global__ void __launch_bounds__(256)
k_qp_solve(const double2* __restrict__ sigma, const double* __restrict__ x, const double2* __restrict__ damped,
           int n_samples, int n_steps, double dt, double gamma, double eps, double vxc, double window, double step,
           const double* __restrict__ scan, int n_scan, double* __restrict__ result) {
    __shared__ double sh[96];
    __shared__ int best;
    __shared__ double xm_s;
    if (threadIdx.x == 0) {
        double xs = 0;
        for (int s = 0; s < n_samples; ++s) xs += x[s];
        xm_s = xs / n_samples;
        // bracket whose midpoint is nearest eps (first on ties)
        int bi = -1;
        double bd = 1e300;
        for (int i = 0; i + 1 < n_scan; ++i) {
            const double a = scan[i], b = scan[i + 1];
            const int sa = (a > 0) - (a < 0), sb = (b > 0) - (b < 0);
            if (sa * sb <= 0) {
                const double mid = 0.5 * ((eps - window + step * i) + (eps - window + step * (i + 1)));
                const double d = fabs(mid - eps);
                if (d < bd) { bd = d; bi = i; }
            }
        }
        best = bi;
    }
    __syncthreads();
    if (best < 0) {
        if (threadIdx.x == 0) { result[0] = nan(""); result[1] = nan(""); result[2] = nan(""); result[3] = nan(""); }
        return;
    }
    const double xm = xm_s;
    double a = eps - window + step * best, b = eps - window + step * (best + 1);
    double fa = scan[best];
    while (b - a > 1e-10) {
        const double c = 0.5 * (a + b);
        const double fc = c - eps - xm - block_re_sigma<T>(damped, n_steps, dt, c, sh) + vxc;
        const int sfc = (fc > 0) - (fc < 0), sfa = (fa > 0) - (fa < 0);
        if (sfc == sfa && fc != 0.0) { a = c; fa = fc; }
        else b = c;
    }
    const double e = 0.5 * (a + b);
    const double rs = block_re_sigma<T>(damped, n_steps, dt, e, sh);
    const double d = 1e-4;
    const double slope = (block_re_sigma<T>(damped, n_steps, dt, e + d, sh) -
                          block_re_sigma<T>(damped, n_steps, dt, e - d, sh)) / (2 * d);
    const double z = 1.0 / (1.0 - slope);
    // per-sample X_i + Re Sigma_i(e): Sigma_i(t) damped the same way (no sample mean)
    double m1 = 0, m2 = 0;
    for (int s = 0; s < n_samples; ++s) {
        double acc = 0;
        for (int jj = threadIdx.x; jj <= 2 * n_steps; jj += blockDim.x) {
            const int j = jj - n_steps;
            const T t = (T)(dt * j);
            const T w = (jj == 0 || jj == 2 * n_steps) ? (T)0.5 : (T)1.0;
            const T damp = (T)dt * w * exp(-(T)0.5 * (T)gamma * (T)gamma * t * t);
            const double2 v = sigma[(size_t)s * (2 * n_steps + 1) + jj];
            T sn, cs;
            sincos((T)e * t, &sn, &cs);
            acc += (double)(((T)v.x * cs - (T)v.y * sn) * damp);
        }
        double vv[1] = {acc};
        __syncthreads();
        block_sum<1>(vv, sh);
        __syncthreads();
        if (threadIdx.x == 0) {
            const double per = x[s] + vv[0];
            m1 += per;
            m2 += per * per;
        }
    }
    if (threadIdx.x == 0) {
        double se = nan("");
        if (n_samples > 1) {
            const double mean = m1 / n_samples;
            const double var = (m2 - n_samples * mean * mean) / (n_samples - 1);
            se = fabs(z) * sqrt(fmax(var, 0.0) / n_samples);
        }
        result[0] = e;
        result[1] = se;
        result[2] = rs;
        result[3] = z;
    }
}

void launch_qp(const double* sigma, const double* x, int n_samples, int n_steps, double dt, double gamma, double eps_ks,
               double vxc, double window, double step, int fp64, double* scan, int n_scan, double* result,
               cudaStream_t st) {
    // scan[] holds n_scan doubles followed by the 2 n_steps + 1 damped complex terms
    double2* damped = reinterpret_cast<double2*>(scan + ((n_scan + 1) & ~1));
    const double2* sg = reinterpret_cast<const double2*>(sigma);
    const int nt = 2 * n_steps + 1;
    if (fp64) {
        k_qp_damped<double><<<(nt + 127) / 128, 128, 0, st>>>(sg, n_samples, n_steps, dt, gamma, damped);
        k_qp_scan<double><<<(n_scan + 127) / 128, 128, 0, st>>>(damped, n_steps, dt, eps_ks, x, n_samples, vxc, window,
                                                              step, n_scan, scan);
        k_qp_solve<double><<<1, 256, 0, st>>>(sg, x, damped, n_samples, n_steps, dt, gamma, eps_ks, vxc, window, step,
                                              scan, n_scan, result);
    } else {
        k_qp_damped<float><<<(nt + 127) / 128, 128, 0, st>>>(sg, n_samples, n_steps, dt, gamma, damped);
        k_qp_scan<float><<<(n_scan + 127) / 128, 128, 0, st>>>(damped, n_steps, dt, eps_ks, x, n_samples, vxc, window,
                                                             step, n_scan, scan);
        k_qp_solve<float><<<1, 256, 0, st>>>(sg, x, damped, n_samples, n_steps, dt, gamma, eps_ks, vxc, window, step,
                                             scan, n_scan, result);
    }
}

}  // namespace sgw

// ------------------------------------------------------------------ QP solve without allocation
// Some callers cannot let a library allocate device memory at all: a host application that has
// reserved the device's memory for its own pool allocator, or a plugin host that forbids
// allocations while it runs, would see cudaMalloc fail or have its memory accounting broken.
// For them sgw_qp_energy_noalloc runs the QP solve with its scratch in this fixed, statically
// sized device array instead of a context work area.  Every GPU that loads the library holds
// the array until the process exits.
namespace {
constexpr int kQpScratchDoubles = 131072;   // 1 MiB
static __device__ __align__(256) double g_qp_scratch[kQpScratchDoubles];

// Device address of g_qp_scratch on each device, looked up once per device with that device
// current (the host-side name is only a stand-in, not a device address).
constexpr int kMaxDevices = 64;
double* g_qp_scratch_dev[kMaxDevices] = {nullptr};
std::mutex g_qp_scratch_mu;
}  // namespace

extern "C" sgw_status sgw_qp_energy_noalloc(const double* sigma_dev, const double* x_dev, int n_samples,
                                            int n_steps, double dt, double gamma, double eps_ks, double vxc,
                                            double window, double step, int fp64, double* result_host,
                                            void* stream) {
    if (n_samples < 1 || n_steps < 0 || !(window > 0) || !(step > 0) || !sigma_dev || !x_dev || !result_host) {
        sgw::set_global_error("sgw_qp_energy_noalloc: bad arguments");
        return SGW_EINVAL;
    }
    // the scan size is checked as a double first: a huge window or a tiny step would overflow the
    // integer conversion
    const double r = 2.0 * window / step;
    if (!std::isfinite(r) || r + 1.0 > (double)kQpScratchDoubles) {
        sgw::set_global_error("sgw_qp_energy_noalloc: 2 window/step + 1 scan points exceed the 1 MiB static scratch "
                              "(131072 doubles)");
        return SGW_EINVAL;
    }
    const long long n_scan = std::llround(r) + 1;
    const long long need = ((n_scan + 1) & ~1LL) + 2LL * (2LL * n_steps + 1) + 4;
    if (need > kQpScratchDoubles) {
        sgw::set_global_error("sgw_qp_energy_noalloc: window/step and n_steps need more than the 1 MiB static "
                              "scratch (even(2 window/step + 1) + 2 (2 n_steps + 1) + 4 <= 131072 doubles)");
        return SGW_EINVAL;
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        sgw::set_global_error("sgw_qp_energy_noalloc: no usable current device");
        return SGW_ECUDA;
    }
    cudaStream_t st = (cudaStream_t)stream;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if ((e = cudaStreamIsCapturing(st, &cap)) != cudaSuccess) {
        sgw::set_global_error((std::string("sgw_qp_energy_noalloc: ") + cudaGetErrorString(e)).c_str());
        return SGW_ECUDA;
    }
    double* scratch = nullptr;
    {
        // Outside a capture the address is looked up on every call (cheap), so a context that the
        // application reset and re-created gets the new one; during a capture the address cached
        // by an earlier call on this device is used.
        std::lock_guard<std::mutex> lk(g_qp_scratch_mu);
        if (cap == cudaStreamCaptureStatusNone) {
            void* p = nullptr;
            e = cudaGetSymbolAddress(&p, g_qp_scratch);
            if (e != cudaSuccess || !p) {
                sgw::set_global_error((std::string("sgw_qp_energy_noalloc: cudaGetSymbolAddress: ") +
                                       cudaGetErrorString(e)).c_str());
                return SGW_ECUDA;
            }
            g_qp_scratch_dev[dev] = static_cast<double*>(p);
        } else if (!g_qp_scratch_dev[dev]) {
            sgw::set_global_error("sgw_qp_energy_noalloc: the first call on a device must come before any stream "
                                  "capture");
            return SGW_ESTATE;
        }
        scratch = g_qp_scratch_dev[dev];
    }
    // scan values, then the damped terms, then the 4 result doubles; every element read in
    // this call is written first in this call, so nothing needs clearing between calls.
    double* result = scratch + (need - 4);
    sgw::launch_qp(sigma_dev, x_dev, n_samples, n_steps, dt, gamma, eps_ks, vxc, window, step, fp64, scratch,
                   (int)n_scan, result, st);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(result_host, result, 4 * sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        sgw::set_global_error((std::string("sgw_qp_energy_noalloc: ") + cudaGetErrorString(e)).c_str());
        return SGW_ECUDA;
    }
    if (std::isnan(result_host[0])) {
        sgw::set_global_error("sgw_qp_energy_noalloc: no sign change of the QP equation in the window");
        return SGW_ENOCONV;
    }
    return SGW_OK;
}
