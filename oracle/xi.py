"""FP64 oracle: the sparse stochastic compression of u^R on fragmented segments (Sec. 2.1, Sec. 2.3).

TEST INFRASTRUCTURE: part of the CPU oracle; only tests, the smoke check and the
CPU-baseline leg of the benchmark may use it.

The paper projects u^R(r, t) on N_xi random functions xi_m supported on short fragmented segments of
the grid (fraction f_g of the grid each, segments of L points) and carries U_m(t) = <xi_m|u^R(t)>
instead of u^R on the full grid.  Reading taken here (the construction's details are not given):
xi_m is the sum of K = round(N_g f_g / L) segment draws (nearest integer, halves up); draw k covers
the L contiguous flat grid points starting at L p_{m,k}, p_{m,k} uniform in [0, N_g / L), with an
independent sign per point, and the whole function is scaled by c = 1 / sqrt(N_xi K L dV / N_g):

    xi_m(r) = c sum_k [r in segment p_{m,k}] s_{m,k}(r),

so that E[dV sum_m xi_m xi_m^T] = 1, the identity in the dV inner product (a point is covered by a
draw with probability L / N_g, and signs of different points or draws are independent).  Then
u(r, t) ~ sum_m xi_m(r) U_m(t), the time ordering acts on U_m(t) (it is linear and acts point by
point), and Sigma(t) = dV sum_r phi zeta(t) u(|t|) becomes sum_m [dV sum_r phi zeta(t) xi_m] U_m(|t|).

Random numbers: Philox4x32-10 with key (seed mod 2^32, seed div 2^32) and counter (k, m, sample,
stream); word 0 gives p = floor(word0 (N_g / L) / 2^32), bit l of word 1 the sign of point l of the
segment (set -> -1); L <= 32.
"""
import numpy as np

from .philox import philox4x32_10


def n_draws(ng, f_g, L):
    """K = N_g f_g / L to the nearest integer, halves rounded up, and at least 1."""
    return max(1, int(np.floor(ng * f_g / L + 0.5)))


def draws(seed, stream, sample, n_xi, K, n_seg):
    """Segment indices [n_xi, K] and sign words [n_xi, K] of one sample's xi functions."""
    kk, mm = np.meshgrid(np.arange(K, dtype=np.uint64), np.arange(n_xi, dtype=np.uint64))
    w0, w1, _, _ = philox4x32_10(kk, mm, np.uint64(sample), np.uint64(stream), seed & 0xFFFFFFFF,
                                 (seed >> 32) & 0xFFFFFFFF)
    pos = (w0.astype(np.uint64) * np.uint64(n_seg)) >> np.uint64(32)
    return pos.astype(np.int64), w1


def scale(ng, n_xi, K, L, dV):
    return 1.0 / np.sqrt(n_xi * K * L * dV / ng)


def dense(grid, seed, stream, sample, n_xi, f_g, L):
    """The xi functions as a dense [n_xi, N_g] array (small grids; the definition written out)."""
    ng = grid.ng
    K = n_draws(ng, f_g, L)
    pos, sw = draws(seed, stream, sample, n_xi, K, ng // L)
    c = scale(ng, n_xi, K, L, grid.dV)
    xi = np.zeros((n_xi, ng))
    for m in range(n_xi):
        for k in range(K):
            for l in range(L):
                sgn = -1.0 if (int(sw[m, k]) >> l) & 1 else 1.0
                xi[m, pos[m, k] * L + l] += c * sgn
    return xi


def project(f, grid, seed, stream, sample, n_xi, f_g, L):
    """U_m = <xi_m|f> = dV sum_r xi_m(r) f(r) for f of shape [..., N_g] (segment gathers)."""
    ng = grid.ng
    K = n_draws(ng, f_g, L)
    pos, sw = draws(seed, stream, sample, n_xi, K, ng // L)
    c = scale(ng, n_xi, K, L, grid.dV)
    f = np.asarray(f).reshape(f.shape[:-3] + (ng,)) if np.ndim(f) >= 3 and f.shape[-1] != ng else np.asarray(f)
    bits = ((sw[..., None].astype(np.int64) >> np.arange(L)) & 1)            # [n_xi, K, L]
    sgn = 1.0 - 2.0 * bits
    idx = pos[..., None] * L + np.arange(L)                                   # [n_xi, K, L]
    vals = f[..., idx]                                                        # [..., n_xi, K, L]
    return grid.dV * c * np.sum(vals * sgn, axis=(-1, -2))


def reconstruct(U, grid, seed, stream, sample, n_xi, f_g, L):
    """sum_m xi_m(r) U_m for U of shape [..., n_xi] -> [..., N_g]."""
    ng = grid.ng
    K = n_draws(ng, f_g, L)
    pos, sw = draws(seed, stream, sample, n_xi, K, ng // L)
    c = scale(ng, n_xi, K, L, grid.dV)
    U = np.asarray(U)
    out = np.zeros(U.shape[:-1] + (ng,), dtype=np.result_type(U.dtype, np.float64))
    for m in range(n_xi):
        for k in range(K):
            bits = (int(sw[m, k]) >> np.arange(L)) & 1
            sgn = 1.0 - 2.0 * bits
            seg = slice(pos[m, k] * L, pos[m, k] * L + L)
            out[..., seg] += c * sgn * U[..., m:m + 1]
    return out
