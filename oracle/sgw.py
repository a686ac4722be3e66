"""FP64 oracle: one Monte-Carlo sample of stochastic GW in the sROI form, step by step.

TEST INFRASTRUCTURE: part of the CPU oracle; only tests, the smoke check and the
CPU-baseline leg of the benchmark may use it.  It shares no code with the CUDA path.

The steps follow Sec. 2.1 (Fig. 1) in the paper's order:
  1. white-noise orbitals zeta-bar and eta-bar_l (Sec. 2.1), here Rademacher +-1/sqrt(dV)
     from Philox so that E[|zeta-bar><zeta-bar|] = 1 in the dV inner product;
  2. filtering with the gapped Heaviside filter (Eq. 3): eta_l = P eta-bar_l,
     zeta_occ = P zeta-bar, zeta_unocc = zeta-bar - zeta_occ;
  3. linear-response time-dependent Hartree: a perturbed copy of each eta_l is kicked
     by the potential v_p = v_C * (zeta-bar phi) of the source zeta-bar phi and both copies
     are propagated under H(t) = H0 + v_C * (rho(t) - rho(0)), rho = (2/N_eta) sum |eta_l|^2;
     u^R(t) is the difference of the induced potentials divided by the kick strength
     (the tangent-linear form takes the kick strength to zero exactly);
  4. time ordering of u^R to u (FFT over t, conjugation of the negative frequencies,
     inverse FFT);
  5. zeta propagation: zeta_unocc forward and zeta_occ backward in time (Eq. 4, iG as a
     time correlation function, with iG = -sum_occ for t < 0);
  6. Sigma(t) = dV sum_r phi zeta(t) u(t) (Eq. 5);
  7. Sigma(omega) by the damped transform of Eq. 7 (trapezoid rule over t_j, |j| <= N_tau);
  8. the QP equation (Eq. 6) with the sROI exchange X in the eta basis.
"""
import numpy as np

from . import hamiltonian as ham
from . import chebyshev as cheb
from . import splitop
from .philox import rademacher_words


# ---------------------------------------------------------------- white noise (Sec. 2.1)
def white_noise(grid, seed, stream, sample, n_vec):
    """Real Rademacher orbitals +-1/sqrt(dV), shape [n_vec, n, n, n].

    Vector 0 of a sample is zeta-bar, vectors 1..N_eta are the eta-bar_l.
    """
    out = np.empty((n_vec,) + grid.shape(), dtype=np.float64)
    for v in range(n_vec):
        s = rademacher_words(seed, stream, sample, v, grid.ng).astype(np.float64)
        out[v] = (s / np.sqrt(grid.dV)).reshape(grid.shape())
    return out


class Problem:
    """H0 and the spectral data a sample needs."""

    def __init__(self, grid, vloc, kb, emin, emax, e_homo, e_lumo, phi):
        self.grid = grid
        self.vloc = np.asarray(vloc, dtype=np.float64)
        self.kb = kb
        self.emin, self.emax = emin, emax
        self.e_homo, self.e_lumo = e_homo, e_lumo
        self.phi = np.asarray(phi, dtype=np.float64)

    def h0(self, psi, vext=None):
        return ham.apply_h(psi, self.grid, self.vloc, self.kb, vext)


# ---------------------------------------------------------------- filtering (Eq. 3)
def filter_batch(prob, noise, coeffs):
    """Gapped-filter projection of a batch of white-noise vectors onto the occupied space."""
    return cheb.filter_occupied(prob.h0, noise.astype(np.complex128), coeffs, prob.emin, prob.emax)


# ---------------------------------------------------------------- TDH (Sec. 2.1)
def density(eta, n_eta):
    """rho(r) = (2/N_eta) sum_l |eta_l(r)|^2 (closed shell)."""
    return (2.0 / n_eta) * np.sum(np.abs(eta) ** 2, axis=0)


def tdh_response_tangent(prob, eta, source, n_steps, dt, K, weight=None, split=None):
    """u^R(t_j), j = 0..n_steps, by the tangent-linear (lambda -> 0) pair.

    eta: filtered occupied stochastic orbitals [N_eta, n, n, n]; source: zeta-bar * phi.
    The perturbed copy is represented by its derivative with respect to the kick
    strength: d eta(0) = -i v_p eta(0) for the kick e^{-i lambda v_p}.  Each step holds
    H(t_j) fixed.  `weight` replaces 2/N_eta in the density (2 for exact orbitals).
    split: None for the degree-K Chebyshev step, else the splitop.KBSplit of the KB part
    (or False without KB) for the split-operator step.
    Returns u^R as a real array [n_steps + 1, n, n, n].
    """
    g = prob.grid
    n_eta = eta.shape[0]
    w = (2.0 / n_eta) if weight is None else weight
    vp = ham.poisson(source, g).real
    e = eta.astype(np.complex128)
    de = -1j * vp * e
    rho0 = w * np.sum(np.abs(e) ** 2, axis=0)
    uR = np.zeros((n_steps + 1,) + g.shape())
    for j in range(n_steps + 1):
        rho = w * np.sum(np.abs(e) ** 2, axis=0)
        drho = w * np.sum(2.0 * np.real(np.conj(e) * de), axis=0)
        dvh = ham.poisson(rho - rho0, g).real
        dv = ham.poisson(drho, g).real
        uR[j] = dv
        if j == n_steps:
            break
        if split is None:
            e, de = cheb.propagate_step_tangent(lambda v: prob.h0(v, dvh), e, de, dv,
                                                prob.emin, prob.emax, dt, K)
        else:
            pair = [splitop.split_step_tangent(e[l], de[l], g, prob.vloc + dvh, dv, split or None, dt)
                    for l in range(n_eta)]
            e = np.stack([p[0] for p in pair])
            de = np.stack([p[1] for p in pair])
    return uR


def tdh_response_fd(prob, eta, source, n_steps, dt, K, lam=1e-4, weight=None):
    """u^R(t_j) by the paper's pair of unperturbed and perturbed copies (finite kick lam).

    eta^lam(0) = e^{-i lam v_p} eta(0); both copies propagate under their own
    H^x(t_j) = H0 + v_C * (rho^x(t_j) - rho(0)); u^R = (v_H[rho^lam] - v_H[rho^0]) / lam.
    """
    g = prob.grid
    n_eta = eta.shape[0]
    w = (2.0 / n_eta) if weight is None else weight
    vp = ham.poisson(source, g).real
    e0 = eta.astype(np.complex128)
    el = np.exp(-1j * lam * vp) * e0
    rho0 = w * np.sum(np.abs(e0) ** 2, axis=0)
    uR = np.zeros((n_steps + 1,) + g.shape())
    for j in range(n_steps + 1):
        v0 = ham.poisson(w * np.sum(np.abs(e0) ** 2, axis=0) - rho0, g).real
        vl = ham.poisson(w * np.sum(np.abs(el) ** 2, axis=0) - rho0, g).real
        uR[j] = (vl - v0) / lam
        if j == n_steps:
            break
        e0 = cheb.propagate_step(lambda v: prob.h0(v, v0), e0, prob.emin, prob.emax, dt, K)
        el = cheb.propagate_step(lambda v: prob.h0(v, vl), el, prob.emin, prob.emax, dt, K)
    return uR


# ---------------------------------------------------------------- time ordering
def time_order_length(n_steps):
    """FFT length over t: the smallest power of two >= 4 (n_steps + 1)."""
    m = 1
    while m < 4 * (n_steps + 1):
        m *= 2
    return m


def time_order(uR, M=None):
    """u(t_j), j = 0..N_tau, from the causal u^R(t_j) (axis 0 is time).

    u^R is zero-padded to length M (zero for t < 0), transformed with e^{+i omega t},
    its negative-frequency half is replaced by its complex conjugate (so that
    u(omega) = u^R(|omega|)), and the inverse transform is taken.  u(t) is even in t.
    """
    n = uR.shape[0]
    if M is None:
        M = time_order_length(n - 1)
    x = np.zeros((M,) + uR.shape[1:], dtype=np.complex128)
    x[:n] = uR
    X = np.fft.ifft(x, axis=0) * M            # sum_j x_j e^{+2 pi i j m / M}
    Y = X.copy()
    Y[M // 2 + 1:] = np.conj(X[M // 2 + 1:])
    y = np.fft.fft(Y, axis=0) / M              # (1/M) sum_m Y_m e^{-2 pi i j m / M}
    return y[:n]


# ---------------------------------------------------------------- zeta propagation and Sigma(t)
def sigma_t(prob, zeta_occ, zeta_unocc, u, n_steps, dt, K, split=None):
    """Sigma(t_j), j = -N_tau..N_tau, of one sample (Eq. 4 and Eq. 5).

    zeta(t) = e^{-i H0 t} zeta_unocc for t > 0 and -e^{-i H0 t} zeta_occ for t < 0;
    Sigma(t) = dV sum_r phi(r) zeta(r, t) u(r, |t|).  At t = 0 the two one-sided limits
    are averaged.  Returns a complex array of length 2 N_tau + 1 (index j + N_tau).
    """
    g = prob.grid
    phi = prob.phi
    zp = zeta_unocc.astype(np.complex128)
    zm = zeta_occ.astype(np.complex128)
    out = np.zeros(2 * n_steps + 1, dtype=np.complex128)
    for j in range(n_steps + 1):
        sp = g.dV * np.sum(phi * zp * u[j])
        sm = -g.dV * np.sum(phi * zm * u[j])
        if j == 0:
            out[n_steps] = 0.5 * (sp + sm)
        else:
            out[n_steps + j] = sp
            out[n_steps - j] = sm
        if j == n_steps:
            break
        if split is None:
            zp = cheb.propagate_step(prob.h0, zp, prob.emin, prob.emax, dt, K)
            zm = cheb.propagate_step(prob.h0, zm, prob.emin, prob.emax, -dt, K)
        else:
            zp = splitop.split_step(zp, g, prob.vloc, split or None, dt)
            zm = splitop.split_step(zm, g, prob.vloc, split or None, -dt)
    return out


# ---------------------------------------------------------------- exchange (Eq. 6)
def exchange(prob, eta):
    """sROI exchange X = -(1/N_eta) sum_l <phi eta_l | v_C | phi eta_l>."""
    g = prob.grid
    f = prob.phi * eta
    vf = ham.poisson(f, g)
    return float(-np.real(np.sum(g.dot(f, vf))) / eta.shape[0])


# ---------------------------------------------------------------- Sigma(omega), QP (Eq. 6, 7)
def sigma_omega(sig_t, dt, gamma, omega):
    """Eq. 7 by the trapezoid rule: dt sum_j w_j Sigma(t_j) e^{-gamma^2 t_j^2 / 2} e^{i omega t_j}.

    w_j = 1/2 at j = +-N_tau, 1 otherwise.  omega may be an array.
    """
    nt = (len(sig_t) - 1) // 2
    t = dt * np.arange(-nt, nt + 1)
    w = np.ones(2 * nt + 1)
    w[0] = w[-1] = 0.5
    damped = dt * w * sig_t * np.exp(-0.5 * gamma ** 2 * t ** 2)
    om = np.atleast_1d(np.asarray(omega, dtype=np.float64))
    return np.exp(1j * np.outer(om, t)) @ damped


def qp_root(re_sigma, eps_ks, x, vxc, window=2.0, step=1e-3, tol=1e-10):
    """Root of f(w) = w - eps_ks - x - Re Sigma(w) + vxc nearest eps_ks (Eq. 6).

    Scans [eps_ks - window, eps_ks + window] in steps of `step` for sign changes,
    takes the bracket whose midpoint is nearest eps_ks and bisects it to `tol`.
    Returns None when no sign change is found.
    """
    n = int(round(2 * window / step))
    w = eps_ks - window + step * np.arange(n + 1)
    f = w - eps_ks - x - re_sigma(w) + vxc
    idx = np.nonzero(np.sign(f[:-1]) * np.sign(f[1:]) <= 0)[0]
    if len(idx) == 0:
        return None
    i = idx[np.argmin(np.abs(0.5 * (w[idx] + w[idx + 1]) - eps_ks))]
    a, b = w[i], w[i + 1]
    fa = f[i]
    while b - a > tol:
        c = 0.5 * (a + b)
        fc = c - eps_ks - x - re_sigma(np.array([c]))[0] + vxc
        if np.sign(fc) == np.sign(fa) and fc != 0:
            a, fa = c, fc
        else:
            b = c
    return 0.5 * (a + b)


def qp_energy(sig_t_samples, x_samples, dt, gamma, eps_ks, vxc=0.0):
    """QP energy from per-sample Sigma_i(t) and X_i (Eq. 6), with its standard error.

    The root is taken for the sample means.  The standard error is the linearised
    one: Z * std_i(X_i + Re Sigma_i(eps_qp)) / sqrt(N), Z = 1 / (1 - d Re Sigma / d omega).
    """
    S = np.asarray(sig_t_samples)
    X = np.asarray(x_samples, dtype=np.float64)
    mean_s = S.mean(axis=0)
    mean_x = float(X.mean())
    re_sig = lambda w: sigma_omega(mean_s, dt, gamma, w).real
    e = qp_root(re_sig, eps_ks, mean_x, vxc)
    if e is None:
        return None, None
    n = S.shape[0]
    if n < 2:
        return e, float('nan')
    per = np.array([X[i] + sigma_omega(S[i], dt, gamma, e).real[0] for i in range(n)])
    d = 1e-4
    slope = (re_sig(np.array([e + d]))[0] - re_sig(np.array([e - d]))[0]) / (2 * d)
    z = 1.0 / (1.0 - slope)
    return e, abs(z) * per.std(ddof=1) / np.sqrt(n)


# ---------------------------------------------------------------- one Monte-Carlo sample
def run_sample(prob, coeffs, seed, stream, sample, n_eta, n_steps, dt, K, mode='tangent'):
    """All steps of Fig. 1 for one MC sample; returns (Sigma(t) [2N+1], X, intermediates)."""
    noise = white_noise(prob.grid, seed, stream, sample, n_eta + 1)
    filt = filter_batch(prob, noise, coeffs)
    zbar = noise[0]
    zocc = filt[0]
    zunocc = zbar - zocc
    eta = filt[1:]
    source = zbar * prob.phi
    if mode == 'tangent':
        uR = tdh_response_tangent(prob, eta, source, n_steps, dt, K)
    else:
        uR = tdh_response_fd(prob, eta, source, n_steps, dt, K)
    u = time_order(uR)
    sig = sigma_t(prob, zocc, zunocc, u, n_steps, dt, K)
    x = exchange(prob, eta)
    return sig, x, dict(noise=noise, filt=filt, uR=uR, u=u)
