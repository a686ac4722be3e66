"""FP64 oracle: spectral bounds, the gapped Heaviside filter and the Chebyshev propagator.

TEST INFRASTRUCTURE: part of the CPU oracle; only tests, the smoke check and the
CPU-baseline leg of the benchmark may use it.

* Spectral bounds (Sec. 2.1): shifted power iteration.  Power iteration on H gives
  E_max; power iteration on (H - E_max) gives E_min - E_max.  Both are widened by
  a margin so that the mapped spectrum lies inside [-1, 1].
* Gapped filter (Eq. 3, Sec. 2.1): Theta(mu - H) ~ sum_{n=0}^{N_chb} a_n T_n(H~),
  H~ = (H - Ebar)/dE.  The a_n are the least-squares fit of the step function on
  Chebyshev-Gauss nodes with zero weight inside [E_HOMO, E_LUMO] (the cutoff is
  spread over the gap), plus a small ridge term that makes the fit unique.
* Propagator: e^{-i H dt} = e^{-i Ebar dt} sum_k (2 - delta_k0) (-i)^k J_k(dE dt) T_k(H~)
  (the Jacobi-Anger expansion), truncated at degree K, with H frozen over a step.
All Chebyshev sums here use the plain three-term recurrence
T_0 = psi, T_1 = H~ psi, T_{n+1} = 2 H~ T_n - T_{n-1}.
"""
import numpy as np
import scipy.special


# ---------------------------------------------------------------- spectral bounds
def power_iteration(apply_a, v0, n_iter, dot):
    """Rayleigh quotient <v|A v> of the last iterate of n_iter power steps.

    v_0 = v0/|v0|; for i = 1..n_iter: w = A v_{i-1}; est = <v_{i-1}|w>; v_i = w/|w|.
    """
    v = v0 / np.sqrt(dot(v0, v0).real)
    est = None
    for _ in range(n_iter):
        w = apply_a(v)
        est = dot(v, w).real
        v = w / np.sqrt(dot(w, w).real)
    return est


def spectral_bounds(apply_h, v0, n_iter, dot, margin=0.05):
    """Shifted power iteration for [E_min, E_max] of H (Sec. 2.1).

    Returns (emin, emax) widened by margin * (emax - emin) on each side, and the
    raw estimates (emin_raw, emax_raw).
    """
    emax = power_iteration(apply_h, v0, n_iter, dot)
    shift = power_iteration(lambda v: apply_h(v) - emax * v, v0, n_iter, dot)
    emin = emax + shift
    w = emax - emin
    return (emin - margin * w, emax + margin * w), (emin, emax)


def spectrum_map(emin, emax):
    """Centre Ebar and half-width dE that map [emin, emax] onto [-1, 1]."""
    return 0.5 * (emax + emin), 0.5 * (emax - emin)


# ---------------------------------------------------------------- gapped filter (Eq. 3)
def gapped_filter_coeffs(e_homo, e_lumo, emin, emax, n_cheb, ridge=1e-8):
    """Coefficients a_0..a_{N_chb} of the gapped Heaviside filter (Eq. 3).

    Nodes: the M = 4 (N_chb + 1) Chebyshev-Gauss points x_m = cos(pi (m + 1/2) / M).
    Target: 1 at x <= x_HOMO, 0 at x >= x_LUMO; nodes strictly inside the gap get
    zero weight.  The coefficients minimise
        sum_{nodes outside the gap} (sum_n a_n T_n(x_m) - f(x_m))^2 + ridge * M * |a|^2,
    solved here with a library least-squares routine on the stacked system.
    """
    ebar, de = spectrum_map(emin, emax)
    xh = (e_homo - ebar) / de
    xl = (e_lumo - ebar) / de
    M = 4 * (n_cheb + 1)
    x = np.cos(np.pi * (np.arange(M) + 0.5) / M)
    keep = (x <= xh) | (x >= xl)
    xk = x[keep]
    f = (xk <= xh).astype(np.float64)
    A = np.cos(np.outer(np.arccos(np.clip(xk, -1, 1)), np.arange(n_cheb + 1)))  # T_n(x)
    lam = np.sqrt(ridge * M)
    As = np.vstack([A, lam * np.eye(n_cheb + 1)])
    fs = np.concatenate([f, np.zeros(n_cheb + 1)])
    a, *_ = np.linalg.lstsq(As, fs, rcond=None)
    return a


def cheb_scalar(coeffs, x):
    """sum_n c_n T_n(x) for scalar/array x in [-1, 1] (reconstructed filter)."""
    x = np.asarray(x, dtype=np.float64)
    return np.cos(np.outer(np.arccos(np.clip(x, -1, 1)), np.arange(len(coeffs)))) @ coeffs


def cheb_series(apply_ht, psi, coeffs):
    """sum_n coeffs[n] T_n(H~) psi by the three-term recurrence (coeffs may be complex)."""
    t_prev = psi
    acc = coeffs[0] * psi
    if len(coeffs) == 1:
        return acc
    t_cur = apply_ht(psi)
    acc = acc + coeffs[1] * t_cur
    for n in range(2, len(coeffs)):
        t_next = 2.0 * apply_ht(t_cur) - t_prev
        acc = acc + coeffs[n] * t_next
        t_prev, t_cur = t_cur, t_next
    return acc


def filter_occupied(apply_h, psi, coeffs, emin, emax):
    """Project white noise onto the occupied subspace: sum_n a_n T_n(H~) psi (Eq. 3)."""
    ebar, de = spectrum_map(emin, emax)
    return cheb_series(lambda v: (apply_h(v) - ebar * v) / de, psi, coeffs)


# ---------------------------------------------------------------- propagator
def propagator_coeffs(emin, emax, dt, K):
    """(2 - delta_k0) (-i)^k J_k(dE dt), k = 0..K, and the phase e^{-i Ebar dt}.

    A negative dt gives the backward propagator e^{+i H |dt|}.
    """
    ebar, de = spectrum_map(emin, emax)
    a = de * abs(dt)
    k = np.arange(K + 1)
    c = (2.0 - (k == 0)) * scipy.special.jv(k, a) * ((-1j) ** k)
    if dt < 0:
        c = np.conj(c)
    return c, np.exp(-1j * ebar * dt)


def propagate_step(apply_h, psi, emin, emax, dt, K):
    """One step psi(t + dt) = e^{-i H dt} psi with the degree-K Chebyshev expansion."""
    ebar, de = spectrum_map(emin, emax)
    c, ph = propagator_coeffs(emin, emax, dt, K)
    return ph * cheb_series(lambda v: (apply_h(v) - ebar * v) / de, psi, c)


def propagate_step_tangent(apply_h, psi, dpsi, dv, emin, emax, dt, K):
    """Forward-mode derivative of one Chebyshev step.

    For H(lam) = H + lam * dv (dv a real local potential) and psi(lam) = psi + lam * dpsi,
    returns (U psi, d/dlam [U(lam) psi(lam)] at lam = 0), obtained by differentiating
    the recurrence: t'_0 = dpsi, t'_1 = H~ dpsi + dv~ psi,
    t'_{n+1} = 2 H~ t'_n + 2 dv~ t_n - t'_{n-1}, with dv~ = dv / dE.
    """
    ebar, de = spectrum_map(emin, emax)
    c, ph = propagator_coeffs(emin, emax, dt, K)
    ht = lambda v: (apply_h(v) - ebar * v) / de
    dvt = dv / de
    t_prev, dt_prev = psi, dpsi
    acc = c[0] * psi
    dacc = c[0] * dpsi
    t_cur = ht(psi)
    dt_cur = ht(dpsi) + dvt * psi
    acc = acc + c[1] * t_cur
    dacc = dacc + c[1] * dt_cur
    for n in range(2, K + 1):
        t_next = 2.0 * ht(t_cur) - t_prev
        dt_next = 2.0 * ht(dt_cur) + 2.0 * dvt * t_cur - dt_prev
        acc = acc + c[n] * t_next
        dacc = dacc + c[n] * dt_next
        t_prev, t_cur = t_cur, t_next
        dt_prev, dt_cur = dt_cur, dt_next
    return ph * acc, ph * dacc
