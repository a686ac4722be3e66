"""Pins of the oracle's filter, propagator, spectral bounds, time ordering, transform and
QP solve against dense diagonalisation (LAPACK eigh) and closed forms (no GPU)."""
import numpy as np
import pytest
import scipy.integrate
import scipy.optimize
import scipy.special

from oracle import chebyshev as cheb
from oracle import hamiltonian as ham
from oracle import sgw
from paper_2601_21005_gb300 import synth


@pytest.fixture(scope='module')
def small():
    """10^3 grid, two wells and one s/p KB atom; exact eigenpairs by LAPACK."""
    n, h = 10, 0.6
    g = ham.Grid(n, h)
    rng = np.random.default_rng(3)
    v = synth.gaussian_wells_potential(n, h, [tuple(rng.uniform(0, n * h, 3)) for _ in range(2)],
                                       [2.5, 2.0], [1.0, 1.0])
    kb = ham.KB([synth.kb_projectors(n, h, tuple(rng.uniform(2, n * h - 2, 3)), 0.6, (0.8, -0.3), 1)])
    H = ham.dense_h(g, v, kb)
    assert np.max(np.abs(H - H.conj().T)) < 1e-12
    w, V = np.linalg.eigh(H)
    return g, v, kb, w, V


def _rand(g, seed):
    rng = np.random.default_rng(seed)
    return rng.normal(size=g.shape()) + 1j * rng.normal(size=g.shape())


def test_spectral_bounds_enclose_spectrum(small):
    g, v, kb, w, V = small
    (lo, hi), (rlo, rhi) = cheb.spectral_bounds(lambda x: ham.apply_h(x, g, v, kb), _rand(g, 5), 300, g.dot)
    assert lo < w[0] and hi > w[-1]
    # the raw Rayleigh quotients converge from inside the spectrum
    assert rlo >= w[0] - 1e-9 and rhi <= w[-1] + 1e-9
    assert abs(rlo - w[0]) < 1e-3 * (w[-1] - w[0])
    assert (w[-1] - rhi) < 0.05 * (w[-1] - w[0])


def test_filter_equals_spectral_function_of_h(small):
    """sum_n a_n T_n(H~) psi == V diag(p(lambda)) V^+ psi, p the scalar Chebyshev sum."""
    g, v, kb, w, V = small
    emin, emax = w[0] - 0.5, w[-1] + 0.5
    ebar, de = cheb.spectrum_map(emin, emax)
    n_occ = 2
    a = cheb.gapped_filter_coeffs(w[n_occ - 1], w[n_occ], emin, emax, 200)
    psi = _rand(g, 6)
    got = cheb.filter_occupied(lambda x: ham.apply_h(x, g, v, kb), psi, a, emin, emax)
    p = cheb.cheb_scalar(a, (w - ebar) / de)
    ref = V @ (p * (V.conj().T @ psi.ravel()))
    assert np.max(np.abs(got.ravel() - ref)) < 1e-10 * np.max(np.abs(ref))


def test_filter_approaches_exact_projector(small):
    """|P~ psi - P psi| <= max_i |p(lambda_i) - Theta_i| |psi| and P~ is nearly idempotent."""
    g, v, kb, w, V = small
    emin, emax = w[0] - 0.5, w[-1] + 0.5
    ebar, de = cheb.spectrum_map(emin, emax)
    n_occ = 2
    a = cheb.gapped_filter_coeffs(w[n_occ - 1], w[n_occ], emin, emax, 400)
    theta = (np.arange(len(w)) < n_occ).astype(float)
    p = cheb.cheb_scalar(a, (w - ebar) / de)
    bound = np.max(np.abs(p - theta))
    assert bound < 0.05, 'degree 400 should resolve this gap'
    fH = lambda x: cheb.filter_occupied(lambda y: ham.apply_h(y, g, v, kb), x, a, emin, emax)
    psi = _rand(g, 7)
    P = V[:, :n_occ] @ V[:, :n_occ].conj().T
    err = np.linalg.norm(fH(psi).ravel() - P @ psi.ravel())
    assert err <= bound * np.linalg.norm(psi) * (1 + 1e-9)
    f1 = fH(psi)
    f2 = fH(f1)
    assert np.linalg.norm(f2 - f1) <= 2.5 * bound * np.linalg.norm(psi)
    # trace of the filtered projector ~ N_occ (Hutchinson estimate is exact with the eigenbasis)
    assert abs(np.sum(p) - n_occ) < len(w) * bound


def test_gapped_coeffs_are_the_ridge_least_squares_minimiser():
    """Optimality (normal equations) of the coefficients, written independently of lstsq."""
    emin, emax, eh, el, N = -3.0, 40.0, -1.0, -0.4, 150
    a = cheb.gapped_filter_coeffs(eh, el, emin, emax, N, ridge=1e-8)
    ebar, de = cheb.spectrum_map(emin, emax)
    M = 4 * (N + 1)
    x = np.cos(np.pi * (np.arange(M) + 0.5) / M)
    xh, xl = (eh - ebar) / de, (el - ebar) / de
    keep = (x <= xh) | (x >= xl)
    # T_n(x) by the three-term recurrence
    T = np.zeros((M, N + 1))
    T[:, 0] = 1
    T[:, 1] = x
    for k in range(2, N + 1):
        T[:, k] = 2 * x * T[:, k - 1] - T[:, k - 2]
    A = T[keep]
    f = (x[keep] <= xh).astype(float)
    grad = A.T @ (A @ a - f) + 1e-8 * M * a
    assert np.max(np.abs(grad)) < 1e-9 * M
    # reconstructed filter (cf. Fig. 3): flat 1 below the gap and 0 above, away from the edges
    xs = np.linspace(-1, 1, 4001)
    fx = cheb.cheb_scalar(a, xs)
    assert np.max(np.abs(fx[xs < xh - 0.05] - 1)) < 2e-2
    assert np.max(np.abs(fx[xs > xl + 0.05])) < 2e-2


def test_gapped_filter_converges_with_degree():
    """Error outside the gap falls as the degree grows (the gap is resolved once N >> 1/gap)."""
    emin, emax, eh, el = -3.0, 40.0, -1.0, -0.3
    ebar, de = cheb.spectrum_map(emin, emax)
    xs = np.cos(np.linspace(0, np.pi, 20001))
    out = (xs <= (eh - ebar) / de) | (xs >= (el - ebar) / de)
    errs = []
    for N in (100, 300, 900):
        a = cheb.gapped_filter_coeffs(eh, el, emin, emax, N)
        fx = cheb.cheb_scalar(a, xs)
        errs.append(np.max(np.abs(fx[out] - (xs[out] <= (eh - ebar) / de))))
    assert errs[2] < errs[1] < errs[0]
    assert errs[2] < 1e-3


def test_propagator_matches_exact_exponential(small):
    g, v, kb, w, V = small
    emin, emax = w[0] - 0.5, w[-1] + 0.5
    psi = _rand(g, 8)
    for dt in (0.05, -0.05):
        got = cheb.propagate_step(lambda x: ham.apply_h(x, g, v, kb), psi, emin, emax, dt, 16)
        ref = V @ (np.exp(-1j * w * dt) * (V.conj().T @ psi.ravel()))
        assert np.max(np.abs(got.ravel() - ref)) < 1e-12 * np.max(np.abs(ref))
        # unitary
        assert abs(np.linalg.norm(got) - np.linalg.norm(psi)) < 1e-12 * np.linalg.norm(psi)
    # an eigenvector acquires the phase e^{-i eps dt}
    phi = V[:, 3].reshape(g.shape())
    got = cheb.propagate_step(lambda x: ham.apply_h(x, g, v, kb), phi, emin, emax, 0.05, 16)
    assert np.max(np.abs(got - np.exp(-1j * w[3] * 0.05) * phi)) < 1e-12


def test_bessel_coefficients_reference_values():
    """J_k from scipy against the power series J_k(x) = sum_m (-1)^m (x/2)^{2m+k} / (m! (m+k)!)."""
    c, ph = cheb.propagator_coeffs(-1.0, 1.0, 1.3, 12)
    for k in range(13):
        s = sum((-1) ** m * (0.65) ** (2 * m + k) / (scipy.special.factorial(m) * scipy.special.factorial(m + k))
                for m in range(30))
        assert abs(abs(c[k]) - (1 if k == 0 else 2) * abs(s)) < 1e-15


def test_tangent_step_is_derivative_of_step(small):
    g, v, kb, w, V = small
    emin, emax = w[0] - 1.0, w[-1] + 1.0
    rng = np.random.default_rng(9)
    psi = _rand(g, 10)
    dpsi = _rand(g, 11)
    dv = rng.normal(size=g.shape()) * 0.3
    ap = lambda x: ham.apply_h(x, g, v, kb)
    u, du = cheb.propagate_step_tangent(ap, psi, dpsi, dv, emin, emax, 0.05, 16)
    eps = 1e-6
    up = cheb.propagate_step(lambda x: ap(x) + eps * dv * x, psi + eps * dpsi, emin, emax, 0.05, 16)
    um = cheb.propagate_step(lambda x: ap(x) - eps * dv * x, psi - eps * dpsi, emin, emax, 0.05, 16)
    fd = (up - um) / (2 * eps)
    assert np.max(np.abs(u - cheb.propagate_step(ap, psi, emin, emax, 0.05, 16))) < 1e-13
    assert np.max(np.abs(du - fd)) < 1e-7 * np.max(np.abs(du))


# ------------------------------------------------------------------ time ordering
def test_time_order_closed_form():
    """u^R = theta(t) sin(W t) e^{-t^2/2 tau^2} -> u = (i/2) e^{-i W |t|} e^{-t^2/2 tau^2}
    when the envelope's band (~1/tau) is far below W (Bedrosian) and the window holds it."""
    dt, nt, W, tau = 0.05, 800, 6.0, 6.0
    t = dt * np.arange(nt + 1)
    env = np.exp(-t ** 2 / (2 * tau ** 2))
    uR = np.sin(W * t) * env
    u = sgw.time_order(uR)
    ref = 0.5j * np.exp(-1j * W * t) * env
    assert np.max(np.abs(u - ref)) < 2e-3
    # exact discrete identities: Re u_j = u^R_j / 2 for j > 0, u_0 real
    assert np.max(np.abs(u.real[1:] - 0.5 * uR[1:])) < 1e-13
    # conjugating the wrong half flips the sign of the imaginary part: guard against it
    assert np.sum(u.imag[:20] * ref.imag[:20]) > 0


def test_time_order_is_linear_and_axis_batched():
    rng = np.random.default_rng(4)
    a = rng.normal(size=(41, 3))
    u = sgw.time_order(a)
    for c in range(3):
        assert np.allclose(u[:, c], sgw.time_order(a[:, c]))
    assert sgw.time_order_length(40) == 256


# ------------------------------------------------------------------ Sigma(omega), QP
def test_sigma_omega_gaussian_closed_form():
    """Sigma(t) = e^{-i e0 t} -> sqrt(2 pi)/gamma exp(-(w - e0)^2 / 2 gamma^2) for a long window."""
    dt, nt, g, e0 = 0.05, 400, 0.6, -0.3       # gamma T = 12: truncation below 1e-30
    t = dt * np.arange(-nt, nt + 1)
    s = np.exp(-1j * e0 * t)
    w = np.linspace(-1, 0.5, 31)
    got = sgw.sigma_omega(s, dt, g, w)
    ref = np.sqrt(2 * np.pi) / g * np.exp(-(w - e0) ** 2 / (2 * g * g))
    assert np.max(np.abs(got - ref)) < 1e-8


def test_sigma_omega_truncated_window_matches_quadrature():
    """With gamma T = 3 the window truncation matters; compare with adaptive quadrature of
    the trapezoid's own integrand limit plus its O(dt^2) end correction bound."""
    dt, nt, e0 = 0.05, 200, 0.2
    g = 3.0 / (nt * dt)
    t = dt * np.arange(-nt, nt + 1)
    s = np.exp(-1j * e0 * t) * (1 + 0.3 * np.cos(1.7 * t))
    T = nt * dt
    for w in (-0.5, 0.1, 0.4):
        got = sgw.sigma_omega(s, dt, g, w)[0]
        f = lambda tt: np.exp(-0.5 * g * g * tt * tt) * (1 + 0.3 * np.cos(1.7 * tt)) * np.cos((w - e0) * tt)
        ref = scipy.integrate.quad(f, -T, T, limit=400)[0]
        assert abs(got - ref) < 5e-4


def test_qp_root_single_pole():
    """Re Sigma = a / (w - b): the root of w = e + x + a/(w - b) is a quadratic's root."""
    e, x, a, b = -0.2, -0.05, 0.01, 0.3
    root = sgw.qp_root(lambda w: a / (np.asarray(w) - b), e, x, 0.0, window=0.4)
    # (w - e - x)(w - b) = a  ->  w^2 - (e + x + b) w + (e + x) b - a = 0
    c1, c0 = -(e + x + b), (e + x) * b - a
    cands = np.roots([1.0, c1, c0])
    want = cands[np.argmin(np.abs(cands - e))].real
    assert abs(root - want) < 1e-9


def test_qp_energy_gaussian_sigma_against_brentq():
    dt, nt, g, e0, c = 0.05, 400, 0.6, -0.1, 0.004   # gamma T = 12: no truncation
    t = dt * np.arange(-nt, nt + 1)
    S = [c * np.exp(-1j * e0 * t)] * 3
    e, se = sgw.qp_energy(S, [-0.02] * 3, dt, g, -0.25)
    f = lambda w: w + 0.25 + 0.02 - c * np.sqrt(2 * np.pi) / g * np.exp(-(w - e0) ** 2 / (2 * g * g))
    want = scipy.optimize.brentq(f, -0.6, 0.2, xtol=1e-14)
    assert abs(e - want) < 1e-8
    assert se == pytest.approx(0.0, abs=1e-12)


def test_standard_error_scales_as_inverse_sqrt_n():
    rng = np.random.default_rng(12)
    dt, nt, g = 0.05, 100, 0.6
    t = dt * np.arange(-nt, nt + 1)
    base = 0.003 * np.exp(0.2j * t)
    ses = []
    for n in (16, 256):
        S = [base * (1 + 0.5 * rng.normal()) for _ in range(n)]
        X = list(0.01 * rng.normal(size=n) - 0.1)
        ses.append(sgw.qp_energy(S, X, dt, g, -0.3)[1])
    assert 2.5 < ses[0] / ses[1] < 6.5
