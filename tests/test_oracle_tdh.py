"""Pins of the oracle's linear-response TDH step and of the assembled Sigma(t) (no GPU).

* the tangent-linear pair equals the paper's perturbed-minus-unperturbed pair to O(lambda);
* with the exact occupied orbitals in place of the stochastic eta, the TDH response equals
  the Casida RPA response (dense solve), with an O(dt) error from holding H over a step;
* averaged over a complete set of source vectors, the sampled Sigma(t) equals the
  sum-over-states G0W0 Sigma(t) built from the RPA poles and the KS eigenstates
  (same discrete time ordering), which fixes the signs and factors of Eq. 4 and Eq. 5.
"""
import numpy as np
import pytest

from oracle import chebyshev as cheb
from oracle import hamiltonian as ham
from oracle import sgw
from paper_2601_21005_gb300 import synth

from rpa_reference import casida, eigenstates, induced_potential_modes


def _tiny(n, h, centers, depths, widths=(1.0, 1.0)):
    g = ham.Grid(n, h)
    v = synth.gaussian_wells_potential(n, h, centers, depths, list(widths))
    w, phis = eigenstates(g, v)
    lo, hi = w[0] - 0.05 * (w[-1] - w[0]), w[-1] + 0.05 * (w[-1] - w[0])
    return g, v, w, phis, lo, hi


@pytest.fixture(scope='module')
def sys8():
    return _tiny(8, 0.7, [(1.5, 2.0, 2.5), (4.0, 3.5, 3.0)], [3.0, 2.5])


def test_tangent_pair_equals_finite_kick_pair(sys8):
    g, v, w, phis, lo, hi = sys8
    n_occ = 2
    prob = sgw.Problem(g, v, None, lo, hi, w[n_occ - 1], w[n_occ], phis[0])
    rng = np.random.default_rng(0)
    eta = phis[:n_occ] * (1 + 0.1 * rng.normal(size=(n_occ,) + g.shape()))   # not eigenstates
    src = sgw.white_noise(g, 5, 0, 0, 1)[0] * phis[0]
    a = sgw.tdh_response_tangent(prob, eta, src, 12, 0.05, 16)
    b = sgw.tdh_response_fd(prob, eta, src, 12, 0.05, 16, lam=1e-5)
    scale = np.max(np.abs(a))
    assert scale > 0
    assert np.max(np.abs(a - b)) < 1e-3 * scale
    c = sgw.tdh_response_fd(prob, eta, src, 12, 0.05, 16, lam=1e-4)
    # first order in lambda: the error grows ~10x with a 10x larger kick
    e5, e4 = np.max(np.abs(a - b)), np.max(np.abs(a - c))
    assert 3 < e4 / e5 < 30


def test_deterministic_tdh_matches_casida_rpa(sys8):
    g, v, w, phis, lo, hi = sys8
    n_occ = 2
    prob = sgw.Problem(g, v, None, lo, hi, w[n_occ - 1], w[n_occ], phis[0])
    om, rho = casida(g, w, phis, n_occ)
    src = phis[0] * phis[3] + 0.5 * phis[1] * phis[5]          # a smooth source
    vp = ham.poisson(src, g).real
    proj = g.dV * np.einsum('sxyz,xyz->s', rho, vp)            # <rho_s|v_p>
    errs = []
    T = 1.0
    for dt in (0.05, 0.025):
        ns = int(round(T / dt))
        uR = sgw.tdh_response_tangent(prob, phis[:n_occ].astype(complex), src, ns, dt, 16, weight=2.0)
        t = dt * np.arange(ns + 1)
        got = g.dV * np.einsum('txyz,xyz->t', uR, src)
        ref = -2.0 * np.sin(np.outer(t, om)) @ (proj * proj)
        errs.append(np.max(np.abs(got - ref)) / np.max(np.abs(ref)))
    assert errs[1] < 0.02
    assert 1.6 < errs[0] / errs[1] < 2.4          # first order in dt


@pytest.mark.slow
def test_sampled_sigma_equals_sum_over_states_g0w0():
    n, h = 6, 0.8
    g, v, w, phis, lo, hi = _tiny(n, h, [(1.2, 1.5, 2.0), (3.2, 2.8, 2.6)], [3.0, 2.5])
    n_occ = 1
    phi = phis[0]
    prob = sgw.Problem(g, v, None, lo, hi, w[n_occ - 1], w[n_occ], phi)
    dt, ns, K = 0.02, 25, 16
    # --- reference: sum over RPA poles and KS states, with the same discrete time ordering
    om, rho = casida(g, w, phis, n_occ)
    wm = induced_potential_modes(g, rho).reshape(len(om), -1)        # [S, N]
    t = dt * np.arange(ns + 1)
    WR = -2.0 * np.einsum('ts,sr,sm->trm', np.sin(np.outer(t, om)), wm, wm)   # W_c^R(r, m, t)
    TOW = sgw.time_order(WR)                                            # [t, r, m]
    ph = phis.reshape(len(w), -1)
    f = phi.reshape(-1)
    ref = np.zeros(2 * ns + 1, dtype=complex)
    for j in range(ns + 1):
        gp = np.einsum('a,ar,am->rm', np.exp(-1j * w[n_occ:] * t[j]), ph[n_occ:], ph[n_occ:])
        gm = np.einsum('a,ar,am->rm', np.exp(+1j * w[:n_occ] * t[j]), ph[:n_occ], ph[:n_occ])
        sp = g.dV ** 2 * np.einsum('r,m,rm,rm->', f, f, gp, TOW[j])
        sm = -g.dV ** 2 * np.einsum('r,m,rm,rm->', f, f, gm, TOW[j])
        if j == 0:
            ref[ns] = 0.5 * (sp + sm)
        else:
            ref[ns + j], ref[ns - j] = sp, sm
    # --- oracle pipeline over the complete basis zeta-bar_m = sqrt(N/dV) e_m (exact E[.])
    P = ph[:n_occ].T @ ph[:n_occ] * g.dV                               # occupied projector
    acc = np.zeros(2 * ns + 1, dtype=complex)
    N = g.ng
    for m in range(N):
        zbar = np.zeros(N)
        zbar[m] = np.sqrt(N / g.dV)
        zocc = (P @ zbar).reshape(g.shape())
        zbar = zbar.reshape(g.shape())
        uR = sgw.tdh_response_tangent(prob, phis[:n_occ].astype(complex), zbar * phi, ns, dt, K, weight=2.0)
        u = sgw.time_order(uR)
        acc += sgw.sigma_t(prob, zocc, zbar - zocc, u, ns, dt, K)
    got = acc / N
    rel = np.max(np.abs(got - ref)) / np.max(np.abs(ref))
    assert rel < 0.02
    # the occupied (t < 0) and unoccupied (t > 0) halves are each matched, including sign
    assert np.sum((got[:ns] * np.conj(ref[:ns])).real) > 0
    assert np.sum((got[ns + 1:] * np.conj(ref[ns + 1:])).real) > 0
