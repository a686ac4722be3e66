"""Pins of the split-operator oracle: the kinetic factor against the dense eigendecomposition,
one atom's KB factor against scipy's matrix exponential of the dense operator, second-order
convergence to the exact propagator with local and KB parts, unitarity, time reversibility,
the colouring rule, and its accuracy next to the degree-16 Chebyshev step (no GPU)."""
import numpy as np
import pytest

from oracle import chebyshev as cheb
from oracle import hamiltonian as ham
from oracle import splitop
from paper_2601_21005_gb300 import synth

scipy_linalg = pytest.importorskip('scipy.linalg')


def _system(n=10, h=0.6):
    g = ham.Grid(n, h)
    L = n * h
    centers = [(0.3 * L, 0.35 * L, 0.4 * L), (0.45 * L, 0.4 * L, 0.42 * L), (0.75 * L, 0.7 * L, 0.65 * L)]
    v = synth.gaussian_wells_potential(n, h, centers, [1.5, 1.0, 2.0], [0.8, 0.7, 0.9])
    atoms = [synth.kb_projectors(n, h, c, 0.35, (0.8, -0.3), 1) for c in centers]
    return g, v, atoms


def _exact(H, psi, t):
    lam, w = np.linalg.eigh(H)
    return w @ (np.exp(-1j * t * lam) * (w.conj().T @ psi.reshape(-1)))


def test_kinetic_factor_is_exact():
    g, v, atoms = _system()
    psi = np.random.default_rng(1).normal(size=g.shape()) + 0j
    got = splitop.split_step(psi, g, np.zeros(g.shape()), None, 0.07)
    H = ham.dense_h(g, np.zeros(g.shape()))
    assert np.allclose(got.reshape(-1), _exact(H, psi, 0.07), atol=1e-12)


def test_single_atom_factor_matches_expm():
    g, v, atoms = _system()
    kbs = splitop.KBSplit(atoms[:1], g)
    s, beta, e = atoms[0]
    Va = np.zeros((g.ng, g.ng))
    Va[np.ix_(s, s)] = g.dV * beta.T @ np.diag(e) @ beta          # dV sum_p beta_p E_p beta_p^T
    psi = np.random.default_rng(2).normal(size=g.ng) + 1j * np.random.default_rng(3).normal(size=g.ng)
    tau = 0.31
    want = scipy_linalg.expm(-1j * tau * Va) @ psi
    got = kbs.apply(psi.reshape(g.shape()), tau, descending=False).reshape(-1)
    assert np.max(np.abs(got - want)) < 1e-12


def test_colouring_rule():
    g, v, atoms = _system()
    kbs = splitop.KBSplit(atoms, g)
    # atoms 0 and 1 overlap, atom 2 is far from both
    assert len(set(atoms[0][0]) & set(atoms[1][0])) > 0 and not set(atoms[2][0]) & set(atoms[0][0])
    assert kbs.colour == [0, 1, 0] and kbs.n_colours == 2


def test_second_order_convergence_unitarity_and_reversibility():
    g, v, atoms = _system()
    kb = ham.KB(atoms)
    kbs = splitop.KBSplit(atoms, g)
    H = ham.dense_h(g, v, kb)
    rng = np.random.default_rng(4)
    psi = rng.normal(size=g.shape()) + 1j * rng.normal(size=g.shape())
    t = 0.4
    ref = _exact(H, psi, t)
    errs = []
    for n_steps in (4, 8, 16):
        got = splitop.split_propagate(psi, g, v, kbs, t / n_steps, n_steps).reshape(-1)
        errs.append(np.linalg.norm(got - ref) / np.linalg.norm(ref))
    assert 3.3 < errs[0] / errs[1] < 4.7 and 3.3 < errs[1] / errs[2] < 4.7       # O(dt^2)
    one = splitop.split_step(psi, g, v, kbs, 0.05)
    assert abs(np.linalg.norm(one) / np.linalg.norm(psi) - 1) < 1e-13
    back = splitop.split_step(one, g, v, kbs, -0.05)
    assert np.max(np.abs(back - psi)) < 1e-12 * np.max(np.abs(psi))


def test_accuracy_next_to_the_chebyshev_step():
    """At dt = 0.05 the degree-16 Chebyshev step is exact to rounding; the split step carries the
    O(dt^3) local splitting error (printed for the design notes)."""
    g, v, atoms = _system()
    kb = ham.KB(atoms)
    kbs = splitop.KBSplit(atoms, g)
    H = ham.dense_h(g, v, kb)
    lam = np.linalg.eigvalsh(H)
    lo, hi = lam[0] - 0.05 * (lam[-1] - lam[0]), lam[-1] + 0.05 * (lam[-1] - lam[0])
    psi = np.random.default_rng(5).normal(size=g.shape()) + 0j
    ref = _exact(H, psi, 0.05)
    e_split = np.linalg.norm(splitop.split_step(psi, g, v, kbs, 0.05).reshape(-1) - ref) / np.linalg.norm(ref)
    e_cheb = np.linalg.norm(cheb.propagate_step(lambda x: ham.apply_h(x, g, v, kb), psi, lo, hi, 0.05, 16).reshape(-1)
                            - ref) / np.linalg.norm(ref)
    print('one step dt = 0.05: split-operator error %.2e, Chebyshev-16 error %.2e' % (e_split, e_cheb))
    assert e_cheb < 1e-11 and 1e-7 < e_split < 1e-2


def test_tangent_step_is_the_derivative():
    g, v, atoms = _system()
    kbs = splitop.KBSplit(atoms, g)
    rng = np.random.default_rng(6)
    psi = rng.normal(size=g.shape()) + 1j * rng.normal(size=g.shape())
    dpsi = rng.normal(size=g.shape()) + 1j * rng.normal(size=g.shape())
    dv = rng.normal(size=g.shape())
    _, got = splitop.split_step_tangent(psi, dpsi, g, v, dv, kbs, 0.05)
    h = 1e-5
    fd = (splitop.split_step(psi + h * dpsi, g, v + h * dv, kbs, 0.05)
          - splitop.split_step(psi - h * dpsi, g, v - h * dv, kbs, 0.05)) / (2 * h)
    assert np.max(np.abs(got - fd)) < 1e-8 * np.max(np.abs(fd))
    x, _ = splitop.split_step_tangent(psi, dpsi, g, v, dv, kbs, 0.05)
    assert np.allclose(x, splitop.split_step(psi, g, v, kbs, 0.05), atol=1e-14)


def test_split_tdh_and_sigma_converge_to_the_chebyshev_ones():
    """With the same inputs, the TDH response and Sigma(t) of the split-operator stepper approach
    those of the (exact-per-step) Chebyshev stepper as dt^2 at a fixed final time."""
    from oracle import sgw as osgw
    g, v, atoms = _system()
    kb = ham.KB(atoms)
    kbs = splitop.KBSplit(atoms, g)
    H = ham.dense_h(g, v, kb)
    lam, w = np.linalg.eigh(H)
    lo, hi = lam[0] - 1.0, lam[-1] + 1.0
    phi = w[:, 2].real.reshape(g.shape()) / np.sqrt(g.dV)
    prob = osgw.Problem(g, v, kb, lo, hi, lam[1], lam[2], phi)
    rng = np.random.default_rng(7)
    eta = np.stack([(w[:, :2] @ rng.normal(size=2)).reshape(g.shape()) for _ in range(2)])
    src = np.sign(rng.normal(size=g.shape())) * phi
    t = 0.4
    diffs = []
    for n in (8, 16):
        a = osgw.tdh_response_tangent(prob, eta, src, n, t / n, 16)
        b = osgw.tdh_response_tangent(prob, eta, src, n, t / n, 16, split=kbs)
        diffs.append(np.linalg.norm(a[-1] - b[-1]) / np.linalg.norm(a[-1]))
    assert 3.0 < diffs[0] / diffs[1] < 5.0
    zo = eta[0]
    zu = src - zo
    sd = []
    for n in (8, 16):
        u = np.stack([np.cos(2.0 * j * t / n) * phi for j in range(n + 1)]).astype(np.complex128)
        a = osgw.sigma_t(prob, zo, zu, u, n, t / n, 16)
        b = osgw.sigma_t(prob, zo, zu, u, n, t / n, 16, split=kbs)
        sd.append(abs(a[-1] - b[-1]) + abs(a[0] - b[0]))        # Sigma(+-t) at the final time
    assert 3.0 < sd[0] / sd[1] < 5.0
