"""Pins of the xi-compression oracle: the gather projection against the dense definition, the
resolution of the identity in expectation (Monte Carlo over samples), exact reconstruction in the
full-rank limit structure, and unbiasedness of the compressed Sigma(t) (no GPU)."""
import numpy as np

from oracle import hamiltonian as ham
from oracle import xi


def test_projection_matches_the_dense_definition():
    g = ham.Grid(4, 0.5)                        # 64 points, segments of 8
    f = np.random.default_rng(1).normal(size=(3, g.ng))
    for sample in (0, 5):
        X = xi.dense(g, 11, 7, sample, 6, 0.25, 8)
        U = xi.project(f, g, 11, 7, sample, 6, 0.25, 8)
        assert np.allclose(U, g.dV * f @ X.T, atol=1e-12)
        back = xi.reconstruct(U, g, 11, 7, sample, 6, 0.25, 8)
        assert np.allclose(back, U @ X, atol=1e-12)


def test_identity_in_expectation():
    """dV sum_m xi_m xi_m^T averaged over many samples tends to the identity: diagonal 1 and
    off-diagonal 0 within a few standard errors of the Monte-Carlo mean."""
    g = ham.Grid(4, 0.5)
    n = 3000
    acc = np.zeros((g.ng, g.ng))
    acc2 = np.zeros((g.ng, g.ng))
    for s in range(n):
        X = xi.dense(g, 3, 9, s, 4, 0.25, 8)
        A = g.dV * X.T @ X
        acc += A
        acc2 += A * A
    mean = acc / n
    se = np.sqrt(np.maximum(acc2 / n - mean ** 2, 1e-30) / n)
    dev = np.abs(mean - np.eye(g.ng)) / se
    assert np.max(dev) < 5.0
    assert abs(np.mean(np.diag(mean)) - 1.0) < 0.02


def test_compressed_overlap_is_unbiased():
    """<a|u> through the xi basis, sum_m <a|xi_m> <xi_m|u>, averages to <a|u>."""
    g = ham.Grid(4, 0.5)
    rng = np.random.default_rng(2)
    a, u = rng.normal(size=g.ng), rng.normal(size=g.ng)
    exact = g.dV * a @ u
    vals = []
    for s in range(4000):
        Ua = xi.project(a, g, 5, 9, s, 4, 0.25, 8)
        Uu = xi.project(u, g, 5, 9, s, 4, 0.25, 8)
        vals.append(np.sum(Ua * Uu))
    vals = np.array(vals)
    assert abs(vals.mean() - exact) < 4 * vals.std() / np.sqrt(len(vals))


def test_number_of_draws_rounds_halves_up():
    # N_g f_g / L = 4.5 and 5.5 round to 5 and 6 (not to the even neighbour); at least one draw
    assert xi.n_draws(4096, 4.5 * 32 / 4096, 32) == 5
    assert xi.n_draws(4096, 5.5 * 32 / 4096, 32) == 6
    assert xi.n_draws(4096, 6.4 * 32 / 4096, 32) == 6
    assert xi.n_draws(4096, 1e-9, 32) == 1
