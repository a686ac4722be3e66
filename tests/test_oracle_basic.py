"""Pins of the oracle's building blocks against published values, closed forms and
independent library routines (no GPU)."""
import numpy as np
import pytest
import scipy.special

from oracle import hamiltonian as ham
from oracle import sgw
from oracle.philox import philox4x32_10, philox_scalar, rademacher_words
from paper_2601_21005_gb300 import synth


# ------------------------------------------------------------------ Philox
# Known-answer vectors of Philox4x32-10 published with the SC'11 paper's Random123 library
# (counter, key, expected output), stored as a text fixture.
def _kat():
    rows = []
    with open(__file__.replace('test_oracle_basic.py', 'golden/philox4x32_10_kat.txt')) as f:
        for line in f:
            if line.strip() and not line.startswith('#'):
                w = [int(x, 16) for x in line.split()]
                rows.append((w[0:4], w[4:6], w[6:10]))
    return rows


@pytest.mark.parametrize('ctr,key,want', _kat())
def test_philox_known_answers(ctr, key, want):
    assert list(philox_scalar(ctr, key)) == want
    got = philox4x32_10(*[np.array([c], dtype=np.uint32) for c in ctr], key[0], key[1])
    assert [int(g[0]) for g in got] == want


def test_philox_round_structure_matches_numpy_64bit():
    # numpy ships an independent Philox4x64-10; it increments the counter before
    # each block, so its first block is the generator at counter (1, 0, 0, 0).
    key = (0x1234567, 0x89ABCDEF)
    bg = np.random.Philox(key=np.array(key, dtype=np.uint64),
                          counter=np.zeros(4, dtype=np.uint64))
    raw = [int(x) for x in bg.random_raw(8)]
    assert raw[:4] == list(philox_scalar((1, 0, 0, 0), key, width=64))
    assert raw[4:] == list(philox_scalar((2, 0, 0, 0), key, width=64))


def test_white_noise_law():
    g = ham.Grid(8, 0.5)
    z = sgw.white_noise(g, 7, 1, 0, 3)
    assert np.allclose(np.abs(z), 1 / np.sqrt(g.dV))
    # different vectors / samples / streams are different draws
    z2 = sgw.white_noise(g, 7, 1, 1, 1)
    assert not np.array_equal(z[0], z2[0])
    assert not np.array_equal(z[0], z[1])
    s = rademacher_words(99, 0, 0, 0, 1 << 16).astype(float)
    assert abs(s.mean()) < 5 / np.sqrt(len(s))
    # E[zeta zeta^T] = I / dV: off-diagonal sample correlation is O(1/sqrt(N))
    c = np.mean(s[:-1] * s[1:])
    assert abs(c) < 5 / np.sqrt(len(s))


# ------------------------------------------------------------------ grid and Hamiltonian
def _analytic_kinetic_matrix(n, h):
    """T_{jj'} = (1/N) sum_k |k|^2/2 e^{i k (r_j - r_j')} on the periodic grid."""
    g = ham.Grid(n, h)
    N = g.ng
    idx = np.arange(N)
    z, y, x = idx // (n * n), (idx // n) % n, idx % n
    m = np.fft.fftfreq(n) * n
    kz, ky, kx = np.meshgrid(m, m, m, indexing='ij')
    kk = 2 * np.pi / (n * h)
    T = np.zeros((N, N), dtype=np.complex128)
    for a, b, c, tk in zip(kz.ravel(), ky.ravel(), kx.ravel(), 0.5 * kk ** 2 * (kz ** 2 + ky ** 2 + kx ** 2).ravel()):
        ph = np.exp(2j * np.pi * (a * z + b * y + c * x) / n)
        T += tk * np.outer(ph, np.conj(ph)) / N
    return T


def test_dense_h_matches_analytic_kinetic_plus_potential():
    n, h = 4, 0.7
    g = ham.Grid(n, h)
    rng = np.random.default_rng(0)
    v = rng.normal(size=g.shape())
    H = ham.dense_h(g, v)
    ref = _analytic_kinetic_matrix(n, h) + np.diag(v.ravel())
    assert np.max(np.abs(H - ref)) < 1e-12


def test_plane_wave_is_kinetic_eigenvector():
    n, h = 12, 0.5
    g = ham.Grid(n, h)
    Z, Y, X = synth.grid_coords(n, h)
    k = 2 * np.pi / g.L * np.array([2, -3, 1])
    pw = np.exp(1j * (k[0] * X + k[1] * Y + k[2] * Z))
    out = ham.apply_h(pw, g, np.zeros(g.shape()))
    assert np.max(np.abs(out - 0.5 * k @ k * pw)) < 1e-11


def test_kinetic_cutoff_caps_energy():
    g = ham.Grid(8, 0.5, ecut=5.0)
    assert g.T.max() == pytest.approx(5.0)
    assert np.all(g.T <= 5.0)


def _small_system(n=10, h=0.6, seed=3):
    g = ham.Grid(n, h)
    rng = np.random.default_rng(seed)
    v = synth.gaussian_wells_potential(n, h, [tuple(rng.uniform(0, n * h, 3)) for _ in range(2)],
                                       [2.0, 1.5], [1.0, 1.0])
    c = tuple(rng.uniform(2, n * h - 2, 3))
    kb = ham.KB([synth.kb_projectors(n, h, c, 0.6, (0.8, -0.3), 1)])
    return g, v, kb


def test_h_is_hermitian_with_kb():
    g, v, kb = _small_system()
    rng = np.random.default_rng(1)
    a = rng.normal(size=g.shape()) + 1j * rng.normal(size=g.shape())
    b = rng.normal(size=g.shape()) + 1j * rng.normal(size=g.shape())
    lhs = g.dot(a, ham.apply_h(b, g, v, kb))
    rhs = np.conj(g.dot(b, ham.apply_h(a, g, v, kb)))
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def test_kb_apply_matches_dense_projector_sum():
    g, v, kb = _small_system()
    N = g.ng
    P = np.zeros((N, N))
    for sup, beta, e in kb.atoms:
        for p in range(beta.shape[0]):
            col = np.zeros(N)
            col[sup] = beta[p]
            P += e[p] * g.dV * np.outer(col, col)
    rng = np.random.default_rng(2)
    psi = rng.normal(size=g.shape()) + 1j * rng.normal(size=g.shape())
    assert np.allclose(kb.apply(psi, g).ravel(), P @ psi.ravel(), atol=1e-12)
    # projectors are normalised on the grid
    for sup, beta, e in kb.atoms:
        assert np.allclose(g.dV * np.sum(beta * beta, axis=1), 1.0)


# ------------------------------------------------------------------ Poisson
def test_poisson_cosine_closed_form():
    n, h = 16, 0.5
    g = ham.Grid(n, h)
    Z, Y, X = synth.grid_coords(n, h)
    k = 2 * np.pi / g.L * np.array([1, 2, 0])
    rho = np.cos(k[0] * X + k[1] * Y)
    v = ham.poisson(rho, g).real
    assert np.max(np.abs(v - 4 * np.pi / (k @ k) * rho)) < 1e-12


def test_poisson_gaussian_pair_energy():
    """Two opposite Gaussian charges (width s, distance d): closed-form Hartree energy
    E = q^2/(s sqrt(pi)) - q^2 erf(d/(2 s))/d; the periodic images add a dipole term
    of order 2 pi p^2 / (3 L^3), which bounds the tolerance."""
    n, h = 64, 0.4
    g = ham.Grid(n, h)
    Z, Y, X = synth.grid_coords(n, h)
    s, d, q = 0.8, 2.0, 1.0
    c = 0.5 * g.L
    def gauss(x0):
        r2 = (X - x0) ** 2 + (Y - c) ** 2 + (Z - c) ** 2
        return q * np.exp(-r2 / (2 * s * s)) / (2 * np.pi * s * s) ** 1.5
    rho = gauss(c - d / 2) - gauss(c + d / 2)
    v = ham.poisson(rho, g).real
    E = 0.5 * g.dV * np.sum(rho * v)
    ref = q * q / (s * np.sqrt(np.pi)) - q * q * scipy.special.erf(d / (2 * s)) / d
    p = q * d
    tol = 2 * (2 * np.pi * p * p / (3 * g.L ** 3)) + 1e-6
    assert abs(E - ref) < tol
