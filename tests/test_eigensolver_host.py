"""The harness's interior eigensolver (states next to the gap, for systems too large to hold every
occupied state) on the CPU: its Chebyshev series pinned by exact eigenvalues and by numpy's own
Chebyshev evaluation, and the whole solver, run through a stand-in context whose calls the FP64
oracle answers, against dense diagonalisation of the 16^3 wells (no GPU)."""
import numpy as np
import pytest

from oracle import chebyshev as cheb
from oracle import hamiltonian as ham
from oracle import sgw as osgw
from paper_2601_21005_gb300 import eigensolver as es
from paper_2601_21005_gb300 import synth

torch = pytest.importorskip('torch')


@pytest.fixture(scope='module')
def wells():
    s = synth.wells()
    g = ham.Grid(s['n'], s['h'])
    H = ham.dense_h(g, s['vloc']).real
    w, V = np.linalg.eigh(0.5 * (H + H.T))
    (lo, hi), _ = cheb.spectral_bounds(lambda v: ham.apply_h(v, g, s['vloc']), np.ones(g.shape(), dtype=complex),
                                       100, g.dot)
    return s, g, w, V, lo, hi


def test_step_series_counts_the_states_below(wells):
    s, g, w, V, lo, hi = wells
    c, h = 0.5 * (hi + lo), 0.5 * (hi - lo)
    for n_below in (4, 9):
        e = 0.5 * (w[n_below - 1] + w[n_below])                       # mid-gap between two levels
        coef = es.step_coeffs(e, lo, hi, 2000)
        count = np.sum(np.polynomial.chebyshev.chebval((w - c) / h, coef))
        assert abs(count - n_below) < 0.05, (n_below, count)


def test_gaussian_series_matches_the_gaussian():
    lo, hi, center, sigma = -3.0, 40.0, 1.3, 0.8
    coef = es.gaussian_coeffs(center, sigma, lo, hi, 400)
    e = np.linspace(lo, hi, 2001)
    x = (e - 0.5 * (hi + lo)) / (0.5 * (hi - lo))
    ref = np.exp(-(e - center) ** 2 / (2 * sigma ** 2))
    assert np.max(np.abs(np.polynomial.chebyshev.chebval(x, coef) - ref)) < 1e-8


class OracleCtx:
    """The context calls the eigensolver makes, answered by the FP64 oracle on CPU tensors."""

    def __init__(self, s, g):
        self.s, self.g = s, g
        self.ng, self.dV, self.device = g.ng, g.dV, None
        self.lo = self.hi = None

    def _h(self, v):
        return ham.apply_h(v, self.g, self.s['vloc'])

    def white_noise(self, seed, stream, sample0, n_samples, n_vec, out):
        assert n_samples == 1
        w = osgw.white_noise(self.g, seed, stream, sample0, n_vec)
        out.copy_(torch.from_numpy(w.reshape(n_vec, -1).astype(np.complex64)))

    def set_spectrum(self, lo, hi):
        self.lo, self.hi = lo, hi

    def apply_h(self, X, Y):
        x = X.numpy().reshape((-1,) + self.g.shape()).astype(np.complex128)
        Y.copy_(torch.from_numpy(self._h(x).reshape(X.shape).astype(np.complex64)))

    def filter_occupied(self, coeffs, X, out):
        x = X.numpy().reshape((-1,) + self.g.shape()).astype(np.complex128)
        y = cheb.filter_occupied(self._h, x, np.asarray(coeffs), self.lo, self.hi)
        out.copy_(torch.from_numpy(y.reshape(X.shape).astype(np.complex64)))


def test_moments_count_and_gap(wells):
    """Probe moments through the stand-in context: the estimated count at mid-gap is n_occ within
    its standard error, and the density minimum compatible with 4 states lies in the HOMO-LUMO gap."""
    s, g, w, V, lo, hi = wells
    ctx = OracleCtx(s, g)
    mu = es.cheb_moments(ctx, lo, hi, n_probe=64, degree=600, device=torch.device('cpu'))
    assert np.allclose(mu[:, 0], g.ng, rtol=1e-6)                     # T_0 = 1: dV <v|v> = N_g
    n, se, dos = es.count_and_dos(mu, [0.5 * (w[3] + w[4])], lo, hi)
    assert abs(n[0] - 4) < 4 * se[0] + 0.05
    e, n_e, se_e = es.find_gap(mu, 4, lo, hi)
    assert w[3] < e < w[4]


def test_states_near_gap_match_dense_diagonalisation(wells):
    s, g, w, V, lo, hi = wells
    ctx = OracleCtx(s, g)
    e_h, e_l, phi, info = es.states_near_gap(ctx, 4, lo, hi, m=8, sigma=0.4, n_probe=64, count_degree=600,
                                             window_degree=300, max_iter=80, tol=1e-4, device=torch.device('cpu'))
    assert w[3] < info['gap_centre'] < w[4]
    assert abs(e_h - w[3]) < 1e-5 and abs(e_l - w[4]) < 1e-5
    ref = V[:, 3] / np.sqrt(g.dV)
    assert abs(g.dV * np.dot(phi.ravel(), ref)) > 0.999
