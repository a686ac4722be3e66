"""GPU parity of the row path (grids of side 2^a 3^b: 48, 96 and 288, whose planes are split into
units of 8 x rows plus y- and z-line passes) against the FP64 oracle: H psi, the occupied filter,
the propagator, a whole MC sample through the pipeline (filter, TDH, time ordering, Sigma(t),
exchange) on a small KB cluster at 48^3, H psi at 96^3 and on the 288^3 large-cluster grid, and
the split operator refused there.  Tolerances as on the plane path (FP32 arithmetic)."""
import numpy as np
import pytest

from oracle import chebyshev as cheb
from oracle import hamiltonian as ham
from oracle import sgw as osgw
from paper_2601_21005_gb300 import build, synth

import gpu_common as gc

torch = pytest.importorskip('torch')
pytestmark = pytest.mark.gpu


@pytest.fixture(scope='module', autouse=True)
def _built():
    assert torch.cuda.is_available(), 'GPU tests need CUDA'
    build.build()


def _sgw():
    from paper_2601_21005_gb300 import sgw
    return sgw


@pytest.fixture(scope='module')
def cluster48():
    s = gc.small_cluster(n=48)                     # Si5H12 with s/p KB on Si and s on H, 24 bohr box
    g = ham.Grid(s['n'], s['h'])
    kb = ham.KB(s['kb_atoms'])
    h = lambda v: ham.apply_h(v, g, s['vloc'], kb)
    (lo, hi), _ = cheb.spectral_bounds(h, _rand_c(g.shape(), 99), 150, g.dot)
    return s, g, kb, (lo, hi)


def _ctx(s, max_batch, spectrum=None):
    c = _sgw().Context(s['n'], s['h'], max_batch=max_batch)
    c.set_potential(gc.to_dev(s['vloc'].ravel(), torch, torch.float32), s['kb_atoms'])
    if spectrum is not None:
        c.set_spectrum(*spectrum)
    return c


def _rand_c(shape, seed):
    r = np.random.default_rng(seed)
    return r.normal(size=shape) + 1j * r.normal(size=shape)


def _apply_h_check(s, g, kb, B, seed, tol):
    x = _rand_c((B,) + g.shape(), seed)
    c = _ctx(s, B)
    xd = gc.to_dev(x.reshape(B, -1), torch, torch.complex64)
    yd = torch.empty_like(xd)
    c.apply_h(xd, yd)
    got = yd.cpu().numpy()
    for b in range(B):
        ref = ham.apply_h(x[b].astype(np.complex64).astype(np.complex128), g, s['vloc'], kb)
        assert gc.rel_err(got[b].reshape(g.shape()), ref) < tol
    return c, xd, yd


def test_rows_apply_h_48(cluster48):
    s, g, kb, _ = cluster48
    c, xd, yd = _apply_h_check(s, g, kb, 3, 1, 1e-5)
    # vector by vector: a ragged batch gives the same vectors
    y1 = torch.empty_like(xd[1:2])
    c.apply_h(xd[1:2].contiguous(), y1)
    assert torch.equal(y1[0], yd[1])


def test_rows_filter_48(cluster48):
    s, g, kb, (lo, hi) = cluster48
    N, B = 100, 3
    a = cheb.gapped_filter_coeffs(-0.3, -0.1, lo, hi, N)
    c = _ctx(s, B, (lo, hi))
    noise = torch.empty(B, g.ng, dtype=torch.complex64, device='cuda')
    c.white_noise(5, 1, 0, 1, B, noise)
    out = torch.empty_like(noise)
    c.filter_occupied(a, noise, out)
    ref = cheb.filter_occupied(lambda v: ham.apply_h(v, g, s['vloc'], kb),
                               osgw.white_noise(g, 5, 1, 0, B).astype(np.complex128), a, lo, hi)
    got = out.cpu().numpy().reshape(ref.shape)
    for b in range(B):
        assert gc.rel_err(got[b], ref[b]) < 2e-6 * N


def test_rows_propagate_48(cluster48):
    s, g, kb, (lo, hi) = cluster48
    B = 4
    x = _rand_c((B,) + g.shape(), 3)
    x /= np.sqrt(np.sum(np.abs(x) ** 2, axis=(1, 2, 3), keepdims=True))
    dirs = np.array([1, -1, 1, -1], dtype=np.int8)
    c = _ctx(s, B, (lo, hi))
    h = lambda v: ham.apply_h(v, g, s['vloc'], kb)
    xd = gc.to_dev(x.reshape(B, -1), torch, torch.complex64)
    ref = x.astype(np.complex64).astype(np.complex128)
    for nsteps, tol in ((1, 1e-5), (4, 2e-5 * 5)):
        c.propagate(xd, nsteps, 0.05, 16, dirs)
        for b in range(B):
            for _ in range(nsteps):
                ref[b] = cheb.propagate_step(h, ref[b], lo, hi, 0.05 * dirs[b], 16)
        got = xd.cpu().numpy().reshape(ref.shape)
        for b in range(B):
            assert gc.rel_err(got[b], ref[b]) < tol, (nsteps, b)
            assert abs(np.linalg.norm(got[b]) - np.linalg.norm(ref[b])) < 1e-5 * np.linalg.norm(ref[b])


@pytest.fixture(scope='module')
def ks48(cluster48):
    """HOMO, LUMO and the HOMO orbital of the 48^3 cluster (16 occupied states, 0.10 Ha gap)."""
    s = cluster48[0]
    g, kb, w, phis = gc.oracle_eigs(s, s['n_occ'] + 1)
    return w[s['n_occ'] - 1], w[s['n_occ']], phis[s['n_occ'] - 1]


def test_rows_whole_sample_48(cluster48, ks48):
    """One MC sample through the pipeline (white noise, filter, exchange, TDH with KB, time
    ordering, zeta propagation and Sigma(t)) against the oracle's whole sample at equal seeds,
    with the cluster's own HOMO/LUMO and HOMO orbital."""
    from paper_2601_21005_gb300.pipeline import Pipeline
    s, g, kb, (lo, hi) = cluster48
    eh, el, phi = ks48
    a = cheb.gapped_filter_coeffs(eh, el, lo, hi, 64)
    N, n_eta = 6, 2
    pl = Pipeline(s['n'], s['h'], s['vloc'], s['kb_atoms'], phi, eh, el, n_eta=n_eta, n_steps=N, dt=0.05,
                  cheb_deg=16, samples_per_batch=1, seed=7, stream_id=1, spectrum=(lo, hi), coeffs=a)
    sig, x = pl.run(1)
    torch.cuda.synchronize()
    prob = osgw.Problem(g, s['vloc'], kb, lo, hi, eh, el, phi.astype(np.float32).astype(np.float64))
    ref, xr, _ = osgw.run_sample(prob, a, 7, 1, 0, n_eta, N, 0.05, 16)
    got = sig.cpu().numpy()[0]
    assert gc.rel_err(got, ref) < 1e-3
    assert abs(x[0].item() - xr) < 1e-4 * abs(xr)


def test_rows_apply_h_96():
    s = synth.si_cluster(n=96, h=0.5, radius=6.0)
    g = ham.Grid(s['n'], s['h'])
    _apply_h_check(s, g, ham.KB(s['kb_atoms']), 2, 4, 1e-5)


def test_rows_apply_h_288():
    """The 288^3 grid of the large cluster (23.9 M points, 191 MB per vector), one vector with the
    KB part of a small cluster at the box centre, every element against the oracle."""
    s = synth.si_cluster(n=288, h=0.5, radius=4.5)
    g = ham.Grid(s['n'], s['h'])
    _apply_h_check(s, g, ham.KB(s['kb_atoms']), 1, 5, 2e-5)


def test_rows_split_operator_refused(cluster48):
    s, g, kb, (lo, hi) = cluster48
    c = _ctx(s, 2, (lo, hi))
    x = torch.zeros(2, g.ng, dtype=torch.complex64, device='cuda')
    with pytest.raises(RuntimeError):
        c.propagate_split(x, 1, 0.05)


def _phi48(g):
    phi = synth.smooth_orbital(g.n, g.h, (12.0, 12.0, 12.0), width=2.5)
    return (phi / np.sqrt(g.dV * np.sum(phi ** 2))).astype(np.float32)


def test_rows_exchange_48(cluster48):
    s, g, kb, _ = cluster48
    n_s, n_eta = 2, 2
    eta = (0.1 * _rand_c((n_s, n_eta) + g.shape(), 7)).astype(np.complex64)
    phi = _phi48(g)
    c = _ctx(s, 2 * n_eta)
    x = torch.empty(n_s, dtype=torch.float64, device='cuda')
    c.exchange(gc.to_dev(eta.reshape(n_s * n_eta, -1), torch, torch.complex64), gc.to_dev(phi.ravel(), torch, torch.float32),
               n_s, n_eta, x)
    prob = osgw.Problem(g, s['vloc'], None, 0, 1, 0, 0, phi.astype(np.float64))
    for si in range(n_s):
        ref = osgw.exchange(prob, eta[si].astype(np.complex128))
        assert abs(x[si].item() - ref) < 1e-5 * abs(ref)


@pytest.mark.parametrize('with_kb', [False, True])
def test_rows_tdh_48(cluster48, with_kb):
    s, g, kb, (lo, hi) = cluster48
    n_s, n_eta, N = 2, 2, 3
    eta = (0.05 * _rand_c((n_s, n_eta) + g.shape(), 8)).astype(np.complex64)
    phi = _phi48(g)
    r = np.random.default_rng(9)
    src = (np.sign(r.normal(size=(n_s,) + g.shape())) * phi).astype(np.float32)
    c = _sgw().Context(s['n'], s['h'], max_batch=2 * n_s * n_eta)
    c.set_potential(gc.to_dev(s['vloc'].ravel(), torch, torch.float32), s['kb_atoms'] if with_kb else [])
    c.set_spectrum(lo, hi)
    uR = torch.empty(n_s, N + 1, g.ng, dtype=torch.float32, device='cuda')
    c.tdh_response(gc.to_dev(eta.reshape(n_s * n_eta, -1), torch, torch.complex64),
                   gc.to_dev(src.reshape(n_s, -1), torch, torch.float32), n_s, n_eta, N, 0.05, 16, uR)
    got = uR.cpu().numpy().reshape((n_s, N + 1) + g.shape())
    prob = osgw.Problem(g, s['vloc'], kb if with_kb else None, lo, hi, 0, 0, phi.astype(np.float64))
    for si in range(n_s):
        ref = osgw.tdh_response_tangent(prob, eta[si].astype(np.complex128), src[si].astype(np.float64), N, 0.05, 16)
        assert gc.rel_err(got[si], ref) < 2e-4, (si, [gc.rel_err(got[si, j], ref[j]) for j in range(N + 1)])


def test_rows_sigma_48(cluster48):
    s, g, kb, (lo, hi) = cluster48
    n_s, N = 2, 3
    zeta = _rand_c((n_s, 2) + g.shape(), 5).astype(np.complex64)
    u = (0.3 * _rand_c((n_s, N + 1) + g.shape(), 6)).astype(np.complex64)
    phi = _phi48(g)
    c = _ctx(s, 2 * n_s, (lo, hi))
    sig = torch.empty(n_s, 2 * N + 1, dtype=torch.complex128, device='cuda')
    c.sigma_c(gc.to_dev(zeta.reshape(2 * n_s, -1), torch, torch.complex64), gc.to_dev(phi.ravel(), torch, torch.float32),
              gc.to_dev(u.reshape(n_s, N + 1, -1), torch, torch.complex64), n_s, N, 0.05, 16, sig, 1)
    got = sig.cpu().numpy()
    prob = osgw.Problem(g, s['vloc'], kb, lo, hi, 0, 0, phi.astype(np.float64))
    for si in range(n_s):
        ref = osgw.sigma_t(prob, zeta[si, 0].astype(np.complex128), zeta[si, 1].astype(np.complex128),
                           u[si].astype(np.complex128), N, 0.05, 16)
        assert gc.rel_err(got[si], ref) < 2e-4
