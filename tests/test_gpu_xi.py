"""The xi-compressed path on the GPU against the oracle: U_m(t_j) = <xi_m|u^R(t_j)> from the TDH
response, its time ordering, and Sigma(t) from the time-ordered U, with the same Philox draws.
Tolerances as for the full-grid forms (the projection adds K L-term FP32 sums per function)."""
import numpy as np
import pytest

from oracle import chebyshev as cheb
from oracle import sgw as osgw
from oracle import xi as oxi
from paper_2601_21005_gb300 import build, synth

import gpu_common as gc

torch = pytest.importorskip('torch')
pytestmark = pytest.mark.gpu

XI = dict(seed=77, stream=0x5A11, n_xi=96, f_g=0.05, L=32)


def _xi_tuple(sample0):
    return (XI['seed'], XI['stream'], sample0, XI['n_xi'], XI['f_g'], XI['L'])


def test_xi_tdh_time_order_and_sigma():
    build.build()
    from paper_2601_21005_gb300 import sgw
    s = synth.wells()
    g, kb, w, phis = gc.oracle_eigs(s, 8)
    lo, hi = -4.0, 45.0
    n_s, n_eta, N, sample0 = 2, 3, 10, 5
    prob = osgw.Problem(g, s['vloc'], None, lo, hi, w[3], w[4], phis[3])
    rng = np.random.default_rng(9)
    eta = (0.05 * (rng.normal(size=(n_s, n_eta) + g.shape()) + 1j * rng.normal(size=(n_s, n_eta) + g.shape()))
           ).astype(np.complex64)
    src = (np.sign(rng.normal(size=(n_s,) + g.shape())) * phis[3]).astype(np.float32)
    c = sgw.Context(s['n'], s['h'], max_batch=2 * n_s * n_eta)
    c.set_potential(gc.to_dev(s['vloc'].ravel(), torch, torch.float32), [])
    c.set_spectrum(lo, hi)
    nx = XI['n_xi']
    U = torch.empty(n_s, N + 1, nx, dtype=torch.float32, device='cuda')
    c.tdh_response_xi(gc.to_dev(eta.reshape(n_s * n_eta, -1), torch, torch.complex64),
                      gc.to_dev(src.reshape(n_s, -1), torch, torch.float32), n_s, n_eta, N, 0.05, 16,
                      _xi_tuple(sample0), U)
    Ug = U.cpu().numpy()
    Uref = []
    for si in range(n_s):
        uR = osgw.tdh_response_tangent(prob, eta[si].astype(np.complex128), src[si].astype(np.float64), N, 0.05, 16)
        Ur = oxi.project(uR.reshape(N + 1, -1), g, XI['seed'], XI['stream'], sample0 + si, nx, XI['f_g'], XI['L'])
        Uref.append(Ur)
        assert gc.rel_err(Ug[si], Ur) < 3e-4
    # time ordering of the compressed series
    Uto = torch.empty(n_s, N + 1, nx, dtype=torch.complex64, device='cuda')
    c.time_order_points(U, Uto, n_s, N, nx)
    Utog = Uto.cpu().numpy()
    for si in range(n_s):
        ref = osgw.time_order(Ug[si].astype(np.float64))
        assert gc.rel_err(Utog[si], ref) < 2e-6
    # Sigma(t) in the xi basis against the oracle's Sigma(t) on the reconstructed u
    zeta = (rng.normal(size=(n_s, 2) + g.shape()) + 1j * rng.normal(size=(n_s, 2) + g.shape())).astype(np.complex64)
    phi = phis[3].astype(np.float32)
    sig = torch.empty(n_s, 2 * N + 1, dtype=torch.complex128, device='cuda')
    c.sigma_c_xi(gc.to_dev(zeta.reshape(2 * n_s, -1), torch, torch.complex64), gc.to_dev(phi.ravel(), torch, torch.float32),
                 Uto, n_s, N, 0.05, 16, _xi_tuple(sample0), sig, 1)
    got = sig.cpu().numpy()
    for si in range(n_s):
        urec = oxi.reconstruct(Utog[si].astype(np.complex128), g, XI['seed'], XI['stream'], sample0 + si, nx,
                               XI['f_g'], XI['L']).reshape((N + 1,) + g.shape())
        ref = osgw.sigma_t(prob, zeta[si, 0].astype(np.complex128), zeta[si, 1].astype(np.complex128), urec, N, 0.05, 16)
        assert gc.rel_err(got[si], ref) < 3e-4


def test_xi_arguments_are_checked():
    build.build()
    from paper_2601_21005_gb300 import sgw
    s = synth.wells()
    c = sgw.Context(s['n'], s['h'], max_batch=4)
    c.set_potential(gc.to_dev(s['vloc'].ravel(), torch, torch.float32), [])
    c.set_spectrum(-4.0, 45.0)
    eta = torch.zeros(2, c.ng, dtype=torch.complex64, device='cuda')
    src = torch.zeros(1, c.ng, dtype=torch.float32, device='cuda')
    U = torch.empty(1, 3, 8, dtype=torch.float32, device='cuda')
    for bad in ((1, 2, 0, 0, 0.1, 32), (1, 2, 0, 8, 0.0, 32), (1, 2, 0, 8, 0.1, 33), (1, 2, 0, 8, 0.1, 24),
                (1, 2, -1, 8, 0.1, 32)):
        with pytest.raises(RuntimeError):
            c.tdh_response_xi(eta, src, 1, 2, 2, 0.05, 16, bad, U)


def test_pipeline_xi_sample_indexing():
    """The TDH chunks (per-chunk sample offsets) and the single Sigma call over the run (run offset)
    draw the same xi functions: two chunks of one sample equal one chunk of two samples."""
    build.build()
    from paper_2601_21005_gb300.pipeline import Pipeline
    s = synth.wells()
    g, kb, w, phis = gc.oracle_eigs(s, 8)
    out = []
    for ns, group in ((1, 2), (2, 1)):
        pl = Pipeline(s['n'], s['h'], s['vloc'], [], phis[3], w[3], w[4], n_eta=2, n_steps=6, dt=0.05, cheb_deg=16,
                      n_cheb=64, samples_per_batch=ns, zeta_group=group, spectrum=(-4.0, 45.0),
                      xi=dict(n_xi=40, f_g=0.05, L=32))
        sig, x = pl.run(2, sample0=3)
        out.append(sig.cpu().numpy())
        pl.ctx.close()
    assert gc.rel_err(out[0], out[1]) < 1e-6
