"""The split-operator propagator on the GPU against the FP64 split-operator oracle (same scheme,
same atom colours): 32^3 cluster with KB projectors in both directions, 16^3 wells, sampled
vectors of a 64-vector batch at 64^3; unitarity, time reversibility and graph replay.

Tolerance: each step is two FP32 xy transforms and one z transform (relative ~ log2(N_g) 2^-24)
plus FP32 phases and KB factors; 1e-5 per step, so 3e-5 for three steps."""
import numpy as np
import pytest

from oracle import hamiltonian as ham
from oracle import splitop
from paper_2601_21005_gb300 import build, synth

import gpu_common as gc

torch = pytest.importorskip('torch')
pytestmark = pytest.mark.gpu


def _ctx(s, mb, stream=None):
    from paper_2601_21005_gb300 import sgw
    c = sgw.Context(s['n'], s['h'], max_batch=mb, stream=stream)
    c.set_potential(gc.to_dev(s['vloc'].ravel(), torch, torch.float32), s['kb_atoms'])
    return c


def _check(s, B, steps, dt, seed, samples=None):
    build.build()
    g = ham.Grid(s['n'], s['h'])
    kbs = splitop.KBSplit(s['kb_atoms'], g) if s['kb_atoms'] else None
    c = _ctx(s, B)
    x = torch.empty(B, g.ng, dtype=torch.complex64, device='cuda')
    c.white_noise(seed, 5, 0, 1, B, x)
    x0 = x.cpu().numpy()
    dirs = np.array([1, -1] * (B // 2), dtype=np.int8)
    c.propagate_split(x, steps, dt, dirs)
    got = x.cpu().numpy()
    for b in (range(B) if samples is None else samples):
        ref = splitop.split_propagate(x0[b].reshape(g.shape()), g, s['vloc'], kbs, dt * dirs[b], steps)
        assert gc.rel_err(got[b].reshape(g.shape()), ref) < 1e-5 * steps, b
    n0, n1 = np.linalg.norm(x0, axis=1), np.linalg.norm(got, axis=1)
    assert np.max(np.abs(n1 / n0 - 1)) < 1e-5
    # back in time: the scheme is time reversible
    c.propagate_split(x, steps, dt, -dirs)
    assert gc.rel_err(x.cpu().numpy(), x0) < 2e-5 * steps
    return c


def test_split_cluster32_with_kb():
    s = gc.small_cluster()
    assert s['kb_atoms']
    _check(s, 6, 3, 0.05, 41)


def test_split_wells16():
    _check(synth.wells(), 4, 3, 0.05, 42)


def test_split_fullsize_sampled():
    _check(synth.si_cluster(), 64, 2, 0.05, 43, samples=(0, 33, 63))


def test_split_graph_replay_is_bit_identical():
    build.build()
    s = gc.small_cluster()
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        a, b = _ctx(s, 8, st.cuda_stream), _ctx(s, 8, st.cuda_stream)
        b.set_graph_mode(True)
        xs = []
        for c in (a, b):
            x = torch.empty(8, s['n'] ** 3, dtype=torch.complex64, device='cuda')
            c.white_noise(44, 5, 0, 1, 8, x)
            for _ in range(3):
                c.propagate_split(x, 4, 0.05)
            xs.append(x)
    st.synchronize()
    assert torch.equal(xs[0], xs[1])


def test_split_tdh_and_sigma_match_the_split_oracle():
    """The TDH tangent pair and Sigma(t) with the split-operator step (cheb_deg = 0) against the
    oracle's split-operator forms, on the 32^3 cluster with KB projectors."""
    from oracle import sgw as osgw
    build.build()
    s = gc.small_cluster()
    g = ham.Grid(s['n'], s['h'])
    kb = ham.KB(s['kb_atoms'])
    kbs = splitop.KBSplit(s['kb_atoms'], g)
    rng = np.random.default_rng(8)
    n_s, n_eta, N = 2, 3, 12
    phi = synth.smooth_orbital(g.n, g.h, (8.0, 8.0, 8.0))
    eta = (0.05 * (rng.normal(size=(n_s, n_eta) + g.shape()) + 1j * rng.normal(size=(n_s, n_eta) + g.shape()))
           ).astype(np.complex64)
    src = (np.sign(rng.normal(size=(n_s,) + g.shape())) * phi).astype(np.float32)
    c = _ctx(s, 2 * n_s * n_eta)
    uR = torch.empty(n_s, N + 1, g.ng, dtype=torch.float32, device='cuda')
    c.tdh_response(gc.to_dev(eta.reshape(n_s * n_eta, -1), torch, torch.complex64),
                   gc.to_dev(src.reshape(n_s, -1), torch, torch.float32), n_s, n_eta, N, 0.05, 0, uR)
    got = uR.cpu().numpy().reshape((n_s, N + 1) + g.shape())
    prob = osgw.Problem(g, s['vloc'], kb, -5.0, 70.0, 0, 0, phi)
    for si in range(n_s):
        ref = osgw.tdh_response_tangent(prob, eta[si].astype(np.complex128), src[si].astype(np.float64), N, 0.05,
                                        16, split=kbs)
        assert gc.rel_err(got[si], ref) < 2e-4
    zeta = (rng.normal(size=(n_s, 2) + g.shape()) + 1j * rng.normal(size=(n_s, 2) + g.shape())).astype(np.complex64)
    u = (0.3 * (rng.normal(size=(n_s, N + 1) + g.shape()) + 1j * rng.normal(size=(n_s, N + 1) + g.shape()))
         ).astype(np.complex64)
    sig = torch.empty(n_s, 2 * N + 1, dtype=torch.complex128, device='cuda')
    c.sigma_c(gc.to_dev(zeta.reshape(2 * n_s, -1), torch, torch.complex64),
              gc.to_dev(phi.ravel().astype(np.float32), torch, torch.float32),
              gc.to_dev(u.reshape(n_s, N + 1, -1), torch, torch.complex64), n_s, N, 0.05, 0, sig, 1)
    got = sig.cpu().numpy()
    for si in range(n_s):
        ref = osgw.sigma_t(prob, zeta[si, 0].astype(np.complex128), zeta[si, 1].astype(np.complex128),
                           u[si].astype(np.complex128), N, 0.05, 16, split=kbs)
        assert gc.rel_err(got[si], ref) < 2e-4


def test_split_pipeline_tracks_the_chebyshev_pipeline():
    """The whole 16^3 sample with split-operator TDH and zeta steps stays within the split scheme's
    O(dt^2) error of the Chebyshev pipeline on the same samples (200 steps of dt = 0.05)."""
    from paper_2601_21005_gb300.pipeline import Pipeline
    build.build()
    s = synth.wells()
    g, kb, w, phis = gc.oracle_eigs(s, 8)
    res = {}
    for prop in ('chebyshev', 'split'):
        pl = Pipeline(s['n'], s['h'], s['vloc'], [], phis[3], w[3], w[4], n_eta=8, n_steps=200, dt=0.05,
                      cheb_deg=16, n_cheb=128, samples_per_batch=2, seed=12, spectrum=(-4.0, 45.0), propagator=prop)
        sig, x = pl.run(4)
        res[prop] = (sig.cpu().numpy(), x.cpu().numpy(), pl.qp(sig, x, w[3])['eps_qp'])
    a, b = res['chebyshev'], res['split']
    assert np.array_equal(a[1], b[1])                       # the exchange does not propagate
    assert np.linalg.norm(a[0] - b[0]) < 2e-2 * np.linalg.norm(a[0])
    assert abs(a[2] - b[2]) * 27.2114 < 0.05
