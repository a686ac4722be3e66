"""CUDA-graph mode of the propagation loops: replayed graphs give the same bits as direct launches,
and on the launch-bound 16^3 case they are faster."""
import time

import numpy as np
import pytest

from paper_2601_21005_gb300 import build, synth

import gpu_common as gc

torch = pytest.importorskip('torch')
pytestmark = pytest.mark.gpu


def _ctx(s, mb, stream):
    from paper_2601_21005_gb300 import sgw
    c = sgw.Context(s['n'], s['h'], max_batch=mb, stream=stream.cuda_stream)
    c.set_potential(gc.to_dev(s['vloc'].ravel(), torch, torch.float32), s['kb_atoms'])
    c.set_spectrum(float(s['vloc'].min()) - 2.0, 0.5 * 3 * (np.pi / s['h']) ** 2 + 2.0)
    return c


def test_graph_replay_is_bit_identical():
    assert torch.cuda.is_available()
    build.build()
    s = gc.small_cluster()
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        a, b = _ctx(s, 16, st), _ctx(s, 16, st)
        b.set_graph_mode(True)
        ng = s['n'] ** 3
        for c in (a, b):
            c.x = torch.empty(8, ng, dtype=torch.complex64, device='cuda')
            c.white_noise(3, 1, 0, 1, 8, c.x)
            c.y = torch.empty_like(c.x)
        coeff = np.linspace(1.0, 0.1, 41)
        for rep in range(3):                              # capture once, replay twice
            for c in (a, b):
                c.filter_occupied(coeff, c.x, c.y)
                c.propagate(c.y, 3, 0.05, 16, np.array([1, -1] * 4, dtype=np.int8))
            st.synchronize()
            assert torch.equal(a.y, b.y), rep
        # TDH and Sigma(t)
        n_s, n_eta, N = 2, 2, 4
        phi = gc.to_dev(synth.smooth_orbital(s['n'], s['h'], (8.0, 8.0, 8.0)).ravel(), torch, torch.float32)
        outs = []
        for c in (a, b):
            src = (c.x[:n_s].real.contiguous() * phi).contiguous()
            uR = torch.empty(n_s, N + 1, ng, dtype=torch.float32, device='cuda')
            u = torch.empty(n_s, N + 1, ng, dtype=torch.complex64, device='cuda')
            sig = torch.empty(n_s, 2 * N + 1, dtype=torch.complex128, device='cuda')
            for rep in range(2):
                z = c.y[:2 * n_s].clone()
                c.tdh_response(c.y[:n_s * n_eta].contiguous(), src, n_s, n_eta, N, 0.05, 16, uR)
                c.time_order(uR, u, n_s, N)
                c.sigma_c(z, phi, u, n_s, N, 0.05, 16, sig)
            st.synchronize()
            outs.append((uR.clone(), sig.clone()))
        assert torch.equal(outs[0][0], outs[1][0])
        assert torch.equal(outs[0][1], outs[1][1])


def test_graph_replay_of_the_tiny_pipeline_is_bit_identical():
    """Graph replay and direct launches give the same bits; the two timings are printed (not
    asserted: the GPUs are shared, so a timing comparison is no correctness check)."""
    from paper_2601_21005_gb300.pipeline import Pipeline
    s = synth.wells()
    g, kb, w, phis = gc.oracle_eigs(s, 8)
    times = {}
    res = {}
    for graphs in (False, True):
        pl = Pipeline(s['n'], s['h'], s['vloc'], [], phis[3], w[3], w[4], n_eta=8, n_steps=200, dt=0.05,
                      cheb_deg=16, n_cheb=128, samples_per_batch=1, seed=9, graphs=graphs,
                      spectrum=(-4.0, 45.0))
        sig = torch.empty(1, 401, dtype=torch.complex128, device='cuda')
        x = torch.empty(1, dtype=torch.float64, device='cuda')
        pl.run_batch(0, sig, x)                           # warm-up (and capture)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for b in range(5):
            pl.run_batch(0, sig, x)
        torch.cuda.synchronize()
        times[graphs] = (time.perf_counter() - t0) / 5
        res[graphs] = sig.clone()
    print('tiny pipeline per sample: direct %.1f ms, graphs %.1f ms' % (1e3 * times[False], 1e3 * times[True]))
    assert torch.equal(res[False], res[True])


def test_grouped_zeta_runs_match_single_chunks():
    """A run of 3 chunks whose zeta pairs propagate together gives, sample by sample, the same bits
    as three separate one-chunk runs (per-vector arithmetic does not depend on the batch)."""
    from paper_2601_21005_gb300.pipeline import Pipeline
    s = synth.wells()
    g, kb, w, phis = gc.oracle_eigs(s, 8)
    kw = dict(n_eta=4, n_steps=20, dt=0.05, cheb_deg=16, n_cheb=64, samples_per_batch=2, seed=21,
              spectrum=(-4.0, 45.0))
    one = Pipeline(s['n'], s['h'], s['vloc'], [], phis[3], w[3], w[4], zeta_group=1, **kw)
    grp = Pipeline(s['n'], s['h'], s['vloc'], [], phis[3], w[3], w[4], zeta_group=3, **kw)
    assert grp.run_samples == 6 and one.run_samples == 2
    s1, x1 = one.run(6, sample0=40)
    s3, x3 = grp.run(6, sample0=40)
    torch.cuda.synchronize()
    assert torch.equal(s1, s3) and torch.equal(x1, x3)
