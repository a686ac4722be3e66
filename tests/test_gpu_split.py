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
