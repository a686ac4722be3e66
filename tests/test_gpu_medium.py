"""The 128^3 medium cluster: Si657H300 (2928 electrons; 957 local wells, 657 atoms with s/p KB
projectors) built by the same rule as the 64^3 one, with 256 stochastic orbitals propagated in one
batch (every launch covers all 256) and the time loop replayed as a CUDA graph.  Checked: graph
replay gives the same bits as direct launches, every one of the 256 vectors keeps its norm, and
sampled vectors match the FP64 oracle step by step; H.psi on sampled vectors.

The spectral interval is a closed-form bound from the inputs (no estimate from the GPU path):
lambda in [min V_loc + E_p M, (1/2) 3 (pi/h)^2 + E_s M], M = the largest number of projector
supports that meet at one grid point (2 here), with 0.1 Ha of margin on each side for the small
non-orthogonality of one atom's s and p projectors on the grid (each is normalised on the grid)."""
import numpy as np
import pytest

from oracle import chebyshev as cheb
from oracle import hamiltonian as ham
from paper_2601_21005_gb300 import build, synth

import gpu_common as gc

torch = pytest.importorskip('torch')
pytestmark = pytest.mark.gpu

N, H, RADIUS, B = 128, 0.5, 28.0, 256


@pytest.fixture(scope='module')
def medium():
    assert torch.cuda.is_available()
    build.build()
    from paper_2601_21005_gb300 import sgw
    s = synth.si_cluster(n=N, h=H, radius=RADIUS)
    assert s['name'] == 'Si657H300' and 2 * s['n_occ'] == 2928
    g = ham.Grid(N, H)
    kb = ham.KB(s['kb_atoms'])
    mult = np.zeros(N ** 3, dtype=np.int32)
    for idx, _, _ in s['kb_atoms']:
        mult[idx] += 1
    M = int(mult.max())
    e_s, e_p = synth.SI_PARAMS['Es'], synth.SI_PARAMS['Ep']
    lo = float(s['vloc'].min()) + min(e_p, 0.0) * M - 0.1
    hi = 0.5 * 3 * (np.pi / H) ** 2 + max(e_s, 0.0) * M + 0.1
    st = torch.cuda.Stream()
    ctx = sgw.Context(N, H, max_batch=B, stream=st.cuda_stream)
    with torch.cuda.stream(st):
        ctx.set_potential(gc.to_dev(s['vloc'].ravel(), torch, torch.float32), s['kb_atoms'])
    ctx.set_spectrum(lo, hi)
    return s, g, kb, ctx, st, (lo, hi)


def test_medium_cluster_256_orbitals_graph_loop(medium):
    s, g, kb, ctx, st, (lo, hi) = medium
    dirs = np.array([1, -1] * (B // 2), dtype=np.int8)
    with torch.cuda.stream(st):
        x = torch.empty(B, N ** 3, dtype=torch.complex64, device='cuda')
        ctx.white_noise(31, 4, 0, 1, B, x)
        x0 = x.clone()
        y = x.clone()
        ctx.set_graph_mode(True)
        ctx.propagate(x, 2, 0.05, 16, dirs)           # captured as one graph, replayed
        ctx.set_graph_mode(False)
        ctx.propagate(y, 2, 0.05, 16, dirs)           # direct launches
        n0 = torch.linalg.vector_norm(x0, dim=1)
        n1 = torch.linalg.vector_norm(x, dim=1)
    st.synchronize()
    assert torch.equal(x, y)
    assert float(torch.max(torch.abs(n1 / n0 - 1))) < 1e-5
    h = lambda v: ham.apply_h(v, g, s['vloc'], kb)
    for b in (0, 255):
        ref = x0[b].cpu().numpy().reshape(g.shape()).astype(np.complex128)
        for _ in range(2):
            ref = cheb.propagate_step(h, ref, lo, hi, 0.05 * dirs[b], 16)
        assert gc.rel_err(x[b].cpu().numpy().reshape(g.shape()), ref) < 2e-5


def test_medium_cluster_apply_h(medium):
    s, g, kb, ctx, st, _ = medium
    with torch.cuda.stream(st):
        x = torch.empty(8, N ** 3, dtype=torch.complex64, device='cuda')
        ctx.white_noise(32, 4, 0, 1, 8, x)
        y = torch.empty_like(x)
        ctx.apply_h(x, y)
    st.synchronize()
    for b in (0, 7):
        ref = ham.apply_h(x[b].cpu().numpy().reshape(g.shape()).astype(np.complex128), g, s['vloc'], kb)
        assert gc.rel_err(y[b].cpu().numpy().reshape(g.shape()), ref) < 1e-5
