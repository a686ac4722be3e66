"""Edge and degenerate cases of the entry points on the GPU: empty batches and sample counts,
zero time steps, the largest batch a context takes (and one more, refused), a degree-0 filter,
dt = 0 propagation (identity for both steppers), zero vectors, and a QP window without a root."""
import numpy as np
import pytest

from oracle import chebyshev as cheb
from oracle import hamiltonian as ham
from paper_2601_21005_gb300 import build, synth

import gpu_common as gc

torch = pytest.importorskip('torch')
pytestmark = pytest.mark.gpu


@pytest.fixture(scope='module')
def ctx():
    assert torch.cuda.is_available()
    build.build()
    from paper_2601_21005_gb300 import sgw
    s = gc.small_cluster()
    c = sgw.Context(s['n'], s['h'], max_batch=6)
    c.set_potential(gc.to_dev(s['vloc'].ravel(), torch, torch.float32), s['kb_atoms'])
    c.set_spectrum(float(s['vloc'].min()) - 2.0, 0.5 * 3 * (np.pi / s['h']) ** 2 + 2.0)
    return s, c


def _noise(c, B, seed=1):
    x = torch.empty(B, c.ng, dtype=torch.complex64, device='cuda')
    c.white_noise(seed, 3, 0, 1, B, x)
    return x


def test_empty_inputs_are_no_ops(ctx):
    s, c = ctx
    e = torch.empty(0, c.ng, dtype=torch.complex64, device='cuda')
    c.apply_h(e, torch.empty_like(e))
    c.filter_occupied(np.ones(5), e, torch.empty_like(e))
    c.propagate(e, 3, 0.05, 16)
    c.propagate_split(e, 3, 0.05)
    c.white_noise(1, 1, 0, 0, 4, e)
    phi = torch.zeros(c.ng, dtype=torch.float32, device='cuda')
    c.exchange(e, phi, 0, 4, torch.empty(0, dtype=torch.float64, device='cuda'))
    c.time_order(torch.empty(0, 3, c.ng, dtype=torch.float32, device='cuda'),
                 torch.empty(0, 3, c.ng, dtype=torch.complex64, device='cuda'), 0, 2)
    torch.cuda.synchronize()


def test_zero_steps_leave_vectors_unchanged(ctx):
    s, c = ctx
    x = _noise(c, 4)
    x0 = x.clone()
    c.propagate(x, 0, 0.05, 16)
    c.propagate_split(x, 0, 0.05)
    torch.cuda.synchronize()
    assert torch.equal(x, x0)


def test_dt_zero_is_the_identity(ctx):
    s, c = ctx
    x = _noise(c, 4)
    x0 = x.clone()
    c.propagate_split(x, 2, 0.0)                      # every factor is 1: only the FFT round trips remain
    assert gc.rel_err(x.cpu().numpy(), x0.cpu().numpy()) < 5e-6
    c.propagate(x, 2, 0.0, 16)                        # J_0(0) = 1, J_k(0) = 0
    assert gc.rel_err(x.cpu().numpy(), x0.cpu().numpy()) < 1e-5


def test_zero_vectors_stay_zero(ctx):
    s, c = ctx
    z = torch.zeros(3, c.ng, dtype=torch.complex64, device='cuda')
    y = torch.empty_like(z)
    c.apply_h(z, y)
    c.propagate(z, 1, 0.05, 16)
    c.propagate_split(z, 1, 0.05)
    torch.cuda.synchronize()
    assert float(torch.max(torch.abs(y))) == 0.0 and float(torch.max(torch.abs(z))) == 0.0


def test_degree_zero_filter_scales(ctx):
    s, c = ctx
    x = _noise(c, 2)
    y = torch.empty_like(x)
    c.filter_occupied(np.array([0.25]), x, y)
    assert np.allclose(y.cpu().numpy(), 0.25 * x.cpu().numpy(), rtol=0, atol=1e-7)


def test_largest_batch_and_one_more(ctx):
    s, c = ctx
    x = _noise(c, 6)
    y = torch.empty_like(x)
    c.apply_h(x, y)                                    # max_batch = 6 is accepted
    g = ham.Grid(s['n'], s['h'])
    ref = ham.apply_h(x[5].cpu().numpy().reshape(g.shape()).astype(np.complex128), g, s['vloc'], ham.KB(s['kb_atoms']))
    assert gc.rel_err(y[5].cpu().numpy().reshape(g.shape()), ref) < 1e-5
    big = torch.empty(7, c.ng, dtype=torch.complex64, device='cuda')
    for call in (lambda: c.apply_h(big, torch.empty_like(big)), lambda: c.propagate(big, 1, 0.05, 16),
                 lambda: c.propagate_split(big, 1, 0.05), lambda: c.filter_occupied(np.ones(3), big, big.clone())):
        with pytest.raises(RuntimeError):
            call()


def test_bad_directions_and_degrees_are_refused(ctx):
    s, c = ctx
    x = _noise(c, 2)
    with pytest.raises(RuntimeError):
        c.propagate(x, 1, 0.05, 16, np.array([1, 0], dtype=np.int8))
    with pytest.raises(RuntimeError):
        c.propagate_split(x, 1, 0.05, np.array([2, 1], dtype=np.int8))
    with pytest.raises(RuntimeError):
        c.propagate(x, 1, 0.05, 0)                     # the plain Chebyshev call needs degree >= 1


def test_qp_window_without_a_root_reports_no_convergence(ctx):
    s, c = ctx
    # Sigma = 0 and X = 5 Ha: the root of w - eps - X = 0 lies 5 Ha away, outside a 1 Ha window
    sig = torch.zeros(3, 21, dtype=torch.complex128, device='cuda')
    x = torch.full((3,), 5.0, dtype=torch.float64, device='cuda')
    with pytest.raises(RuntimeError):
        c.qp_energy(sig, x, 3, 10, 0.05, 1.0, -0.2, 0.0, 1.0, 1e-3, 1)
