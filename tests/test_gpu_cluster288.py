"""The 288^3 grid's kernels (kernels_cluster.cu: z lines, the row form of the xy pass with 36-row
units, and the two-pass form with one thread-block cluster of 8 CTAs per xy plane) against the FP64 oracle on the large cluster itself (Si7055H1596: 7055 Si with
s/p KB projectors, 11 M support points, so every 36-row unit carries many slots and colours):
H psi element by element, one degree-16 Chebyshev propagation step, reversibility of a
forward-backward pair, and the results under every plane-pass and line form (bit-identical where
only the thread that computes a butterfly changes, within FP32 rounding where warp FFTs replace
radix stages) and any batch composition."""
import numpy as np
import pytest

from oracle import chebyshev as cheb
from oracle import hamiltonian as ham
from paper_2601_21005_gb300 import build, synth

import gpu_common as gc

torch = pytest.importorskip('torch')
pytestmark = pytest.mark.gpu


@pytest.fixture(scope='module')
def large288():
    assert torch.cuda.is_available()
    build.build()
    s = synth.si_cluster(n=288, h=0.5, radius=61.0)
    g = ham.Grid(s['n'], s['h'])
    kb = ham.KB(s['kb_atoms'])
    # an interval that encloses the spectrum: local well depths, the kinetic maximum 3 (pi/h)^2 / 2
    # and the KB energies (projectors normalised, |E| <= 1.2)
    lo = float(s['vloc'].min()) - 2.0
    hi = float(s['vloc'].max()) + 1.5 * (np.pi / s['h']) ** 2 + 8.0
    from paper_2601_21005_gb300 import sgw
    c = sgw.Context(s['n'], s['h'], max_batch=3)
    c.set_potential(gc.to_dev(s['vloc'].ravel(), torch, torch.float32), s['kb_atoms'])
    c.set_spectrum(lo, hi)
    return s, g, kb, (lo, hi), c


_ORACLE = {}          # oracle results shared by the parametrised cases


def _oracle(key, fn):
    if key not in _ORACLE:
        _ORACLE[key] = fn()
    return _ORACLE[key]


def _vec(g, seed):
    r = np.random.default_rng(seed)
    x = r.normal(size=g.shape()) + 1j * r.normal(size=g.shape())
    return (x / np.sqrt(np.sum(np.abs(x) ** 2))).astype(np.complex64)


@pytest.mark.parametrize('line_form', [0, 3, 4])
def test_cluster_apply_h_288_large_cluster(large288, line_form):
    s, g, kb, _, c = large288
    x = np.stack([_vec(g, 1), _vec(g, 2)])
    xd = gc.to_dev(x.reshape(2, -1), torch, torch.complex64)
    yd = torch.empty_like(xd)
    c.set_tuning(c.TUNE_LINE_FORM, line_form)
    c.apply_h(xd, yd)
    c.set_tuning(c.TUNE_LINE_FORM, 0)
    got = yd.cpu().numpy()
    ref = _oracle('apply_h', lambda: ham.apply_h(x[1].astype(np.complex128), g, s['vloc'], kb))
    assert gc.rel_err(got[1].reshape(g.shape()), ref) < 2e-5


@pytest.mark.parametrize('line_form', [0, 3, 4])
def test_cluster_propagate_288_large_cluster(large288, line_form):
    s, g, kb, (lo, hi), c = large288
    x0 = _vec(g, 3)
    x = np.stack([x0, x0])
    xd = gc.to_dev(x.reshape(2, -1), torch, torch.complex64)
    c.set_tuning(c.TUNE_LINE_FORM, line_form)
    c.propagate(xd, 1, 0.05, 16, np.array([1, -1], dtype=np.int8))
    got = xd.cpu().numpy()
    ref = _oracle('propagate', lambda: cheb.propagate_step(lambda v: ham.apply_h(v, g, s['vloc'], kb),
                                                           x0.astype(np.complex128), lo, hi, 0.05, 16))
    assert gc.rel_err(got[0].reshape(g.shape()), ref) < 1e-5
    for b in range(2):              # norms in FP64: a float32 sum of 24 M squares loses ~1e-4
        assert abs(np.linalg.norm(got[b].astype(np.complex128)) - 1.0) < 1e-5
    # back again: U(-dt) U(dt) = 1 (vector 0 forward then backward, vector 1 backward then forward)
    c.propagate(xd, 1, 0.05, 16, np.array([-1, 1], dtype=np.int8))
    back = xd.cpu().numpy()
    c.set_tuning(c.TUNE_LINE_FORM, 0)
    for b in range(2):
        assert gc.rel_err(back[b], x0.reshape(-1)) < 1e-5


def test_cluster_launch_choices_and_batches_are_bit_identical(large288):
    s, g, kb, _, c = large288
    x = np.stack([_vec(g, 4), _vec(g, 5), _vec(g, 6)])
    ref = None
    outs = {}
    for variant in (0, 1, 2):
        for form in (0, 1, 2, 3, 4):
            c.set_tuning(c.TUNE_PLANE_VARIANT, variant)
            c.set_tuning(c.TUNE_LINE_FORM, form)
            xd = gc.to_dev(x.reshape(3, -1), torch, torch.complex64)
            c.propagate(xd, 1, 0.05, 8)
            outs[(variant, form)] = xd
    ref = outs[(0, 0)]
    for (variant, form), xd in outs.items():
        # z-line forms 0 and 1 differ only in which thread computes a butterfly, and the two cluster
        # forms (1, 2) only in how many warps share the lines: the same bits
        if form == 1:
            assert torch.equal(xd, outs[(variant, 0)]), (variant, form)
        if variant == 2:
            assert torch.equal(xd, outs[(1, form)]), (variant, form)
        # warp FFTs (the cluster form's y lines, z-line form 2) and the two-stage 16 x 18
        # transform (form 3: z lines and the row form's y lines; form 4: its rows too) order the
        # sums differently from the radix stages: equal to FP32 rounding
        assert gc.rel_err(xd.cpu().numpy(), ref.cpu().numpy()) < 1e-5, (variant, form)
    c.set_tuning(c.TUNE_PLANE_VARIANT, 0)
    # the operand hints (L2 prefetch, streaming cache policy) change no arithmetic: the same bits
    for form in (0, 4):
        c.set_tuning(c.TUNE_LINE_FORM, form)
        for ops in (0, 2, 3):
            c.set_tuning(c.TUNE_PLANE_OPERANDS, ops)
            xd = gc.to_dev(x.reshape(3, -1), torch, torch.complex64)
            c.propagate(xd, 1, 0.05, 8)
            assert torch.equal(xd, outs[(0, form)]), (form, ops)
    c.set_tuning(c.TUNE_PLANE_OPERANDS, 1)
    c.set_tuning(c.TUNE_LINE_FORM, 0)
    one = gc.to_dev(x[1].reshape(1, -1), torch, torch.complex64)
    c.propagate(one, 1, 0.05, 8)
    assert torch.equal(one[0], ref[1])
