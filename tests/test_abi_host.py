"""The C-ABI library loads, exports every entry point include/sgw.h declares, and its
host-side FP64 routines agree with the oracle (no GPU needed for any of this)."""
import os
import re
import ctypes

import numpy as np
import pytest

from oracle import chebyshev as cheb
from paper_2601_21005_gb300 import build, sgw

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope='module')
def lib():
    build.build()
    return sgw.lib()


def _declared():
    src = open(os.path.join(ROOT, 'include', 'sgw.h')).read()
    src = re.sub(r'/\*.*?\*/', '', src, flags=re.S)
    return sorted(set(re.findall(r'\b(sgw_[a-z0-9_]+)\s*\(', src)))


def test_header_declares_the_entry_points():
    names = _declared()
    for need in ('sgw_setup_grid', 'sgw_set_potential', 'sgw_filter_occupied', 'sgw_propagate',
                 'sgw_sigma_c', 'sgw_qp_energy', 'sgw_tdh_response', 'sgw_time_order'):
        assert need in names


def test_library_exports_every_declared_symbol(lib):
    for name in _declared():
        assert hasattr(lib, name), name
        assert isinstance(getattr(lib, name), ctypes._CFuncPtr)
    # the binding wraps every declared symbol
    assert sorted(sgw.exported_symbols()) == _declared()


def test_version_and_error_plumbing(lib):
    assert 'sm_103a' in sgw.sgw_version()
    with pytest.raises(sgw.SgwError):
        sgw.sgw_gapped_filter_coeffs(-0.1, -0.2, -1.0, 1.0, 10)   # e_lumo < e_homo


@pytest.mark.parametrize('K,a,dt', [(16, -3.0, 0.05), (16, 5.0, -0.05), (24, 10.0, 0.1), (3, 1.0, 0.2)])
def test_propagator_coeffs_match_oracle(lib, K, a, dt):
    emin, emax = a - 40.0, a + 20.0
    c, ph = sgw.sgw_propagator_coeffs(emin, emax, dt, K)
    co, pho = cheb.propagator_coeffs(emin, emax, dt, K)
    assert np.max(np.abs(c - co)) < 1e-14
    assert abs(ph - pho) < 1e-14


@pytest.mark.parametrize('N,eh,el', [(128, -1.09, -0.84), (300, -0.2, 0.1), (1500, -0.134, -0.007), (60, 2.0, 2.0)])
def test_gapped_coeffs_match_oracle(lib, N, eh, el):
    emin, emax = -2.5, 62.0
    a = sgw.sgw_gapped_filter_coeffs(eh, el, emin, emax, N)
    ao = cheb.gapped_filter_coeffs(eh, el, emin, emax, N)
    # both solve the same strictly convex ridge least-squares problem (different algorithms)
    assert np.max(np.abs(a - ao)) < 1e-7
    xs = np.linspace(-1, 1, 2001)
    assert np.max(np.abs(cheb.cheb_scalar(a, xs) - cheb.cheb_scalar(ao, xs))) < 1e-6


def test_control_variate_sizes_match_oracle(lib):
    from oracle import mlp as omlp
    for m2 in (1, 3, 10, 17):
        assert sgw.sgw_cv_feature_count(m2) == omlp.feature_count(m2)
        assert sgw.sgw_cv_shell_count(m2) == omlp.shell_count(m2)
    assert sgw.sgw_cv_linear_size(20, 1603) == 2 * 20 + 1603 + 20 * 1603
    assert sgw.sgw_cv_linear_size(0, 5) == 0


@pytest.mark.parametrize('n', [40, 100, 256, 12])
def test_setup_refuses_unsupported_grid_sides(lib, n):
    """Grid sides other than 16, 32, 64, 128 (plane path) and 48, 96, 288 (row path) are refused on
    the host, before any device call, with SGW_EINVAL and a message naming the supported sides."""
    p = ctypes.c_void_p()
    st = lib.sgw_setup_grid(ctypes.byref(p), n, n, n, 0.5, 0.0, 1, 0, None)
    assert st == 1 and not p.value
    assert b'48,96,288' in lib.sgw_last_error(None)


def test_setup_refuses_non_cubic_grids(lib):
    p = ctypes.c_void_p()
    assert lib.sgw_setup_grid(ctypes.byref(p), 48, 48, 96, 0.5, 0.0, 1, 0, None) == 1
