"""Thin Python binding of libsgw (include/sgw.h): argument marshalling only.

Every function keeps the C name and forwards plain pointers and sizes; device arrays are
passed as torch CUDA tensors (their data pointers), host arrays as numpy arrays.  All
computation happens in the CUDA library; if it is not built or cannot be loaded, every
call raises.
"""
import ctypes
import os

import numpy as np

from . import build as _build

_lib = None

PROF_KINDS = ['plane_step', 'pencil', 'kb_project', 'plane_fwd', 'tdh_density', 'sigma', 'time_order', 'other',
              'split_inv', 'lines']

SGW_STATUS = {0: 'SGW_OK', 1: 'SGW_EINVAL', 2: 'SGW_ENOMEM', 3: 'SGW_ECUDA', 4: 'SGW_ESTATE',
              5: 'SGW_ETIMEOUT', 6: 'SGW_ENOCONV'}


class SgwError(RuntimeError):
    def __init__(self, fn, status, msg):
        super().__init__('%s -> %s: %s' % (fn, SGW_STATUS.get(status, status), msg))
        self.status = status


_c = ctypes
_P = _c.c_void_p
_SIGS = {
    'sgw_version': ([], _c.c_char_p),
    'sgw_last_error': ([_P], _c.c_char_p),
    'sgw_setup_grid': ([_c.POINTER(_P), _c.c_int, _c.c_int, _c.c_int, _c.c_double, _c.c_double, _c.c_int, _c.c_int, _P], _c.c_int),
    'sgw_destroy': ([_P], None),
    'sgw_set_stream': ([_P, _P], _c.c_int),
    'sgw_set_graph_mode': ([_P, _c.c_int], _c.c_int),
    'sgw_set_tuning': ([_P, _c.c_int, _c.c_int], _c.c_int),
    'sgw_get_tuning': ([_P, _c.c_int, _P], _c.c_int),
    'sgw_autotune': ([_P, _c.c_int, _c.c_int, _P], _c.c_int),
    'sgw_set_potential': ([_P, _P, _c.c_int, _P, _P, _P, _P, _P], _c.c_int),
    'sgw_apply_h': ([_P, _P, _P, _c.c_int], _c.c_int),
    'sgw_spectral_bounds': ([_P, _c.c_int, _c.c_uint64, _c.c_double, _P, _P, _P], _c.c_int),
    'sgw_set_spectrum': ([_P, _c.c_double, _c.c_double], _c.c_int),
    'sgw_gapped_filter_coeffs': ([_c.c_double, _c.c_double, _c.c_double, _c.c_double, _c.c_int, _c.c_double, _P], _c.c_int),
    'sgw_propagator_coeffs': ([_c.c_double, _c.c_double, _c.c_double, _c.c_int, _P, _P], _c.c_int),
    'sgw_filter_occupied': ([_P, _P, _c.c_int, _P, _P, _c.c_int], _c.c_int),
    'sgw_white_noise': ([_P, _c.c_uint64, _c.c_uint32, _c.c_int, _c.c_int, _c.c_int, _P], _c.c_int),
    'sgw_prepare_sample': ([_P, _P, _P, _P, _c.c_int, _c.c_int, _P, _P, _P], _c.c_int),
    'sgw_propagate': ([_P, _P, _c.c_int, _c.c_int, _c.c_double, _c.c_int, _P], _c.c_int),
    'sgw_propagate_split': ([_P, _P, _c.c_int, _c.c_int, _c.c_double, _P], _c.c_int),
    'sgw_tdh_response': ([_P, _P, _P, _c.c_int, _c.c_int, _c.c_int, _c.c_double, _c.c_int, _c.c_double, _P], _c.c_int),
    'sgw_time_order': ([_P, _P, _P, _c.c_int, _c.c_int], _c.c_int),
    'sgw_time_order_points': ([_P, _P, _P, _c.c_int, _c.c_int, _c.c_int], _c.c_int),
    'sgw_tdh_response_xi': ([_P, _P, _P, _c.c_int, _c.c_int, _c.c_int, _c.c_double, _c.c_int, _c.c_double,
                             _c.c_uint64, _c.c_uint32, _c.c_int, _c.c_int, _c.c_double, _c.c_int, _P], _c.c_int),
    'sgw_sigma_c_xi': ([_P, _P, _P, _P, _c.c_int, _c.c_int, _c.c_double, _c.c_int, _c.c_int, _c.c_uint64,
                        _c.c_uint32, _c.c_int, _c.c_int, _c.c_double, _c.c_int, _P], _c.c_int),
    'sgw_sigma_c': ([_P, _P, _P, _P, _c.c_int, _c.c_int, _c.c_double, _c.c_int, _c.c_int, _P], _c.c_int),
    'sgw_exchange': ([_P, _P, _P, _c.c_int, _c.c_int, _P], _c.c_int),
    'sgw_sigma_omega': ([_P, _P, _c.c_int, _c.c_int, _c.c_double, _c.c_double, _P, _c.c_int, _c.c_int, _P], _c.c_int),
    'sgw_cv_feature_count': ([_c.c_int], _c.c_int),
    'sgw_cv_features': ([_P, _P, _c.c_int, _c.c_int, _P, _c.c_int, _P], _c.c_int),
    'sgw_cv_standardize': ([_P, _P, _c.c_int, _c.c_int, _c.c_int, _P, _P, _P], _c.c_int),
    'sgw_cv_standardize_f32': ([_P, _P, _c.c_int, _c.c_int, _c.c_int, _P, _P], _c.c_int),
    'sgw_cv_rows': ([_P, _P, _c.c_int, _P, _P, _c.c_int, _c.c_int, _P, _P, _P], _c.c_int),
    'sgw_cv_shell_count': ([_c.c_int], _c.c_int),
    'sgw_cv_shell_sums': ([_P, _P, _c.c_int, _c.c_int, _P], _c.c_int),
    'sgw_cv_linear_size': ([_c.c_int, _c.c_int], _c.c_int64),
    'sgw_cv_linear_fit': ([_P, _P, _P, _c.c_int, _c.c_int, _c.c_int, _c.c_double, _P], _c.c_int),
    'sgw_cv_linear_apply': ([_P, _P, _P, _c.c_int, _c.c_int, _c.c_int, _P, _P], _c.c_int),
    'sgw_cv_linear_rows': ([_P, _P, _P, _c.c_int, _P, _c.c_int, _c.c_int, _c.c_int, _P, _P], _c.c_int),
    'sgw_mlp_create': ([_c.POINTER(_P), _c.c_int, _c.c_int, _c.c_int, _c.c_int, _c.c_uint64, _c.c_int, _P], _c.c_int),
    'sgw_mlp_destroy': ([_P], None),
    'sgw_mlp_last_error': ([_P], _c.c_char_p),
    'sgw_mlp_param_count': ([_P], _c.c_int64),
    'sgw_mlp_set_params': ([_P, _P, _c.c_int64], _c.c_int),
    'sgw_mlp_get_params': ([_P, _P, _c.c_int64], _c.c_int),
    'sgw_mlp_forward': ([_P, _P, _c.c_int, _P], _c.c_int),
    'sgw_mlp_set_loss_weights': ([_P, _P, _c.c_int], _c.c_int),
    'sgw_mlp_gradients': ([_P, _P, _P, _c.c_int, _P, _P], _c.c_int),
    'sgw_mlp_adam_step': ([_P, _c.c_float], _c.c_int),
    'sgw_mlp_train_epoch': ([_P, _P, _P, _c.c_int, _c.c_int, _c.c_float, _P], _c.c_int),
    'sgw_qp_energy_noalloc': ([_P, _P, _c.c_int, _c.c_int, _c.c_double, _c.c_double, _c.c_double, _c.c_double,
                               _c.c_double, _c.c_double, _c.c_int, _P, _P], _c.c_int),
    'sgw_profile': ([_P, _c.c_int], _c.c_int),
    'sgw_profile_read': ([_P, _c.c_int, _P, _P, _P], _c.c_int),
    'sgw_launch_count': ([_P, _P], _c.c_int),
    'sgw_qp_energy': ([_P, _P, _P, _c.c_int, _c.c_int, _c.c_double, _c.c_double, _c.c_double, _c.c_double,
                       _c.c_double, _c.c_double, _c.c_int, _P], _c.c_int),
}


def lib():
    """Load libsgw.so (raises if it is missing or cannot be loaded)."""
    global _lib
    if _lib is None:
        if not os.path.exists(_build.LIB):
            raise RuntimeError('libsgw.so is not built (%s); run __graft_entry__.build() or '
                               'python -m paper_2601_21005_gb300.build' % _build.LIB)
        L = ctypes.CDLL(_build.LIB)
        for name, (args, res) in _SIGS.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib = L
    return _lib


def exported_symbols():
    return list(_SIGS)


def _dev(t, dtype=None):
    """Data pointer of a contiguous CUDA tensor (None -> NULL)."""
    if t is None:
        return None
    if not hasattr(t, 'data_ptr'):
        raise TypeError('expected a torch tensor')
    if not t.is_cuda:
        raise ValueError('expected a CUDA tensor')
    if not t.is_contiguous():
        raise ValueError('expected a contiguous tensor')
    if dtype is not None and t.dtype != dtype:
        raise ValueError('expected dtype %s, got %s' % (dtype, t.dtype))
    return t.data_ptr()


def _host(a, dtype):
    if a is None:
        return None, None
    a = np.ascontiguousarray(a, dtype=dtype)
    return a, a.ctypes.data_as(_P)


def _check(fn, st, ctx=None):
    if st != 0:
        msg = lib().sgw_last_error(ctx)
        raise SgwError(fn, st, msg.decode() if msg else '')


# ------------------------------------------------------------------ host-only routines
def sgw_version():
    return lib().sgw_version().decode()


def sgw_gapped_filter_coeffs(e_homo, e_lumo, emin, emax, n_cheb, ridge=1e-8):
    out = np.zeros(n_cheb + 1)
    _check('sgw_gapped_filter_coeffs',
           lib().sgw_gapped_filter_coeffs(e_homo, e_lumo, emin, emax, n_cheb, ridge, out.ctypes.data_as(_P)))
    return out


def sgw_propagator_coeffs(emin, emax, dt, cheb_deg):
    c = np.zeros(2 * (cheb_deg + 1))
    ph = np.zeros(2)
    _check('sgw_propagator_coeffs',
           lib().sgw_propagator_coeffs(emin, emax, dt, cheb_deg, c.ctypes.data_as(_P), ph.ctypes.data_as(_P)))
    return c[0::2] + 1j * c[1::2], ph[0] + 1j * ph[1]


def sgw_qp_energy_noalloc(sigma, x, n_samples, n_steps, dt, gamma, eps_ks, vxc=0.0, window=2.0, step=1e-3,
                          fp64=1, stream=None):
    """QP solve that allocates no device memory (for callers whose device memory is owned by
    another allocator); scratch is a fixed 1 MiB array inside the library.  Same result as
    Context.qp_energy."""
    import torch
    if stream is None:
        stream = torch.cuda.current_stream().cuda_stream
    r = np.zeros(4)
    _check('sgw_qp_energy_noalloc',
           lib().sgw_qp_energy_noalloc(_dev(sigma, torch.complex128), _dev(x, torch.float64), n_samples, n_steps, dt,
                                       gamma, eps_ks, vxc, window, step, fp64, r.ctypes.data_as(_P), _P(stream)))
    return dict(eps_qp=r[0], se=r[1], re_sigma=r[2], z=r[3])


def sgw_cv_feature_count(m2max):
    return lib().sgw_cv_feature_count(m2max)


def sgw_cv_shell_count(m2max):
    return lib().sgw_cv_shell_count(m2max)


def sgw_cv_linear_size(p, o):
    return lib().sgw_cv_linear_size(p, o)


class MLP:
    """Owns one sgw_mlp (the control-variate network).  Methods mirror sgw_mlp_*."""

    def __init__(self, n_in, width, n_out, max_batch, seed=0, device=0, stream=None):
        import torch
        if stream is None:
            stream = torch.cuda.current_stream(device).cuda_stream
        p = _P()
        _check('sgw_mlp_create', lib().sgw_mlp_create(ctypes.byref(p), n_in, width, n_out, max_batch, seed, device,
                                                      _P(stream)))
        self._p = p
        self.n_in, self.width, self.n_out, self.max_batch = n_in, width, n_out, max_batch

    def close(self):
        if getattr(self, '_p', None):
            lib().sgw_mlp_destroy(self._p)
            self._p = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _ck(self, fn, st):
        if st != 0:
            msg = lib().sgw_mlp_last_error(self._p)
            raise SgwError(fn, st, msg.decode() if msg else '')

    def param_count(self):
        return lib().sgw_mlp_param_count(self._p)

    def set_params(self, flat):
        a, pa = _host(flat, np.float32)
        self._ck('sgw_mlp_set_params', lib().sgw_mlp_set_params(self._p, pa, len(a)))

    def get_params(self):
        out = np.zeros(self.param_count(), dtype=np.float32)
        self._ck('sgw_mlp_get_params', lib().sgw_mlp_get_params(self._p, out.ctypes.data_as(_P), len(out)))
        return out

    def set_loss_weights(self, w):
        a, pa = _host(w, np.float32)
        self._ck('sgw_mlp_set_loss_weights', lib().sgw_mlp_set_loss_weights(self._p, pa, self.n_out))

    def forward(self, x, y):
        import torch
        self._ck('sgw_mlp_forward', lib().sgw_mlp_forward(self._p, _dev(x, torch.float32), x.shape[0],
                                                         _dev(y, torch.float32)))

    def gradients(self, x, t, want_grads=False):
        import torch
        loss = _c.c_double()
        g = np.zeros(self.param_count(), dtype=np.float32) if want_grads else None
        self._ck('sgw_mlp_gradients', lib().sgw_mlp_gradients(self._p, _dev(x, torch.float32), _dev(t, torch.float32),
                                                             x.shape[0], _c.byref(loss),
                                                             g.ctypes.data_as(_P) if want_grads else None))
        return loss.value, g

    def adam_step(self, lr):
        self._ck('sgw_mlp_adam_step', lib().sgw_mlp_adam_step(self._p, lr))

    def train_epoch(self, x, t, batch, lr):
        import torch
        loss = _c.c_double()
        self._ck('sgw_mlp_train_epoch', lib().sgw_mlp_train_epoch(self._p, _dev(x, torch.float32),
                                                                 _dev(t, torch.float32), x.shape[0], batch, lr,
                                                                 _c.byref(loss)))
        return loss.value


# ------------------------------------------------------------------ context
class Context:
    """Owns one sgw_ctx for an n^3 grid (n in 16, 32, 64, 128, or 48, 96, 288 on the row path).
    Methods mirror the C entry points (sgw_<name> -> <name>)."""

    def __init__(self, n, h, ecut=0.0, max_batch=1, device=0, stream=None):
        import torch
        L = lib()
        self.n, self.h, self.ng, self.dV = n, h, n ** 3, h ** 3
        self.device = device
        if stream is None:
            stream = torch.cuda.current_stream(device).cuda_stream
        p = _P()
        st = L.sgw_setup_grid(ctypes.byref(p), n, n, n, h, ecut, max_batch, device, _P(stream))
        _check('sgw_setup_grid', st, None)
        self._p = p
        self.max_batch = max_batch

    def close(self):
        if getattr(self, '_p', None):
            lib().sgw_destroy(self._p)
            self._p = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _ck(self, fn, st):
        _check(fn, st, self._p)

    def set_stream(self, stream):
        self._ck('sgw_set_stream', lib().sgw_set_stream(self._p, _P(stream)))

    def set_graph_mode(self, enable):
        self._ck('sgw_set_graph_mode', lib().sgw_set_graph_mode(self._p, 1 if enable else 0))

    (TUNE_PLANE_OPERANDS, TUNE_PLANE_LOOKAHEAD, TUNE_PENCIL_LOOKAHEAD, TUNE_PLANE_VARIANT, TUNE_LINE_FORM,
     TUNE_KEYS) = 0, 1, 2, 3, 4, 5

    def set_tuning(self, key, value):
        self._ck('sgw_set_tuning', lib().sgw_set_tuning(self._p, int(key), int(value)))

    def get_tuning(self, key):
        v = _c.c_int(0)
        self._ck('sgw_get_tuning', lib().sgw_get_tuning(self._p, int(key), _c.byref(v)))
        return v.value

    def autotune(self, batch, reps=3):
        """Time the candidate lookaheads on a scratch batch; returns the chosen value per key."""
        out = (_c.c_int * self.TUNE_KEYS)()
        self._ck('sgw_autotune', lib().sgw_autotune(self._p, int(batch), int(reps), out))
        return list(out)

    def set_potential(self, vloc_dev, kb_atoms=()):
        """kb_atoms: list of (support flat indices, beta [n_proj, n_sup], e [n_proj])."""
        import torch
        n_atoms = len(kb_atoms)
        if n_atoms:
            nproj = np.array([b.shape[0] for (_, b, _) in kb_atoms], dtype=np.int32)
            off = np.zeros(n_atoms + 1, dtype=np.int64)
            off[1:] = np.cumsum([len(s) for (s, _, _) in kb_atoms])
            idx = np.concatenate([np.asarray(s, dtype=np.int32) for (s, _, _) in kb_atoms])
            beta = np.zeros((off[-1], 4), dtype=np.float32)
            e = np.zeros((n_atoms, 4), dtype=np.float32)
            for a, (s, b, ee) in enumerate(kb_atoms):
                beta[off[a]:off[a + 1], :b.shape[0]] = np.asarray(b).T
                e[a, :len(ee)] = ee
        else:
            nproj = off = idx = beta = e = None
        a1, p1 = _host(nproj, np.int32)
        a2, p2 = _host(off, np.int64)
        a3, p3 = _host(idx, np.int32)
        a4, p4 = _host(beta, np.float32)
        a5, p5 = _host(e, np.float32)
        self._ck('sgw_set_potential', lib().sgw_set_potential(self._p, _dev(vloc_dev, torch.float32), n_atoms,
                                                               p1, p2, p3, p4, p5))

    def apply_h(self, x, out):
        import torch
        self._ck('sgw_apply_h', lib().sgw_apply_h(self._p, _dev(x, torch.complex64), _dev(out, torch.complex64),
                                                 x.numel() // self.ng))

    def spectral_bounds(self, n_iter, seed, margin=0.05):
        lo, hi, raw = _c.c_double(), _c.c_double(), np.zeros(2)
        self._ck('sgw_spectral_bounds', lib().sgw_spectral_bounds(self._p, n_iter, seed, margin, _c.byref(lo),
                                                                 _c.byref(hi), raw.ctypes.data_as(_P)))
        return (lo.value, hi.value), (raw[0], raw[1])

    def set_spectrum(self, emin, emax):
        self._ck('sgw_set_spectrum', lib().sgw_set_spectrum(self._p, emin, emax))

    def filter_occupied(self, coeffs, x, out):
        import torch
        c, pc = _host(coeffs, np.float64)
        self._ck('sgw_filter_occupied', lib().sgw_filter_occupied(self._p, pc, len(c) - 1, _dev(x, torch.complex64),
                                                                 _dev(out, torch.complex64), x.numel() // self.ng))

    def white_noise(self, seed, stream_id, sample0, n_samples, n_vec, out):
        import torch
        self._ck('sgw_white_noise', lib().sgw_white_noise(self._p, seed, stream_id, sample0, n_samples, n_vec,
                                                         _dev(out, torch.complex64)))

    def prepare_sample(self, noise, filt, phi, n_samples, n_eta, eta, zeta, source):
        import torch
        self._ck('sgw_prepare_sample', lib().sgw_prepare_sample(self._p, _dev(noise, torch.complex64),
                                                               _dev(filt, torch.complex64), _dev(phi, torch.float32),
                                                               n_samples, n_eta, _dev(eta, torch.complex64),
                                                               _dev(zeta, torch.complex64),
                                                               _dev(source, torch.float32)))

    def propagate(self, psi, n_steps, dt, cheb_deg, dirs=None):
        import torch
        d, pd = _host(dirs, np.int8)
        self._ck('sgw_propagate', lib().sgw_propagate(self._p, _dev(psi, torch.complex64), psi.numel() // self.ng,
                                                     n_steps, dt, cheb_deg, pd))

    def propagate_split(self, psi, n_steps, dt, dirs=None):
        import torch
        d, pd = _host(dirs, np.int8)
        self._ck('sgw_propagate_split', lib().sgw_propagate_split(self._p, _dev(psi, torch.complex64),
                                                                 psi.numel() // self.ng, n_steps, dt, pd))

    def tdh_response(self, eta, source, n_samples, n_eta, n_steps, dt, cheb_deg, uR, weight=0.0):
        import torch
        self._ck('sgw_tdh_response', lib().sgw_tdh_response(self._p, _dev(eta, torch.complex64),
                                                           _dev(source, torch.float32), n_samples, n_eta, n_steps, dt,
                                                           cheb_deg, weight, _dev(uR, torch.float32)))

    def time_order_points(self, uR, u, n_samples, n_steps, n_points):
        import torch
        self._ck('sgw_time_order_points', lib().sgw_time_order_points(self._p, _dev(uR, torch.float32),
                                                                     _dev(u, torch.complex64), n_samples, n_steps,
                                                                     n_points))

    def tdh_response_xi(self, eta, source, n_samples, n_eta, n_steps, dt, cheb_deg, xi, U, weight=0.0):
        """xi = (seed, stream, sample0, n_xi, f_g, L); U [n_samples][n_steps + 1][n_xi] float."""
        import torch
        seed, stream, sample0, n_xi, f_g, L = xi
        self._ck('sgw_tdh_response_xi', lib().sgw_tdh_response_xi(
            self._p, _dev(eta, torch.complex64), _dev(source, torch.float32), n_samples, n_eta, n_steps, dt,
            cheb_deg, weight, seed, stream, sample0, n_xi, f_g, L, _dev(U, torch.float32)))

    def sigma_c_xi(self, zeta, phi, u, n_samples, n_steps, dt, cheb_deg, xi, sigma, fp64_accum=1):
        import torch
        seed, stream, sample0, n_xi, f_g, L = xi
        self._ck('sgw_sigma_c_xi', lib().sgw_sigma_c_xi(
            self._p, _dev(zeta, torch.complex64), _dev(phi, torch.float32), _dev(u, torch.complex64), n_samples,
            n_steps, dt, cheb_deg, fp64_accum, seed, stream, sample0, n_xi, f_g, L, _dev(sigma, torch.complex128)))

    def time_order(self, uR, u, n_samples, n_steps):
        import torch
        self._ck('sgw_time_order', lib().sgw_time_order(self._p, _dev(uR, torch.float32), _dev(u, torch.complex64),
                                                       n_samples, n_steps))

    def sigma_c(self, zeta, phi, u, n_samples, n_steps, dt, cheb_deg, sigma, fp64_accum=1):
        import torch
        self._ck('sgw_sigma_c', lib().sgw_sigma_c(self._p, _dev(zeta, torch.complex64), _dev(phi, torch.float32),
                                                 _dev(u, torch.complex64), n_samples, n_steps, dt, cheb_deg,
                                                 fp64_accum, _dev(sigma, torch.complex128)))

    def exchange(self, eta, phi, n_samples, n_eta, x):
        import torch
        self._ck('sgw_exchange', lib().sgw_exchange(self._p, _dev(eta, torch.complex64), _dev(phi, torch.float32),
                                                   n_samples, n_eta, _dev(x, torch.float64)))

    def sigma_omega(self, sigma, n_samples, n_steps, dt, gamma, omega, out, fp64=1):
        import torch
        self._ck('sgw_sigma_omega', lib().sgw_sigma_omega(self._p, _dev(sigma, torch.complex128), n_samples, n_steps,
                                                         dt, gamma, _dev(omega, torch.float64), omega.numel(), fp64,
                                                         _dev(out, torch.complex128)))

    def qp_energy(self, sigma, x, n_samples, n_steps, dt, gamma, eps_ks, vxc=0.0, window=2.0, step=1e-3, fp64=1):
        import torch
        r = np.zeros(4)
        self._ck('sgw_qp_energy', lib().sgw_qp_energy(self._p, _dev(sigma, torch.complex128), _dev(x, torch.float64),
                                                     n_samples, n_steps, dt, gamma, eps_ks, vxc, window, step, fp64,
                                                     r.ctypes.data_as(_P)))
        return dict(eps_qp=r[0], se=r[1], re_sigma=r[2], z=r[3])

    def profile(self, enable):
        self._ck('sgw_profile', lib().sgw_profile(self._p, 1 if enable else 0))

    def profile_read(self):
        out = {}
        for k, name in enumerate(PROF_KINDS):
            ms, n, by = _c.c_double(), _c.c_int64(), _c.c_double()
            self._ck('sgw_profile_read', lib().sgw_profile_read(self._p, k, _c.byref(ms), _c.byref(n), _c.byref(by)))
            out[name] = dict(ms=ms.value, launches=n.value, alg_bytes=by.value)
        return out

    def launch_count(self):
        n = _c.c_int64()
        self._ck('sgw_launch_count', lib().sgw_launch_count(self._p, _c.byref(n)))
        return n.value

    def cv_features(self, noise, n_samples, n_vec, phi, m2max, feat):
        import torch
        self._ck('sgw_cv_features', lib().sgw_cv_features(self._p, _dev(noise, torch.complex64), n_samples, n_vec,
                                                         _dev(phi, torch.float32), m2max, _dev(feat, torch.float32)))

    def cv_standardize(self, y, mu, sd, t, compute_stats=True):
        import torch
        self._ck('sgw_cv_standardize', lib().sgw_cv_standardize(self._p, _dev(y, torch.float64), y.shape[0],
                                                               y.shape[1], 1 if compute_stats else 0,
                                                               _dev(mu, torch.float64), _dev(sd, torch.float64),
                                                               _dev(t, torch.float32)))

    def cv_standardize_f32(self, x, mu, sd, compute_stats=True):
        import torch
        self._ck('sgw_cv_standardize_f32', lib().sgw_cv_standardize_f32(self._p, _dev(x, torch.float32), x.shape[0],
                                                                       x.shape[1], 1 if compute_stats else 0,
                                                                       _dev(mu, torch.float64),
                                                                       _dev(sd, torch.float64)))

    def cv_shell_sums(self, feat, m2max, out):
        import torch
        self._ck('sgw_cv_shell_sums', lib().sgw_cv_shell_sums(self._p, _dev(feat, torch.float32), feat.shape[0], m2max,
                                                             _dev(out, torch.float32)))

    def cv_linear_fit(self, x, y, ridge, model):
        import torch
        self._ck('sgw_cv_linear_fit', lib().sgw_cv_linear_fit(self._p, _dev(x, torch.float32), _dev(y, torch.float64),
                                                             x.shape[0], x.shape[1], y.shape[1], float(ridge),
                                                             _dev(model, torch.float64)))

    def cv_linear_apply(self, model, x, o, out, y=None):
        """out = f(x), or y - f(x) when y is given."""
        import torch
        self._ck('sgw_cv_linear_apply', lib().sgw_cv_linear_apply(self._p, _dev(model, torch.float64),
                                                                 _dev(x, torch.float32), x.shape[0], x.shape[1], o,
                                                                 _dev(y, torch.float64), _dev(out, torch.float64)))

    def cv_linear_rows(self, model, x_cheap, x_paired, y, y_out):
        import torch
        self._ck('sgw_cv_linear_rows', lib().sgw_cv_linear_rows(self._p, _dev(model, torch.float64),
                                                               _dev(x_cheap, torch.float32), x_cheap.shape[0],
                                                               _dev(x_paired, torch.float32), x_paired.shape[0],
                                                               x_paired.shape[1], y.shape[1], _dev(y, torch.float64),
                                                               _dev(y_out, torch.float64)))

    def cv_rows(self, f_cheap, f_paired, y_paired, mu, sd, rows):
        import torch
        nc = 0 if f_cheap is None else f_cheap.shape[0]
        self._ck('sgw_cv_rows', lib().sgw_cv_rows(self._p, _dev(f_cheap, torch.float32), nc,
                                                 _dev(f_paired, torch.float32), _dev(y_paired, torch.float64),
                                                 y_paired.shape[0], y_paired.shape[1], _dev(mu, torch.float64),
                                                 _dev(sd, torch.float64), _dev(rows, torch.float64)))
