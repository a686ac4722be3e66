"""Runs the FP64 oracle's independent pieces of a batch on several host cores.

TEST INFRASTRUCTURE: part of the CPU oracle; only tests, the smoke check and the
CPU-baseline leg of the benchmark may use it.  It holds no arithmetic of its own: every
number comes from the functions of `sgw` and `chebyshev`, called exactly as
`sgw.run_sample` calls them, on pieces that the method computes independently:

* the gapped filter (Eq. 3) acts on each white-noise vector separately, so the N_eta + 1
  vectors of every sample are filtered in separate processes;
* the TDH response, time ordering, zeta propagation, Sigma(t) (Eq. 4-5) and exchange of a
  sample need only that sample's filtered vectors and the target orbital phi, so each
  (sample, phi) pair runs in its own process -- the HOMO and the LUMO of a sample share
  its noise and its filter.

Processes are started with the 'spawn' method (never forked), so a caller that has already
initialised a GPU context can use the pool safely.
"""
import multiprocessing as mp
import os

import numpy as np

from . import hamiltonian as ham
from . import sgw as osgw

_STATE = {}


def _init(n, h, vloc, kb_atoms, emin, emax, e_homo, e_lumo, threads):
    # each worker runs single-threaded BLAS/FFT work; the pool supplies the parallelism
    for k in ('OMP_NUM_THREADS', 'OPENBLAS_NUM_THREADS', 'MKL_NUM_THREADS'):
        os.environ[k] = str(threads)
    g = ham.Grid(n, h)
    kb = ham.KB(kb_atoms) if kb_atoms else None
    _STATE['prob'] = osgw.Problem(g, vloc, kb, emin, emax, e_homo, e_lumo, np.zeros(g.shape()))


def _filter_vector(args):
    vec, coeffs = args
    return osgw.filter_batch(_STATE['prob'], vec[None], coeffs)[0]


def _sample_response(args):
    """Steps 3-8 of `sgw.run_sample` for one sample and one target orbital."""
    zbar, filt, phi, n_steps, dt, K = args
    p0 = _STATE['prob']
    prob = osgw.Problem(p0.grid, p0.vloc, p0.kb, p0.emin, p0.emax, p0.e_homo, p0.e_lumo, phi)
    zocc = filt[0]
    zunocc = zbar - zocc
    eta = filt[1:]
    uR = osgw.tdh_response_tangent(prob, eta, zbar * prob.phi, n_steps, dt, K)
    u = osgw.time_order(uR)
    sig = osgw.sigma_t(prob, zocc, zunocc, u, n_steps, dt, K)
    x = osgw.exchange(prob, eta)
    return sig, x


def run_samples(system, spectrum, e_homo, e_lumo, coeffs, seed, stream, samples, n_eta, phis, n_steps, dt, K,
                processes=None):
    """Sigma_i(t) and X_i of every (orbital, sample): the oracle's `run_sample` for each phi in
    `phis` and each sample index in `samples`, with the noise and filter of a sample shared by
    its orbitals.

    system: dict with n, h, vloc, kb_atoms (the synthetic input); spectrum: (emin, emax).
    Returns (sigma [len(phis)][len(samples)][2 n_steps + 1] complex, x [len(phis)][len(samples)]).
    """
    n, h = system['n'], system['h']
    g = ham.Grid(n, h)
    noise = [osgw.white_noise(g, seed, stream, s, n_eta + 1) for s in samples]
    nproc = processes or min(os.cpu_count() or 1, max(len(samples) * (n_eta + 1), 1))
    ctx = mp.get_context('spawn')
    init = (n, h, np.asarray(system['vloc'], dtype=np.float64), system['kb_atoms'], spectrum[0], spectrum[1],
            e_homo, e_lumo, 1)
    with ctx.Pool(nproc, initializer=_init, initargs=init) as pool:
        jobs = [(noise[i][v], coeffs) for i in range(len(samples)) for v in range(n_eta + 1)]
        flat = pool.map(_filter_vector, jobs, chunksize=1)
        filt = [np.stack(flat[i * (n_eta + 1):(i + 1) * (n_eta + 1)]) for i in range(len(samples))]
        jobs = [(noise[i][0], filt[i], np.asarray(phi, dtype=np.float64), n_steps, dt, K)
                for phi in phis for i in range(len(samples))]
        res = pool.map(_sample_response, jobs, chunksize=1)
    ns = len(samples)
    sig = [[res[o * ns + i][0] for i in range(ns)] for o in range(len(phis))]
    xs = [[res[o * ns + i][1] for i in range(ns)] for o in range(len(phis))]
    return np.array(sig), np.array(xs)
