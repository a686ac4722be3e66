"""The oracle's process-pool driver (`oracle.parallel`) against its serial definition
(`oracle.sgw.run_sample`): the pool only splits a batch into the pieces the method computes
independently, so every Sigma_i(t) and X_i must agree with the serial sample to rounding."""
import numpy as np

from oracle import chebyshev as cheb
from oracle import parallel
from oracle import sgw as osgw
from paper_2601_21005_gb300 import synth

import gpu_common as gc


def test_pool_matches_serial_samples_for_two_orbitals():
    s = synth.wells()
    g, kb, w, phis = gc.oracle_eigs(s, 6)
    lo, hi = -4.0, 45.0
    a = cheb.gapped_filter_coeffs(w[3], w[4], lo, hi, 32)
    n_eta, N, dt, K = 4, 6, 0.05, 12
    samples = [3, 5]
    sig, xs = parallel.run_samples(s, (lo, hi), w[3], w[4], a, 77, 2, samples, n_eta, [phis[3], phis[4]], N, dt, K,
                                   processes=2)
    assert sig.shape == (2, 2, 2 * N + 1) and xs.shape == (2, 2)
    for o, phi in enumerate((phis[3], phis[4])):
        prob = osgw.Problem(g, s['vloc'], None, lo, hi, w[3], w[4], phi)
        for i, smp in enumerate(samples):
            ref, x, _ = osgw.run_sample(prob, a, 77, 2, smp, n_eta, N, dt, K)
            assert np.max(np.abs(sig[o, i] - ref)) <= 1e-12 * np.max(np.abs(ref))
            assert abs(xs[o, i] - x) <= 1e-12 * abs(x)
    # the two orbitals give different self-energies from the same noise
    assert np.max(np.abs(sig[0] - sig[1])) > 1e-3 * np.max(np.abs(sig[0]))
