"""Writes tests/golden/qp_gap_si35h36_64.npz: oracle-only inputs and expected values of the QP-gap
parity case on the 64^3 Si35H36 cluster (h = 0.5 bohr, 176 electrons, s/p KB on Si).

    python tests/golden/make_qp_gap_64.py [--processes P]

Everything stored comes from the FP64 oracle (`oracle/`) on the seeded synthetic input
(`paper_2601_21005_gb300/synth.py`, which holds no arithmetic of the method):

* the Kohn-Sham inputs of Sec. 2.1 (E_HOMO, E_LUMO and both orbitals): ARPACK (scipy `eigsh`,
  the textbook Lanczos routine) on the oracle's H0 for the lowest 90 states; the orbitals are
  stored rounded to float32, and the expected values below are computed from those rounded
  orbitals, so the parity test hands both sides the identical phi;
* the spectral interval: the oracle's shifted power iteration (Sec. 2.1), 200 iterations,
  5% margin;
* the gapped-filter coefficients of degree 2000 (Eq. 3);
* Sigma_i(t) (Eq. 4-5) and X_i of 2 Monte-Carlo samples for phi = HOMO and phi = LUMO (the same
  noise and filter for both), N_eta = 8, 20 steps of dt = 0.05 with the degree-16 Chebyshev
  propagator, and the QP energies of Eq. 6-7 (gamma = 3 / (N_tau dt)) with their gap.

The filter degree and KB part are those of the 64^3 workload; N_tau is cut from 400 to 20 so
that the oracle finishes in minutes.
"""
import argparse
import os
import sys
import time

import numpy as np
import scipy.sparse.linalg as sla

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import chebyshev as cheb      # noqa: E402
from oracle import hamiltonian as ham     # noqa: E402
from oracle import parallel               # noqa: E402
from oracle import sgw as osgw            # noqa: E402
from oracle.philox import rademacher_words  # noqa: E402
from paper_2601_21005_gb300 import synth  # noqa: E402

N_CHEB, N_ETA, N_STEPS, DT, K = 2000, 8, 20, 0.05, 16
SEED, STREAM, SAMPLES = 2000, 1, (0, 1)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument('--processes', type=int, default=None)
    ap.add_argument('--out', default=os.path.join(HERE, 'qp_gap_si35h36_64.npz'))
    args = ap.parse_args()
    t0 = time.time()
    s = synth.si_cluster(n=64, h=0.5, radius=10.5)
    g = ham.Grid(64, 0.5)
    kb = ham.KB(s['kb_atoms'])
    n_occ = s['n_occ']

    def h0(v):
        return ham.apply_h(v, g, s['vloc'], kb)

    op = sla.LinearOperator((g.ng, g.ng), matvec=lambda x: h0(x.reshape(g.shape()).astype(np.complex128))
                            .real.reshape(-1), dtype=np.float64)
    w, v = sla.eigsh(op, k=n_occ + 2, which='SA', tol=1e-10, v0=np.ones(g.ng))
    order = np.argsort(w)
    w, v = w[order], v[:, order]
    # dV-norm of H phi - E phi (phi = v / sqrt(dV))
    res = [float(np.linalg.norm(op.matvec(v[:, i]) - w[i] * v[:, i])) for i in (n_occ - 1, n_occ)]
    phis = []
    for i in (n_occ - 1, n_occ):
        p = v[:, i].reshape(g.shape()) / np.sqrt(g.dV)
        if p.sum() < 0:
            p = -p
        phis.append(p.astype(np.float32))
    e_homo, e_lumo = float(w[n_occ - 1]), float(w[n_occ])
    print('KS: E_HOMO %.8f E_LUMO %.8f (degeneracies %s) residuals %s  [%.0f s]'
          % (e_homo, e_lumo, np.round(w[n_occ - 4:n_occ + 2], 8), res, time.time() - t0), flush=True)
    v0 = rademacher_words(SEED, 0xB0B0, 0, 0, g.ng).astype(np.float64).reshape(g.shape()) + 0j
    (emin, emax), raw = cheb.spectral_bounds(h0, v0, 200, g.dot, 0.05)
    coeffs = cheb.gapped_filter_coeffs(e_homo, e_lumo, emin, emax, N_CHEB)
    print('spectrum [%.6f, %.6f] (raw %s)  [%.0f s]' % (emin, emax, raw, time.time() - t0), flush=True)
    sig, xs = parallel.run_samples(s, (emin, emax), e_homo, e_lumo, coeffs, SEED, STREAM, list(SAMPLES), N_ETA,
                                   [p.astype(np.float64) for p in phis], N_STEPS, DT, K, processes=args.processes)
    gamma = 3.0 / (N_STEPS * DT)
    qp, se = [], []
    for o, eps in enumerate((e_homo, e_lumo)):
        e, err = osgw.qp_energy(list(sig[o]), list(xs[o]), DT, gamma, eps)
        qp.append(e)
        se.append(err)
    print('QP HOMO %.6f LUMO %.6f Ha, gap %.4f eV  [%.0f s]' % (qp[0], qp[1], (qp[1] - qp[0]) * 27.211386245988,
                                                             time.time() - t0), flush=True)
    np.savez_compressed(args.out, phi_homo=phis[0], phi_lumo=phis[1], e_homo=e_homo, e_lumo=e_lumo,
                        eig_residuals=np.array(res), emin=emin, emax=emax, coeffs=coeffs, seed=SEED, stream=STREAM,
                        samples=np.array(SAMPLES), n_eta=N_ETA, n_steps=N_STEPS, dt=DT, cheb_deg=K,
                        sigma=sig, x=xs, qp=np.array(qp), se=np.array(se))


if __name__ == '__main__':
    main()
