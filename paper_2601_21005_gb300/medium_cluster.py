"""The control variate on the 128^3 medium cluster (a measurement).

    python -m paper_2601_21005_gb300.medium_cluster [--train 48] [--paired-batches 4] [--cheap 4096]

Builds the H-capped Si cluster Si657H300 on a 128^3 grid (h = 0.5 bohr, radius 28 bohr, s/p KB on
Si), takes E_HOMO, E_LUMO and the HOMO orbital from the interior eigensolver
(eigensolver.states_near_gap), and runs the pipeline with 16 MC samples per run (256 TDH orbitals
per launch), u^R in the xi basis of the paper's runs (N_xi = 10^4, f_g = 0.003; full-grid u of 16
samples over 400 steps would take 100 GB) and the occupied filter of degree --n-cheb.  It
trains the control variate on --train plain samples and compares, at equal error on the QP energy
(+-0.03 eV), the plain estimator with the control-variate estimator (control_variate.study):
variance gains of the linear part alone, of the linear part with the network on its residual and of
the network alone, and the time to the target with and without the training.  Prints the KS inputs
as one JSON line, then the study as another.
"""
import argparse
import json
import time

import numpy as np

HA_EV = 27.211386245988


def main():
    import torch
    from . import build, sgw, synth
    from .control_variate import study
    from .eigensolver import states_near_gap
    from .pipeline import Pipeline
    ap = argparse.ArgumentParser()
    ap.add_argument('--steps', type=int, default=400)
    ap.add_argument('--n-cheb', type=int, default=4000)
    ap.add_argument('--train', type=int, default=48)
    ap.add_argument('--paired-batches', type=int, default=4, help='runs of 16 paired samples')
    ap.add_argument('--cheap', type=int, default=4096)
    ap.add_argument('--ks-degree', type=int, default=4000)
    ap.add_argument('--ks-iter', type=int, default=30, help='interior-solver iterations')
    args = ap.parse_args()
    build.build()
    n, h = 128, 0.5
    s = synth.si_cluster(n=n, h=h, radius=28.0)
    t0 = time.perf_counter()
    kctx = sgw.Context(n, h, max_batch=16)
    kctx.set_potential(torch.as_tensor(s['vloc'].reshape(-1).astype(np.float32)).cuda(), s['kb_atoms'])
    (emin, emax), _ = kctx.spectral_bounds(200, 1000, 0.05)
    e_homo, e_lumo, phi, info = states_near_gap(kctx, s['n_occ'], emin, emax, m=16, count_degree=3000,
                                                window_degree=args.ks_degree, max_iter=args.ks_iter)
    kctx.close()
    ks = dict(e_homo=e_homo, e_lumo=e_lumo, gap_eV=(e_lumo - e_homo) * HA_EV, max_residual=info['max_residual'],
              gap_centre=info['gap_centre'], seconds=round(time.perf_counter() - t0, 1))
    print(json.dumps(dict(ks=ks)), flush=True)
    pl = Pipeline(n, h, s['vloc'], s['kb_atoms'], phi, e_homo, e_lumo, n_eta=8, n_steps=args.steps, dt=0.05,
                  cheb_deg=16, n_cheb=args.n_cheb, samples_per_batch=16, zeta_group=1, seed=4000, stream_id=1,
                  spectrum=(emin, emax), graphs=True, xi=dict(n_xi=10000, f_g=0.003, L=32))
    # the plain form is charged the time of the paired runs (the plain pipeline plus features that
    # take milliseconds); the training runs come first and capture the graphs
    res = study(pl, e_homo, args.train, args.paired_batches, args.cheap, 0, None)
    plain_s = res['seconds_per_sample']['plain']
    print(json.dumps(dict(
        workload='%s cluster, 128^3 grid h=0.5 bohr, %d electrons, 16 MC samples (256 TDH orbitals) per run, '
                 '%d steps, filter degree %d, xi-compressed u (N_xi=10000, f_g=0.003)'
                 % (s['name'], 2 * s['n_occ'], args.steps, args.n_cheb),
        ks=ks, gamma=pl.gamma, plain_seconds_per_sample=round(plain_s, 3), control_variate=res)))


if __name__ == '__main__':
    main()
