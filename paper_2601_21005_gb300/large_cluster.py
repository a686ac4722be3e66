"""Whole MC samples on the 288^3 large-cluster grid with the xi-compressed u (a measurement).

    python -m paper_2601_21005_gb300.large_cluster [--steps 20] [--radius 61] [--n-xi 10000]

Builds the H-capped Si cluster of the given radius on a 288^3 grid (h = 0.5 bohr; radius 61 gives
Si7055H1596) with local and KB potentials, estimates the spectral interval on the GPU, and runs one
pipeline batch (one sample: white noise, a degree-2000 occupied filter, exchange, TDH with the
sparse stochastic projection of u^R, time ordering of the overlaps, zeta propagation and Sigma(t))
for --steps time steps, timed with CUDA events and with the per-kernel-kind device times.  Without
--ks the occupied window and the target orbital are synthetic and the run measures cost and memory,
not a QP energy; with --ks, E_HOMO, E_LUMO and the HOMO orbital come from the interior eigensolver
(eigensolver.states_near_gap: kernel-polynomial gap search, Gaussian-filtered subspace iteration) and
the HOMO/LUMO gap is reported.  Prints one JSON line.
"""
import argparse
import json
import time

import numpy as np


def main():
    import torch
    from . import build, synth
    from .pipeline import Pipeline
    ap = argparse.ArgumentParser()
    ap.add_argument('--steps', type=int, default=20)
    ap.add_argument('--radius', type=float, default=61.0)
    ap.add_argument('--n-xi', type=int, default=10000)
    ap.add_argument('--f-g', type=float, default=0.003)
    ap.add_argument('--n-cheb', type=int, default=2000)
    ap.add_argument('--ks', action='store_true', help='KS inputs from the interior eigensolver')
    ap.add_argument('--gap-only', action='store_true',
                    help='only the kernel-polynomial gap search (state count and density of states near n_occ)')
    ap.add_argument('--ks-max-iter', type=int, default=60)
    args = ap.parse_args()
    build.build()
    n, h = 288, 0.5
    t0 = time.perf_counter()
    s = synth.si_cluster(n=n, h=h, radius=args.radius)
    t_sys = time.perf_counter() - t0
    c = 0.5 * n * h
    ks = None
    if args.gap_only:
        from . import sgw
        from .eigensolver import cheb_moments, count_and_dos, find_gap
        t1 = time.perf_counter()
        kctx = sgw.Context(n, h, max_batch=16)
        kctx.set_potential(torch.as_tensor(s['vloc'].reshape(-1).astype(np.float32)).cuda(), s['kb_atoms'])
        (emin, emax), _ = kctx.spectral_bounds(200, 1000, 0.05)
        mu = cheb_moments(kctx, emin, emax, 16, 2000)
        ef, n_ef, se_ef = find_gap(mu, s['n_occ'], emin, emax)
        e = np.linspace(ef - 0.3, ef + 0.3, 61)
        cnt, se, dos = count_and_dos(mu, e, emin, emax)
        kctx.close()
        print(json.dumps(dict(workload=s['name'], n_occ=s['n_occ'], spectrum=[emin, emax], gap_centre=ef,
                              count_at_gap=n_ef, count_se=se_ef, seconds=round(time.perf_counter() - t1, 1),
                              scan=dict(e=e.round(4).tolist(), count=cnt.round(1).tolist(), dos=dos.round(1).tolist()))))
        return
    if args.ks:
        from . import sgw
        from .eigensolver import states_near_gap
        t1 = time.perf_counter()
        kctx = sgw.Context(n, h, max_batch=32)
        kctx.set_potential(torch.as_tensor(s['vloc'].reshape(-1).astype(np.float32)).cuda(), s['kb_atoms'])
        (emin, emax), _ = kctx.spectral_bounds(200, 1000, 0.05)
        e_homo, e_lumo, phi, info = states_near_gap(kctx, s['n_occ'], emin, emax, m=32, sigma=0.05, n_probe=16,
                                                    count_degree=2000, window_degree=1500,
                                                    max_iter=args.ks_max_iter, log=lambda m: print(m, flush=True))
        kctx.close()
        ks = dict(e_homo=e_homo, e_lumo=e_lumo, gap_eV=(e_lumo - e_homo) * 27.211386245988,
                  gap_centre=info['gap_centre'], count_at_gap=info['count_at_gap'], count_se=info['count_se'],
                  max_residual=info['max_residual'], seconds=round(time.perf_counter() - t1, 1))
    else:
        e_homo, e_lumo = -0.15, -0.05
        phi = synth.smooth_orbital(n, h, (c, c, c), width=3.0)
        phi /= np.sqrt(h ** 3 * np.sum(phi ** 2))
    N = args.steps
    pl = Pipeline(n, h, s['vloc'], s['kb_atoms'], phi, e_homo, e_lumo, n_eta=8, n_steps=N, dt=0.05, cheb_deg=16,
                  n_cheb=args.n_cheb, samples_per_batch=1, zeta_group=1,
                  xi=dict(n_xi=args.n_xi, f_g=args.f_g, L=32))
    sig = torch.empty(1, 2 * N + 1, dtype=torch.complex128, device=pl.dev)
    x = torch.empty(1, dtype=torch.float64, device=pl.dev)
    torch.cuda.synchronize()
    pl.ctx.profile(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    pl.run_batch(0, sig, x)
    e1.record()
    torch.cuda.synchronize()
    prof = pl.ctx.profile_read()
    pl.ctx.profile(False)
    u_bytes = pl.u.numel() * pl.u.element_size() + pl.uR.numel() * pl.uR.element_size()
    print(json.dumps(dict(
        workload='Si cluster radius %.1f bohr (%d atoms with KB, %d occupied states), 288^3 grid h=0.5 bohr'
                 % (args.radius, len(s['kb_atoms']), s['n_occ']),
        ks=ks, steps=N, n_cheb=args.n_cheb, n_eta=8, xi=dict(n_xi=args.n_xi, f_g=args.f_g, L=32),
        spectrum=[pl.emin, pl.emax], seconds_system=round(t_sys, 1), ms_sample=e0.elapsed_time(e1),
        sigma_finite=bool(torch.isfinite(sig).all().item()), u_bytes=int(u_bytes),
        u_bytes_full_grid_equivalent=int((N + 1) * n ** 3 * 12),
        peak_device_gb=round(torch.cuda.max_memory_allocated() / 1e9, 2),
        kinds={k: dict(ms=round(v['ms'], 1), launches=v['launches']) for k, v in prof.items() if v['launches']})))


if __name__ == '__main__':
    main()
