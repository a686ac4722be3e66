"""Whole MC samples on the 288^3 large-cluster grid with the xi-compressed u (a measurement).

    python -m paper_2601_21005_gb300.large_cluster [--steps 20] [--radius 61] [--n-xi 10000]
    python -m paper_2601_21005_gb300.large_cluster --ks --gap --steps 1000 --n-cheb 7000 --batches 1
    python -m paper_2601_21005_gb300.large_cluster --gap-only --count-degree 8000

Builds the H-capped Si cluster of the given radius on a 288^3 grid (h = 0.5 bohr; radius 61 gives
Si7055H1596) with local and KB potentials, estimates the spectral interval on the GPU, and runs
pipeline batches (4 samples each: white noise, the occupied filter, exchange, TDH with the sparse
stochastic projection of u^R, time ordering of the overlaps, zeta propagation and Sigma(t)), timed
with CUDA events.  Without --ks the occupied window and the target orbital are synthetic and the run
measures cost and memory, not a QP energy.  With --ks, E_HOMO, E_LUMO and the HOMO and LUMO orbitals
come from the interior eigensolver (eigensolver.states_near_gap: kernel-polynomial gap search, a
Gaussian-filtered subspace iteration); with --gap as well, each batch runs once for phi = HOMO and
once for phi = LUMO on the same noise and filter (the filtered batch is reused), and the QP
energies of both (Eq. 6-7, gamma = 3 / (N_tau dt)) and the gap are reported with their standard
errors.  --gap-only runs just the kernel-polynomial state count and density of states near the gap.
Prints one JSON line.
"""
import argparse
import json
import time

import numpy as np

HA_EV = 27.211386245988


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
    ap.add_argument('--samples', type=int, default=1, help='MC samples per batch')
    ap.add_argument('--batches', type=int, default=1)
    ap.add_argument('--ks', action='store_true', help='KS inputs from the interior eigensolver')
    ap.add_argument('--gap', action='store_true', help='with --ks: QP energies of the HOMO and the LUMO and the gap')
    ap.add_argument('--gap-only', action='store_true',
                    help='only the kernel-polynomial gap search (state count and density of states near n_occ)')
    ap.add_argument('--ks-max-iter', type=int, default=60)
    ap.add_argument('--ks-m', type=int, default=24, help='block size of the interior eigensolver')
    ap.add_argument('--ks-degree', type=int, default=8000, help='degree of its Gaussian window')
    ap.add_argument('--count-degree', type=int, default=2000,
                    help='degree of the kernel-polynomial moments (resolution about pi (E_max - E_min) / 2 / degree)')
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
        mu = cheb_moments(kctx, emin, emax, 16, args.count_degree)
        ef, n_ef, se_ef = find_gap(mu, s['n_occ'], emin, emax)
        e = np.linspace(ef - 0.15, ef + 0.15, 61)
        cnt, se, dos = count_and_dos(mu, e, emin, emax)
        kctx.close()
        print(json.dumps(dict(workload=s['name'], n_occ=s['n_occ'], spectrum=[emin, emax], gap_centre=ef,
                              count_at_gap=n_ef, count_se=se_ef, seconds=round(time.perf_counter() - t1, 1),
                              scan=dict(e=e.round(4).tolist(), count=cnt.round(1).tolist(), dos=dos.round(1).tolist()))))
        return
    phi_lumo = None
    if args.ks:
        from . import sgw
        from .eigensolver import states_near_gap
        t1 = time.perf_counter()
        kctx = sgw.Context(n, h, max_batch=max(args.ks_m, 16))
        kctx.set_potential(torch.as_tensor(s['vloc'].reshape(-1).astype(np.float32)).cuda(), s['kb_atoms'])
        (emin, emax), _ = kctx.spectral_bounds(200, 1000, 0.05)
        e_homo, e_lumo, phi, info = states_near_gap(kctx, s['n_occ'], emin, emax, m=args.ks_m, n_probe=16,
                                                    count_degree=args.count_degree, window_degree=args.ks_degree,
                                                    max_iter=args.ks_max_iter, log=lambda m: print(m, flush=True))
        kctx.close()
        phi_lumo = info['phi_lumo']
        ks = dict(e_homo=e_homo, e_lumo=e_lumo, gap_eV=(e_lumo - e_homo) * HA_EV, gap_centre=info['gap_centre'],
                  count_at_gap=info['count_at_gap'], count_se=info['count_se'], max_residual=info['max_residual'],
                  seconds=round(time.perf_counter() - t1, 1))
        print(json.dumps(dict(ks=ks)), flush=True)
    else:
        e_homo, e_lumo = -0.15, -0.05
        phi = synth.smooth_orbital(n, h, (c, c, c), width=3.0)
        phi /= np.sqrt(h ** 3 * np.sum(phi ** 2))
    N, ns = args.steps, args.samples
    pl = Pipeline(n, h, s['vloc'], s['kb_atoms'], phi, e_homo, e_lumo, n_eta=8, n_steps=N, dt=0.05, cheb_deg=16,
                  n_cheb=args.n_cheb, samples_per_batch=ns, zeta_group=1,
                  xi=dict(n_xi=args.n_xi, f_g=args.f_g, L=32))
    orbitals = [('homo', pl.phi.clone(), e_homo)]
    if args.gap and phi_lumo is not None:
        orbitals.append(('lumo', torch.as_tensor(phi_lumo.astype(np.float32).reshape(-1)).to(pl.dev), e_lumo))
    res = {name: (torch.empty(args.batches * ns, 2 * N + 1, dtype=torch.complex128, device=pl.dev),
                  torch.empty(args.batches * ns, dtype=torch.float64, device=pl.dev)) for name, _, _ in orbitals}
    torch.cuda.synchronize()
    pl.ctx.profile(True)
    times = dict(filter=0.0, propagate={name: 0.0 for name, _, _ in orbitals})
    ev = lambda: torch.cuda.Event(enable_timing=True)
    for bt in range(args.batches):
        s0 = bt * ns
        e0, e1 = ev(), ev()
        e0.record()
        pl.filter_batch(s0)
        e1.record()
        torch.cuda.synchronize()
        times['filter'] += e0.elapsed_time(e1)
        for name, ph, _ in orbitals:
            pl.phi.copy_(ph)
            e0, e1 = ev(), ev()
            e0.record()
            pl.propagate_batch(s0, res[name][0][s0:s0 + ns], res[name][1][s0:s0 + ns])
            e1.record()
            torch.cuda.synchronize()
            times['propagate'][name] += e0.elapsed_time(e1)
            print(json.dumps(dict(batch=bt, orbital=name, seconds=round(e0.elapsed_time(e1) * 1e-3, 1))), flush=True)
    prof = pl.ctx.profile_read()
    pl.ctx.profile(False)
    qp = {}
    for name, _, eps in orbitals:
        sig, xs = res[name]
        if sig.shape[0] >= 2 and args.ks:
            r = pl.qp(sig, xs, eps)
            qp[name] = dict(eps_ks_eV=eps * HA_EV, qp_eV=r['eps_qp'] * HA_EV, se_eV=r['se'] * HA_EV, z=r['z'])
    gap = None
    if 'homo' in qp and 'lumo' in qp:
        gap = dict(qp_gap_eV=qp['lumo']['qp_eV'] - qp['homo']['qp_eV'],
                   se_eV_uncorrelated=(qp['lumo']['se_eV'] ** 2 + qp['homo']['se_eV'] ** 2) ** 0.5,
                   ks_gap_eV=(e_lumo - e_homo) * HA_EV)
    u_bytes = pl.u.numel() * pl.u.element_size() + pl.uR.numel() * pl.uR.element_size()
    print(json.dumps(dict(
        workload='Si cluster radius %.1f bohr (%d atoms with KB, %d occupied states), 288^3 grid h=0.5 bohr'
                 % (args.radius, len(s['kb_atoms']), s['n_occ']),
        ks=ks, steps=N, n_cheb=args.n_cheb, n_eta=8, samples=args.batches * ns, gamma=pl.gamma,
        xi=dict(n_xi=args.n_xi, f_g=args.f_g, L=32), spectrum=[pl.emin, pl.emax], seconds_system=round(t_sys, 1),
        seconds_filter=round(times['filter'] * 1e-3, 1),
        seconds_propagate={k: round(v * 1e-3, 1) for k, v in times['propagate'].items()},
        sigma_finite=bool(all(torch.isfinite(r[0]).all().item() for r in res.values())), qp=qp, gap=gap,
        u_bytes=int(u_bytes), u_bytes_full_grid_equivalent=int((N + 1) * n ** 3 * 12 * ns),
        peak_device_gb=round(torch.cuda.max_memory_allocated() / 1e9, 2),
        kinds={k: dict(ms=round(v['ms'], 1), launches=v['launches']) for k, v in prof.items() if v['launches']})))


if __name__ == '__main__':
    main()
