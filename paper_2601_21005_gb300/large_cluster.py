"""Whole MC samples on the 288^3 large-cluster grid with the xi-compressed u (a measurement).

    python -m paper_2601_21005_gb300.large_cluster [--steps 20] [--radius 61] [--n-xi 10000]

Builds the H-capped Si cluster of the given radius on a 288^3 grid (h = 0.5 bohr; radius 61 gives
Si7055H1596) with local and KB potentials, estimates the spectral interval on the GPU, and runs one
pipeline batch (one sample: white noise, a degree-2000 occupied filter, exchange, TDH with the
sparse stochastic projection of u^R, time ordering of the overlaps, zeta propagation and Sigma(t))
for --steps time steps, timed with CUDA events and with the per-kernel-kind device times.  The
occupied window and the target orbital are synthetic (no KS inputs at this size): the run measures
cost and memory, not a QP energy.  Prints one JSON line.
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
    args = ap.parse_args()
    build.build()
    n, h = 288, 0.5
    t0 = time.perf_counter()
    s = synth.si_cluster(n=n, h=h, radius=args.radius)
    t_sys = time.perf_counter() - t0
    c = 0.5 * n * h
    phi = synth.smooth_orbital(n, h, (c, c, c), width=3.0)
    phi /= np.sqrt(h ** 3 * np.sum(phi ** 2))
    N = args.steps
    pl = Pipeline(n, h, s['vloc'], s['kb_atoms'], phi, -0.15, -0.05, n_eta=8, n_steps=N, dt=0.05, cheb_deg=16,
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
        steps=N, n_cheb=args.n_cheb, n_eta=8, xi=dict(n_xi=args.n_xi, f_g=args.f_g, L=32),
        spectrum=[pl.emin, pl.emax], seconds_system=round(t_sys, 1), ms_sample=e0.elapsed_time(e1),
        sigma_finite=bool(torch.isfinite(sig).all().item()), u_bytes=int(u_bytes),
        u_bytes_full_grid_equivalent=int((N + 1) * n ** 3 * 12),
        peak_device_gb=round(torch.cuda.max_memory_allocated() / 1e9, 2),
        kinds={k: dict(ms=round(v['ms'], 1), launches=v['launches']) for k, v in prof.items() if v['launches']})))


if __name__ == '__main__':
    main()
