"""Micro-benchmark of the propagation kernels on one batch (also the small case for ncu).

    python -m paper_2601_21005_gb300.kernel_bench [--n 64] [--batch 64] [--steps 2] [--deg 16]

Sets up the Si35H36 cluster (local + KB potentials) on an n^3 grid, fills a batch of
complex vectors with Philox noise and propagates it n_steps steps with the degree-`deg`
Chebyshev expansion through the C ABI, timing each kernel kind with CUDA events.  Device
memory: four batch-sized complex arrays (0.5 GB at 64^3 x 64).
"""
import argparse
import json

import numpy as np


def main():
    import torch
    from . import build, sgw, synth
    ap = argparse.ArgumentParser()
    ap.add_argument('--n', type=int, default=64)
    ap.add_argument('--batch', type=int, default=64)
    ap.add_argument('--steps', type=int, default=2)
    ap.add_argument('--deg', type=int, default=16)
    ap.add_argument('--no-kb', action='store_true')
    ap.add_argument('--radius', type=float, default=None,
                    help='cluster radius in bohr (default 10.5 = Si35H36; 28.0 = Si657H300 at n = 128)')
    ap.add_argument('--tune', default=None,
                    help='semicolon-separated settings "operands,plane_lookahead,pencil_lookahead,variant,line_tile" '
                         '(a prefix of the tuning keys) to time in turn')
    ap.add_argument('--autotune', action='store_true', help='run the library autotuner first and report its choice')
    ap.add_argument('--split', action='store_true', help='time the split-operator propagator instead of Chebyshev')
    args = ap.parse_args()
    build.build()
    radius = args.radius if args.radius is not None else (10.5 if args.n >= 64 else 4.5)
    s = synth.si_cluster(n=args.n, h=0.5, radius=radius)
    ctx = sgw.Context(args.n, 0.5, max_batch=args.batch)
    ctx.set_potential(torch.as_tensor(s['vloc'].reshape(-1).astype(np.float32)).cuda(),
                      [] if args.no_kb else s['kb_atoms'])
    ctx.set_spectrum(float(s['vloc'].min()) - 1.0, 0.5 * 3 * (np.pi / 0.5) ** 2 + 3.0)
    ng = args.n ** 3
    psi = torch.empty(args.batch, ng, dtype=torch.complex64, device='cuda')
    ctx.white_noise(5, 3, 0, 1, args.batch, psi)
    chosen = ctx.autotune(args.batch) if args.autotune else None
    settings = [None]
    if args.tune:
        settings = [tuple(int(v) for v in t.split(',')) for t in args.tune.split(';')]
    for st in settings:
        if st is not None:
            for k, v in enumerate(st):
                ctx.set_tuning(k, v)
        tuning = [ctx.get_tuning(k) for k in range(ctx.TUNE_KEYS)]
        step = (lambda k: ctx.propagate_split(psi, k, 0.05)) if args.split else \
            (lambda k: ctx.propagate(psi, k, 0.05, args.deg))
        step(1)                                          # warm-up
        torch.cuda.synchronize()
        ctx.profile(True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        step(args.steps)
        e1.record()
        prof = ctx.profile_read()
        ctx.profile(False)
        wall_ms = e0.elapsed_time(e1)
        out = {}
        for k, v in prof.items():
            if v['launches']:
                out[k] = dict(launches=v['launches'], avg_us=round(1e3 * v['ms'] / v['launches'], 2),
                              alg_GBps=round(v['alg_bytes'] / (v['ms'] * 1e-3) / 1e9, 1) if v['alg_bytes'] else None)
        print(json.dumps(dict(n=args.n, batch=args.batch, steps=args.steps, deg=args.deg, tuning=tuning,
                              propagator='split' if args.split else 'chebyshev', autotuned=chosen,
                              pts_vec_steps_per_s=args.n ** 3 * args.batch * args.steps / (wall_ms * 1e-3),
                              kernels=out)), flush=True)


if __name__ == '__main__':
    main()
