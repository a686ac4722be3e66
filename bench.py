#!/usr/bin/env python
"""Benchmark of the stochastic-GW hot path on one node (one process per GPU).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--config NAME]

One step = one pass of the whole hot path over one batch of Monte-Carlo samples of the
workload: white noise, gapped filter (Eq. 3), exchange, linear-response TDH (u^R), time
ordering, zeta propagation with the Sigma(t) accumulation (Eq. 4-5), and the QP solve
(Eq. 6-7) on the samples accumulated so far.  Default workload: the 64^3 Si35H36 cluster
(h = 0.5 bohr, 176 electrons), 4 samples x 16 orbitals (8 eta pairs) = 64 orbitals
propagated for 400 steps of dt = 0.05 with Chebyshev degree 16, filter degree 2000.

The metric counts grid points x propagated orbitals x time steps of the TDH propagation
per second of the whole step.  With --impl reference the FP64 CPU oracle is timed on a
bounded sample of the same workload instead (see `oracle_sample`).
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = 'grid-pt*orbital*steps/s and time to +/-0.03 eV QP energy, chosen vs plain form'
UNIT = 'grid-pt*orbital*steps/s'
HA_EV = 27.211386245988

CONFIGS = {
    # the 64^3 cluster the metric is quoted on
    'si35h36_64': dict(system='si_cluster', n=64, h=0.5, radius=10.5, samples_per_batch=4, zeta_group=4, n_eta=8,
                       n_steps=400, dt=0.05, cheb_deg=16, n_cheb=2000, workload='Si35H36 cluster, 64^3 grid '
                       'h=0.5 bohr, 176 electrons, 64 orbitals per TDH launch (4 MC samples x 8 eta pairs) x '
                       '400 steps; 16 MC samples per step, their 32 zeta vectors propagated together'),
    # the tiny periodic case (parity-test size)
    'wells16': dict(system='wells', n=16, h=0.6, samples_per_batch=1, zeta_group=1, n_eta=8, n_steps=200, dt=0.05,
                    cheb_deg=16, n_cheb=128, workload='6 Gaussian wells, 16^3 grid h=0.6 bohr, 8 electrons, '
                    '16 orbitals x 200 steps'),
}


def load_peaks():
    p = os.path.join(ROOT, 'MEASURED_PEAKS.json')
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return dict(hbm_gbs=float(d['hbm_gbs']), bf16_tflops=float(d['bf16_tflops']), source='measured')
    return dict(hbm_gbs=6800.0, bf16_tflops=1900.0, source='fallback')


class ClockSampler:
    """nvidia-smi clock / throttle-reason samples during the timed region."""
    Q = ('index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,'
         'clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,'
         'clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap')

    def __init__(self, device):
        self.device = device
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix='.csv')
        os.close(fd)
        try:
            self.f = open(self.path, 'w')
            self.proc = subprocess.Popen(['nvidia-smi', '-i', str(self.device), '--query-gpu=' + self.Q,
                                          '--format=csv,noheader,nounits', '-lms', '200'],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return dict(sm_mhz=None, sm_max_mhz=None, reasons=['nvidia-smi unavailable'])
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        rows = []
        with open(self.path) as f:
            for line in f:
                p = [x.strip() for x in line.split(',')]
                if len(p) >= 9:
                    rows.append(p)
        os.unlink(self.path)
        if not rows:
            return dict(sm_mhz=None, sm_max_mhz=None, reasons=['no samples'])
        sm = [float(r[1]) for r in rows if r[1].replace('.', '').isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace('.', '').isdigit()]
        names = ['hw_slowdown', 'hw_thermal_slowdown', 'sw_thermal_slowdown', 'sw_power_cap']
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == 'active'})
        pw = [float(r[3]) for r in rows if r[3].replace('.', '').isdigit()]
        return dict(sm_mhz=statistics.median(sm) if sm else None, sm_max_mhz=max(mx) if mx else None,
                    reasons=reasons, samples=len(rows), power_w_max=max(pw) if pw else None)


# ---------------------------------------------------------------- workload setup (untimed)
def build_system(cfg):
    from paper_2601_21005_gb300 import synth
    if cfg['system'] == 'wells':
        return synth.wells(n=cfg['n'], h=cfg['h'])
    return synth.si_cluster(n=cfg['n'], h=cfg['h'], radius=cfg['radius'])


def kohn_sham_inputs(cfg, sysd, device):
    """E_HOMO, E_LUMO and the HOMO orbital (the preliminary-DFT inputs of Sec. 2.1) from a GPU
    subspace iteration through libsgw, plus the spectral interval by shifted power iteration."""
    import torch
    from paper_2601_21005_gb300 import sgw
    from paper_2601_21005_gb300.eigensolver import lowest_states
    n_occ = sysd['n_occ']
    extra = max(8, n_occ // 4)
    ctx = sgw.Context(cfg['n'], cfg['h'], max_batch=n_occ + 1 + extra, device=device)
    vl = torch.as_tensor(sysd['vloc'].reshape(-1).astype('float32')).cuda(device)
    ctx.set_potential(vl, sysd['kb_atoms'])
    (emin, emax), raw = ctx.spectral_bounds(200, cfg.get('seed', 1000), 0.05)
    w, phis, res = lowest_states(ctx, n_occ + 1, emin, emax, extra=extra)
    ctx.close()
    return dict(e_homo=float(w[n_occ - 1]), e_lumo=float(w[n_occ]), phi=phis[n_occ - 1], emin=emin, emax=emax,
                raw_bounds=raw, eig_residual=res)


def make_pipeline(cfg, sysd, ks, device, seed, fp64=True, graphs=False, autotune=False, zeta_group=None):
    from paper_2601_21005_gb300.pipeline import Pipeline
    return Pipeline(cfg['n'], cfg['h'], sysd['vloc'], sysd['kb_atoms'], ks['phi'], ks['e_homo'], ks['e_lumo'],
                    n_eta=cfg['n_eta'], n_steps=cfg['n_steps'], dt=cfg['dt'], cheb_deg=cfg['cheb_deg'],
                    n_cheb=cfg['n_cheb'], samples_per_batch=cfg['samples_per_batch'], seed=seed, stream_id=1,
                    device=device, spectrum=(ks['emin'], ks['emax']), fp64=fp64, graphs=graphs, autotune=autotune,
                    zeta_group=cfg['zeta_group'] if zeta_group is None else zeta_group)


def step_samples(cfg):
    """MC samples of one bench step (one pipeline run)."""
    return cfg['samples_per_batch'] * cfg['zeta_group']


def units_per_step(cfg):
    """grid points x TDH-propagated orbitals x time steps of one bench step."""
    return cfg['n'] ** 3 * 2 * cfg['n_eta'] * step_samples(cfg) * cfg['n_steps']


# DRAM bytes (read + write, ncu) over algorithmic bytes of one 64-vector k_plane_step launch of the
# current kernel (profiles/plane_step_pencil_64x64.md); traffic per launch = this ratio x the
# launch's algorithmic bytes.  Must be re-measured whenever the plane kernel changes.
PLANE_STEP_DRAM_PER_ALG = 839.2 / 806.4


def roofline(prof, peaks):
    """Dominant kernel kind by device time; achieved = its algorithmic bytes / its event time."""
    kinds = {k: v for k, v in prof.items() if v['launches'] > 0 and v['alg_bytes'] > 0}
    total = sum(v['ms'] for v in prof.values())
    name = max(kinds, key=lambda k: kinds[k]['ms'])
    v = kinds[name]
    gbs = v['alg_bytes'] / (v['ms'] * 1e-3) / 1e9
    peak = peaks['hbm_gbs']
    shares = {k: round(x['ms'] / total, 4) for k, x in prof.items() if x['launches']}
    return dict(bound='hbm', achieved=round(gbs, 1), peak=peak, unit='GB/s', frac=round(gbs / peak, 4),
                traffic=(round(PLANE_STEP_DRAM_PER_ALG * v['alg_bytes'] / v['launches'])
                         if name == 'plane_step' else None),
                traffic_source='ncu dram__bytes_read.sum + dram__bytes_write.sum of a 64-vector launch, '
                               'scaled by algorithmic bytes to the average launch' if name == 'plane_step' else None,
                kernel=name, launches=v['launches'], avg_launch_us=round(1e3 * v['ms'] / v['launches'], 2),
                alg_bytes_per_launch=round(v['alg_bytes'] / v['launches']), peak_source=peaks['source'] + ' hbm_gbs',
                time_shares=shares,
                other_kernels={k: round(x['alg_bytes'] / (x['ms'] * 1e-3) / 1e9, 1) for k, x in kinds.items()})


def time_to_target(pl, sig, xs, eps_ks, seconds_per_sample, target_ev=0.03):
    """Samples needed for a QP standard error of target_ev, from the per-sample spread so far."""
    r = pl.qp(sig, xs, eps_ks)
    n = sig.shape[0]
    se_ev = r['se'] * HA_EV
    per_sample_ev = se_ev * n ** 0.5
    need = max(1.0, (per_sample_ev / target_ev) ** 2)
    return dict(seconds=round(need * seconds_per_sample, 3), samples_needed=round(need, 1),
                per_sample_std_eV=round(per_sample_ev, 4), qp_eV=round(r['eps_qp'] * HA_EV, 5),
                se_eV=round(se_ev, 5), z=round(r['z'], 4), n_samples_used=n)


# ---------------------------------------------------------------- the oracle on the host cores
def oracle_sample(cfg, n_filter_terms=2, n_tdh_steps=1, n_zeta_steps=1, seed=1000):
    """Time the FP64 oracle on a bounded sample of one batch and extrapolate to the batch.

    Timed pieces (one MC sample): n_filter_terms Chebyshev terms of the filter on the
    n_eta + 1 noise vectors, n_tdh_steps TDH steps of the n_eta pairs, n_zeta_steps zeta
    steps of the pair with the Sigma(t) sums, the exchange, and the time ordering of a
    4096-point slice of u^R over the full step count.  The batch time is
      n_samples * (N_chb t_filter + N_tau (t_tdh + t_zeta) + t_x + t_to * N_g / 4096).
    Inputs are the workload's system with a smooth stand-in orbital (timing does not depend
    on the orbital's values).
    """
    import numpy as np
    from oracle import chebyshev as cheb
    from oracle import hamiltonian as ham
    from oracle import sgw as osgw
    from paper_2601_21005_gb300 import synth
    sysd = build_system(cfg)
    g = ham.Grid(cfg['n'], cfg['h'])
    kb = ham.KB(sysd['kb_atoms']) if sysd['kb_atoms'] else None
    L = cfg['n'] * cfg['h']
    phi = synth.smooth_orbital(cfg['n'], cfg['h'], (L / 2, L / 2, L / 2))
    emin, emax = float(sysd['vloc'].min()) - 1.0, 0.5 * 3 * (np.pi / cfg['h']) ** 2 + 1.0
    prob = osgw.Problem(g, sysd['vloc'], kb, emin, emax, emin + 0.5, emin + 0.6, phi)
    ne, N = cfg['n_eta'], cfg['n_steps']
    t = {}
    noise = osgw.white_noise(g, seed, 1, 0, ne + 1)
    t0 = time.perf_counter()
    filt = osgw.filter_batch(prob, noise, np.ones(n_filter_terms + 1) / (n_filter_terms + 1))
    t['filter_term'] = (time.perf_counter() - t0) / n_filter_terms
    eta, zbar = filt[1:], noise[0]
    t0 = time.perf_counter()
    osgw.tdh_response_tangent(prob, eta, zbar * phi, n_tdh_steps, cfg['dt'], cfg['cheb_deg'])
    t['tdh_step'] = (time.perf_counter() - t0) / n_tdh_steps
    u = np.zeros((n_zeta_steps + 1,) + g.shape(), dtype=np.complex128)
    t0 = time.perf_counter()
    osgw.sigma_t(prob, filt[0], zbar - filt[0], u, n_zeta_steps, cfg['dt'], cfg['cheb_deg'])
    t['zeta_step'] = (time.perf_counter() - t0) / n_zeta_steps
    t0 = time.perf_counter()
    osgw.exchange(prob, eta)
    t['exchange'] = time.perf_counter() - t0
    sl = min(4096, g.ng)
    t0 = time.perf_counter()
    osgw.time_order(np.zeros((N + 1, sl)))
    t['time_order'] = (time.perf_counter() - t0) * g.ng / sl
    per_sample = (cfg['n_cheb'] * t['filter_term'] + N * (t['tdh_step'] + t['zeta_step']) + t['exchange']
                  + t['time_order'])
    batch_s = step_samples(cfg) * per_sample
    measured = n_filter_terms * t['filter_term'] + n_tdh_steps * t['tdh_step'] + n_zeta_steps * t['zeta_step'] \
        + t['exchange'] + t['time_order'] * sl / g.ng
    return dict(value=units_per_step(cfg) / batch_s, batch_seconds=batch_s, measured_seconds=measured, parts=t)


def run_reference(args, cfg):
    """--impl reference: the FP64 oracle on the host cores (rank 0 only), K timed bounded samples."""
    rank = int(os.environ.get('RANK', '0'))
    if rank != 0:
        return
    for _ in range(args.warmup):
        oracle_sample(cfg)
    vals, meas = [], []
    for _ in range(args.steps):
        r = oracle_sample(cfg)
        vals.append(r['value'])
        meas.append(r['measured_seconds'])
    v = statistics.median(vals)
    sample = ('per step: 1 MC sample of %s -- %d filter terms on %d vectors, 1 TDH step of %d pairs, '
              '1 zeta step, exchange, time ordering of a 4096-point slice; extrapolated to the batch of %d '
              'samples x (N_chb=%d, N_tau=%d)' % (cfg['workload'], 2, cfg['n_eta'] + 1, cfg['n_eta'],
                                                  step_samples(cfg), cfg['n_cheb'], cfg['n_steps']))
    line = dict(impl='reference', metric=METRIC, value=v, unit=UNIT, n_gpus=args.gpus, steps=args.steps,
                warmup=args.warmup, ms_per_step=1e3 * statistics.median(meas), higher_is_better=True,
                scaling='weak', vs_baseline=None, dtype='f64', data='synthetic',
                config=dict(workload=cfg['workload'], l2='inputs larger than L2'),
                cpu_baseline=dict(value=v, unit=UNIT, cores=1, kind='oracle', sample=sample,
                                  batch_seconds_extrapolated=r['batch_seconds'], parts_s=r['parts']),
                e2e=dict(value=v, unit=UNIT, h2d_bytes_per_step=0, d2h_bytes_per_step=0))
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- our arm
def cpu_baseline_subprocess(args):
    """Run the reference arm once (one bounded sample) in a fresh process with one BLAS thread."""
    env = dict(os.environ, OMP_NUM_THREADS='1', OPENBLAS_NUM_THREADS='1', MKL_NUM_THREADS='1')
    for k in ('RANK', 'WORLD_SIZE', 'LOCAL_RANK'):
        env.pop(k, None)
    cmd = [sys.executable, os.path.join(ROOT, 'bench.py'), '--impl', 'reference', '--steps', '1', '--warmup', '0',
           '--config', args.config]
    r = subprocess.run(cmd, capture_output=True, text=True, env=env, timeout=900)
    for line in r.stdout.splitlines()[::-1]:
        if line.startswith('{'):
            return json.loads(line)['cpu_baseline']
    return dict(value=None, unit=UNIT, cores=1, kind='oracle', sample='failed: ' + r.stderr[-300:])


def run_ours(args, cfg):
    import numpy as np
    import torch
    world = int(os.environ.get('WORLD_SIZE', '1'))
    rank = int(os.environ.get('RANK', '0'))
    local = int(os.environ.get('LOCAL_RANK', '0'))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group('nccl', device_id=torch.device('cuda', local))
    from paper_2601_21005_gb300 import build, replicas
    build.build()
    peaks = load_peaks()
    seed = 1000 * 2
    sysd = build_system(cfg)
    t_setup = time.perf_counter()
    if args.ks_cache and os.path.exists(args.ks_cache):
        z = np.load(args.ks_cache)
        ks = {k: (z[k].item() if z[k].ndim == 0 else z[k]) for k in z.files}
    else:
        ks = kohn_sham_inputs(cfg, sysd, local)
        if args.ks_cache:
            np.savez(args.ks_cache, **{k: np.asarray(v) for k, v in ks.items()})
    pl = make_pipeline(cfg, sysd, ks, local, seed, graphs=args.graphs, autotune=args.autotune)
    t_setup = time.perf_counter() - t_setup
    ns = step_samples(cfg)
    nb_total = args.warmup + args.steps
    sig = torch.empty(nb_total * ns, 2 * cfg['n_steps'] + 1, dtype=torch.complex128, device='cuda')
    xs = torch.empty(nb_total * ns, dtype=torch.float64, device='cuda')
    base = replicas.sample_base(rank)   # each rank draws its own samples: no data-path collective
    eps_ks = ks['e_homo']

    def step(b):
        s0 = b * ns
        pl.run_batch(base + s0, sig[s0:s0 + ns], xs[s0:s0 + ns])
        pl.qp(sig[:s0 + ns], xs[:s0 + ns], eps_ks) if s0 + ns >= 2 else None

    for b in range(args.warmup):
        step(b)
    torch.cuda.synchronize()
    st = torch.cuda.current_stream()
    clocks = ClockSampler(local)
    if not args.graphs:                # per-launch events would disable the graph replay
        pl.ctx.profile(True)
    n0 = pl.ctx.launch_count()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.nvtx.range_push('sgw_timed')
    e0.record(st)
    for b in range(args.warmup, nb_total):
        step(b)
    e1.record(st)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    launches = pl.ctx.launch_count() - n0
    if args.graphs:
        # kernel durations from one more step with per-launch events (direct launches)
        pl.ctx.profile(True)
        step(0)
        prof = pl.ctx.profile_read()
        pl.ctx.profile(False)
    else:
        prof = pl.ctx.profile_read()
        pl.ctx.profile(False)
    ms = replicas.max_over_ranks(ms, dist, 'cuda')
    ms_per_step = ms / args.steps
    value = replicas.job_throughput(units_per_step(cfg), args.steps, world, ms)
    # one QP solve over every rank's samples (gathered after the timed region)
    sig_all, xs_all = replicas.gather_rows(sig, xs, dist)
    tt = time_to_target(pl, sig_all, xs_all, eps_ks, ms_per_step * 1e-3 / (ns * world))

    # end to end through the public API: per step the target orbital comes from pinned host
    # memory and Sigma(t), X and the QP result go back to the host
    phi_h = torch.from_numpy(np.asarray(ks['phi'], dtype=np.float32).reshape(-1)).pin_memory()
    sig_h = torch.empty(ns, 2 * cfg['n_steps'] + 1, dtype=torch.complex128).pin_memory()
    x_h = torch.empty(ns, dtype=torch.float64).pin_memory()
    sig_e = torch.empty(ns, 2 * cfg['n_steps'] + 1, dtype=torch.complex128, device='cuda')
    x_e = torch.empty(ns, dtype=torch.float64, device='cuda')
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    e0.record(st)
    for b in range(args.steps):
        pl.phi.copy_(phi_h, non_blocking=True)
        pl.run_batch(base + 500000 + b * ns, sig_e, x_e)
        sig_h.copy_(sig_e, non_blocking=True)
        x_h.copy_(x_e, non_blocking=True)
        pl.qp(sig_e, x_e, eps_ks)           # returns host scalars (synchronises)
    e1.record(st)
    torch.cuda.synchronize()
    ms_e2e = e0.elapsed_time(e1)
    ms_e2e = replicas.max_over_ranks(ms_e2e, dist, 'cuda')
    e2e = dict(value=replicas.job_throughput(units_per_step(cfg), args.steps, world, ms_e2e), unit=UNIT,
               h2d_bytes_per_step=phi_h.numel() * 4, d2h_bytes_per_step=sig_h.numel() * 16 + x_h.numel() * 8 + 32)
    # plain FP32 form (Sigma reductions, transform and QP in FP32) on the same samples as the
    # mixed form (FP64 there): the eV difference of the QP energy
    prec = precision_comparison(cfg, pl, ks, base)
    cvres = cv_study(args, cfg, pl, ks, base) if args.cv > 0 else None
    # the metric's comparison: time to +-0.03 eV of the chosen form (mixed precision + control
    # variate) and of the plain FP32 form (no control variate, FP32 reductions at their own speed)
    chosen = None
    if cvres is not None:
        plain_s = cvres['time_to_0_03eV_plain_s'] * prec['ms_per_step_plain_fp32'] / prec['ms_per_step_mixed']
        chosen = dict(plain_fp32_seconds=round(plain_s, 1), chosen_seconds=cvres['time_to_0_03eV_cv_s'],
                      chosen_seconds_incl_training=cvres['time_to_0_03eV_cv_incl_training_s'],
                      speedup=round(plain_s / cvres['time_to_0_03eV_cv_s'], 3),
                      speedup_incl_training=round(plain_s / cvres['time_to_0_03eV_cv_incl_training_s'], 3))
    split = split_study(cfg, pl)
    xis = xi_study(args, cfg, sysd, ks, pl, base) if args.xi else None
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    rl = roofline(prof, peaks)
    cpu = cpu_baseline_subprocess(args) if world == 1 and not args.no_cpu_baseline else None
    line = dict(metric=METRIC, value=value, unit=UNIT, n_gpus=world, steps=args.steps, warmup=args.warmup,
                ms_per_step=ms_per_step, higher_is_better=True, scaling='weak', vs_baseline=None, dtype='c64/f32 + f64',
                data='synthetic',
                config=dict(workload=cfg['workload'], n_cheb=cfg['n_cheb'], cheb_deg=cfg['cheb_deg'], dt=cfg['dt'],
                            samples_per_step=ns * world, tdh_orbitals_per_launch=2 * cfg['n_eta'] * cfg['samples_per_batch'],
                            zeta_vectors_per_launch=2 * ns,
                            l2='inputs larger than L2 (about 20 GB live per step)',
                            precision='FP32 propagation, FP64 Sigma/transform/QP', parallelism='dp%d' % world,
                            cuda_graphs=bool(args.graphs),
                            launch_tuning=dict(zip(('plane_operand_prefetch', 'plane_lookahead', 'pencil_lookahead',
                                                    'plane_variant'),
                                                   pl.tuning)) if pl.tuning else 'defaults',
                            roofline_timing='per-kernel CUDA events over the timed region' if not args.graphs else
                            'per-kernel CUDA events over one extra step (graph replay is timed unprofiled)'),
                e2e=e2e, gpu_launches=int(launches), roofline=rl, cpu_baseline=cpu,
                clocks=clk, time_to_0_03eV=tt, time_to_0_03eV_chosen_vs_plain=chosen, precision_forms=prec,
                control_variate=cvres, split_operator=split, xi_compression=xis,
                setup=dict(seconds=round(t_setup, 2), e_homo=ks['e_homo'], e_lumo=ks['e_lumo'],
                           gap_eV=round((ks['e_lumo'] - ks['e_homo']) * HA_EV, 4), emin=ks['emin'], emax=ks['emax'],
                           eig_residual=float(ks['eig_residual'])))
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def precision_comparison(cfg, pl, ks, base):
    """The same step of samples in the mixed form (FP64 Sigma reductions, transform and QP) and in
    the plain FP32 form, each timed with CUDA events after a warm-up run: QP difference and times."""
    import torch
    m = pl.run_samples
    out = {}
    st = torch.cuda.current_stream()
    for name, f in (('mixed_fp64', 1), ('plain_fp32', 0)):
        pl.fp64 = f
        sg = torch.empty(m, 2 * cfg['n_steps'] + 1, dtype=torch.complex128, device='cuda')
        x = torch.empty(m, dtype=torch.float64, device='cuda')
        pl.run_batch(base + 900000, sg, x)                   # warm-up (captures this form's graphs)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        pl.run_batch(base + 900000, sg, x)
        e1.record(st)
        e1.synchronize()
        out[name] = (pl.qp(sg, x, ks['e_homo'])['eps_qp'], e0.elapsed_time(e1))
    pl.fp64 = 1
    return dict(qp_eV_mixed=round(out['mixed_fp64'][0] * HA_EV, 6), qp_eV_plain_fp32=round(out['plain_fp32'][0] * HA_EV, 6),
                diff_eV=abs(out['plain_fp32'][0] - out['mixed_fp64'][0]) * HA_EV, samples=m,
                ms_per_step_mixed=round(out['mixed_fp64'][1], 1), ms_per_step_plain_fp32=round(out['plain_fp32'][1], 1))


def split_pipeline(cfg, pl, runs=1):
    """Whole bench steps with the split-operator TDH and zeta steps (the paper's stepper) on the same
    pipeline, timed with CUDA events; the QP energy of the same samples by both steppers."""
    import torch
    ns = pl.run_samples
    n = runs * ns
    res = {}
    for prop, deg in (('split', 0), ('chebyshev', cfg['cheb_deg'])):
        pl.cheb_deg = deg
        sig = torch.empty(n, 2 * cfg['n_steps'] + 1, dtype=torch.complex128, device=pl.dev)
        xs = torch.empty(n, dtype=torch.float64, device=pl.dev)
        pl.run_batch(800000, sig[:ns], xs[:ns])                       # warm-up (graph capture)
        st = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for r in range(runs):
            pl.run_batch(800000 + r * ns, sig[r * ns:(r + 1) * ns], xs[r * ns:(r + 1) * ns])
        e1.record(st)
        e1.synchronize()
        ms = e0.elapsed_time(e1) / runs
        q = pl.qp(sig, xs, pl.e_homo)
        res[prop] = dict(ms_per_step=ms, value=units_per_step(cfg) / (ms * 1e-3), qp_eV=q['eps_qp'] * HA_EV)
    pl.cheb_deg = cfg['cheb_deg']
    return dict(value=res['split']['value'], ms_per_step=res['split']['ms_per_step'], samples=n,
                qp_eV_split=round(res['split']['qp_eV'], 5), qp_eV_chebyshev=round(res['chebyshev']['qp_eV'], 5),
                chebyshev_value_same_run=res['chebyshev']['value'])


def split_study(cfg, pl, seed=77):
    """Plain propagation (no TDH feedback) of one TDH-sized batch by the split-operator scheme and
    by the degree-K Chebyshev step, on the pipeline's context (graph replay), timed with CUDA events."""
    import torch
    B = 2 * cfg['n_eta'] * cfg['samples_per_batch']
    ng = cfg['n'] ** 3
    out = {}
    with pl.on_stream():
        psi = torch.empty(B, ng, dtype=torch.complex64, device=pl.dev)
        pl.ctx.white_noise(seed, 7, 0, 1, B, psi)
        st = torch.cuda.current_stream()
        for name, steps, fn in (('split', 100, lambda k: pl.ctx.propagate_split(psi, k, cfg['dt'])),
                                ('chebyshev', 10, lambda k: pl.ctx.propagate(psi, k, cfg['dt'], cfg['cheb_deg']))):
            fn(steps)                                    # capture + warm-up
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            for _ in range(3):
                fn(steps)
            e1.record(st)
            e1.synchronize()
            out[name] = ng * B * steps * 3 / (e0.elapsed_time(e1) * 1e-3)
        # accuracy on this system: the same vectors after 20 steps of each (Chebyshev-16 is exact to
        # rounding at this dt, so the difference is the splitting error)
        a = torch.empty(8, ng, dtype=torch.complex64, device=pl.dev)
        pl.ctx.white_noise(seed + 1, 7, 0, 1, 8, a)
        b = a.clone()
        pl.ctx.propagate_split(a, 20, cfg['dt'])
        pl.ctx.propagate(b, 20, cfg['dt'], cfg['cheb_deg'])
        err = float(torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b))
    return dict(unit=UNIT, vectors=B, split_value=out['split'], chebyshev_value=out['chebyshev'],
                ratio=out['split'] / out['chebyshev'], rel_diff_after_20_steps=err,
                pipeline=split_pipeline(cfg, pl),
                note='propagation only (no TDH feedback); the split-operator step carries an O(dt^3) '
                     'splitting error, the degree-16 Chebyshev step is exact to rounding at this dt')


def xi_study(args, cfg, sysd, ks, pl, base, n_xi=10000, f_g=0.003, L=32):
    """The same samples through the full-grid pipeline and through one that carries u^R in the sparse
    stochastic xi basis (n_xi functions of grid fraction f_g in segments of L points, the sizes of the
    paper's runs), each timed with CUDA events after a warm-up run: time per step, bytes of the stored
    u, and the spread the xi projection adds to the per-sample Re Sigma_i(eps_KS) against the Monte-Carlo
    spread of the full-grid values."""
    import numpy as np
    import torch
    from paper_2601_21005_gb300.pipeline import Pipeline
    pxi = Pipeline(cfg['n'], cfg['h'], sysd['vloc'], sysd['kb_atoms'], ks['phi'], ks['e_homo'], ks['e_lumo'],
                   n_eta=cfg['n_eta'], n_steps=cfg['n_steps'], dt=cfg['dt'], cheb_deg=cfg['cheb_deg'],
                   n_cheb=cfg['n_cheb'], samples_per_batch=cfg['samples_per_batch'], seed=pl.seed, stream_id=1,
                   device=pl.dev.index, spectrum=(ks['emin'], ks['emax']), graphs=args.graphs,
                   zeta_group=cfg['zeta_group'], xi=dict(n_xi=n_xi, f_g=f_g, L=L))
    if pl.tuning:
        for key, v in enumerate(pl.tuning):
            pxi.ctx.set_tuning(key, v)
    m = pl.run_samples
    N = cfg['n_steps']
    res = {}
    for name, p in (('full_grid', pl), ('xi', pxi)):
        sg = torch.empty(m, 2 * N + 1, dtype=torch.complex128, device='cuda')
        x = torch.empty(m, dtype=torch.float64, device='cuda')
        p.run_batch(base + 700000, sg, x)                  # warm-up (graph capture)
        st = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        p.run_batch(base + 700000, sg, x)
        e1.record(st)
        e1.synchronize()
        # per-sample Re Sigma_i(eps_KS) on the pipeline's stream (the context launches there)
        with p.on_stream():
            om = torch.tensor([ks['e_homo']], dtype=torch.float64, device='cuda')
            per = torch.empty(m, dtype=torch.complex128, device='cuda')
            for i in range(m):
                p.ctx.sigma_omega(sg[i:i + 1], 1, N, cfg['dt'], p.gamma, om, per[i:i + 1])
        torch.cuda.synchronize()
        res[name] = dict(ms=e0.elapsed_time(e1), per=per.real.cpu().numpy(), qp=p.qp(sg, x, ks['e_homo'])['eps_qp'],
                         u_bytes=p.u.numel() * p.u.element_size() + p.uR.numel() * p.uR.element_size())
    pxi.ctx.close()
    d = res['xi']['per'] - res['full_grid']['per']
    sd_full = float(res['full_grid']['per'].std(ddof=1))
    return dict(n_xi=n_xi, f_g=f_g, L=L, samples=m,
                ms_per_step_full_grid=round(res['full_grid']['ms'], 1), ms_per_step_xi=round(res['xi']['ms'], 1),
                u_bytes_full_grid=int(res['full_grid']['u_bytes']), u_bytes_xi=int(res['xi']['u_bytes']),
                qp_eV_full_grid=round(res['full_grid']['qp'] * HA_EV, 5), qp_eV_xi=round(res['xi']['qp'] * HA_EV, 5),
                re_sigma_sd_eV_full_grid=round(sd_full * HA_EV, 5),
                re_sigma_sd_eV_xi_minus_full=round(float(d.std(ddof=1)) * HA_EV, 5),
                added_variance_ratio=round(float(d.var(ddof=1)) / max(sd_full ** 2, 1e-300), 4),
                note='per-sample Re Sigma_i(eps_KS); the xi form is unbiased over the xi draws, so its added '
                     'variance adds to the Monte-Carlo variance of the same samples')


def cv_study(args, cfg, pl, ks, base):
    """Train the control variate on args.cv plain samples, then time steps of the chosen form
    (one batch of paired samples plus cheap samples per step) against the plain estimator on the
    same paired samples."""
    import torch
    from paper_2601_21005_gb300.control_variate import ControlVariate
    ns = pl.run_samples
    cv = ControlVariate(pl, m2max=10, width=256, max_batch=256, seed=11)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    Yt, Ft = cv.collect(args.cv, base + 300000)
    tr, va = cv.train(Ft, Yt, epochs=200, batch=64, lr=1e-3)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    n_cheap = args.cv_cheap
    st = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    Ys, Fs = [], []
    e0.record(st)
    for b in range(args.cv_paired_batches):
        Y, F = cv.collect(ns, base + 400000 + b * ns)
        Ys.append(Y)
        Fs.append(F)
    Fc = cv.cheap_features(n_cheap, base + 500000)
    Yp, Fp = torch.cat(Ys), torch.cat(Fs)
    S1, X1 = cv.rows(Fc, Fp, Yp)
    r_cv = pl.qp(S1, X1, ks['e_homo'])
    e1.record(st)
    torch.cuda.synchronize()
    sec = e0.elapsed_time(e1) * 1e-3
    S0, X0 = cv.plain_rows(Yp)
    r_pl = pl.qp(S0, X0, ks['e_homo'])
    net_kept = cv.use_net
    cv.use_net = False                    # the linear part alone, on the same rows
    S2, X2 = cv.rows(Fc, Fp, Yp)
    cv.use_net = net_kept
    r_lin = pl.qp(S2, X2, ks['e_homo'])
    n = Yp.shape[0]
    per_sample_s = sec / n                 # paired samples plus their share of the cheap ones
    sd_pl, sd_cv = r_pl['se'] * HA_EV * n ** 0.5, r_cv['se'] * HA_EV * n ** 0.5
    need_pl, need_cv = (sd_pl / 0.03) ** 2, (sd_cv / 0.03) ** 2
    t_plain = need_pl * per_sample_s
    t_cv = need_cv * per_sample_s
    return dict(n_train=args.cv, n_paired=n, n_cheap=n_cheap, train_seconds=round(t_train, 2),
                heldout_loss_first_best=[round(va[0], 4), round(min(va), 4)] if va else None,
                qp_eV_plain=round(r_pl['eps_qp'] * HA_EV, 5), se_eV_plain=round(r_pl['se'] * HA_EV, 5),
                qp_eV_cv=round(r_cv['eps_qp'] * HA_EV, 5), se_eV_cv=round(r_cv['se'] * HA_EV, 5),
                variance_gain=round((r_pl['se'] / r_cv['se']) ** 2, 3),
                variance_gain_linear_part_alone=round((r_pl['se'] / r_lin['se']) ** 2, 3), network_kept=bool(net_kept),
                time_to_0_03eV_plain_s=round(t_plain, 1), time_to_0_03eV_cv_s=round(t_cv, 1),
                time_to_0_03eV_cv_incl_training_s=round(t_cv + t_train, 1),
                speedup=round(t_plain / t_cv, 3), speedup_incl_training=round(t_plain / (t_cv + t_train), 3))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument('--gpus', type=int, default=1)
    ap.add_argument('--steps', type=int, default=5)
    ap.add_argument('--warmup', type=int, default=3)
    ap.add_argument('--impl', default='ours', choices=['ours', 'reference'])
    ap.add_argument('--config', default='si35h36_64', choices=sorted(CONFIGS))
    ap.add_argument('--no-cpu-baseline', action='store_true')
    ap.add_argument('--ks-cache', default=None,
                    help='npz file for the Kohn-Sham inputs (read if present, else computed and written)')
    ap.add_argument('--no-graphs', dest='graphs', action='store_false',
                    help='launch every kernel directly instead of replaying the loops as CUDA graphs')
    ap.add_argument('--no-autotune', dest='autotune', action='store_false',
                    help='keep the default launch hints instead of timing the candidates at setup')
    ap.add_argument('--no-xi', dest='xi', action='store_false', help='skip the xi-compression study')
    ap.add_argument('--cv', type=int, default=128, help='control-variate training samples (0: skip the study)')
    ap.add_argument('--cv-cheap', type=int, default=4096, help='cheap (features-only) samples in the study')
    ap.add_argument('--cv-paired-batches', type=int, default=8,
                    help='runs of paired samples in the study (8 runs of 16: 128 paired corrections)')
    ap.add_argument('--scale', type=float, default=1.0,
                    help='scale N_tau and N_chb together (profiling captures of fewer launches)')
    args = ap.parse_args()
    cfg = dict(CONFIGS[args.config])
    if args.scale != 1.0:
        cfg['n_steps'] = max(2, int(round(cfg['n_steps'] * args.scale)))
        cfg['n_cheb'] = max(2, int(round(cfg['n_cheb'] * args.scale)))
        cfg['workload'] += ' (scaled: N_tau=%d, N_chb=%d)' % (cfg['n_steps'], cfg['n_cheb'])
    if args.impl == 'reference':
        run_reference(args, cfg)
    else:
        run_ours(args, cfg)


if __name__ == '__main__':
    main()
