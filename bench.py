#!/usr/bin/env python
"""Benchmark of the stochastic-GW hot path on one node (one process per GPU).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--config NAME]

Headline workload (default): the large synthetic cluster Si7055H1596 on a 288^3 grid (h = 0.5
bohr, 29,816 electrons, s/p KB projectors on every Si), one batch of 4 Monte-Carlo samples =
64 TDH orbitals (8 eta pairs each) and 8 zeta vectors, u^R carried in the sparse stochastic xi
basis of the paper's runs (N_xi = 10^4, f_g = 0.003, segments of 32; Sec. 2.3, Table 2).  The
batch's white noise and occupied filter (Eq. 3) run once before the timed region (timed
separately: the `filter` object); one bench step is `step_time_steps` time steps of everything
after the filter for that batch: exchange, the linear-response TDH propagation of the 64
orbitals (Chebyshev degree 16, dt = 0.05) with the xi projection of u^R, time ordering, the zeta
propagation with the FP64 Sigma(t) accumulation (Eq. 4-5) and the QP solve (Eq. 6-7).  The
metric counts grid points x TDH orbitals x time steps per second of the whole step.

Secondary workload (object `c2_64`): the 64^3 Si35H36 cluster through the whole path per step
(16 samples: noise, degree-2000 filter, TDH and zeta over 400 steps, QP), with the time to
+-0.03 eV of the plain FP32 form and of the chosen form (mixed precision + control variate).

With --impl reference the FP64 CPU oracle is timed on a bounded sample of the headline workload
on every host core instead (`oracle_sample`).
"""
import argparse
import hashlib
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
    # the large cluster: the largest configuration that fits one GPU
    'si7055h1596_288': dict(
        system='si_cluster', n=288, h=0.5, radius=61.0, samples_per_batch=4, zeta_group=1, n_eta=8,
        step_time_steps=4, n_tau=1000, dt=0.05, cheb_deg=16, n_cheb=7000, xi=dict(n_xi=10000, f_g=0.003, L=32),
        # occupied-filter window: the gap of this cluster in its kernel-polynomial density of states
        # at degree 8000 (below 20 states/Ha from -0.105 to -0.075 Ha, centre -0.0895 Ha, count
        # 14910.0 +- 42 at n_occ = 14908), and a filter degree for a gap of ~0.03 Ha; the target
        # orbital is a stand-in (a normalised Gaussian at the cluster centre): the cost of a step
        # does not depend on it
        e_homo=-0.1045, e_lumo=-0.0745,
        workload='Si7055H1596 cluster, 288^3 grid h=0.5 bohr, 29816 electrons, KB on 7055 Si; one batch of '
                 '4 MC samples = 64 TDH orbitals (8 eta pairs each) + 8 zeta vectors, xi-compressed u '
                 '(N_xi=10000, f_g=0.003, L=32), Chebyshev degree 16, dt=0.05; per step 4 TDH + 4 zeta time '
                 'steps with Sigma(t) and the QP solve after the batch\'s occupied filter (degree 7000, at setup)'),
    # the small cluster, whole path per step
    'si35h36_64': dict(system='si_cluster', n=64, h=0.5, radius=10.5, samples_per_batch=4, zeta_group=4, n_eta=8,
                       n_steps=400, dt=0.05, cheb_deg=16, n_cheb=2000, workload='Si35H36 cluster, 64^3 grid '
                       'h=0.5 bohr, 176 electrons, 64 orbitals per TDH launch (4 MC samples x 8 eta pairs) x '
                       '400 steps; 16 MC samples per step, their 32 zeta vectors propagated together'),
    # the tiny periodic case (parity-test size)
    'wells16': dict(system='wells', n=16, h=0.6, samples_per_batch=1, zeta_group=1, n_eta=8, n_steps=200, dt=0.05,
                    cheb_deg=16, n_cheb=128, workload='6 Gaussian wells, 16^3 grid h=0.6 bohr, 8 electrons, '
                    '16 orbitals x 200 steps'),
}

# ncu DRAM bytes (read + write) over the algorithmic bytes of one launch of a kernel kind, from one
# capture of the kernel source whose sha256 prefix is given; a roofline line reports `traffic`
# only while that source is unchanged.
TRAFFIC = {
    ('plane_step', 64): dict(ratio=839.2 / 806.4, source='kernels_grid.cu', sha='', capture='64-vector launch'),
    # k_rows36_step, third term of a 4-vector kernel_bench step: 5.815 GB read + written against
    # 4.998 GB algorithmic
    # k_rows36_step under operand setting 3 (L2 prefetch + streaming caching) and a line form that keeps
    # warp-FFT rows; third term of a 4-vector kernel_bench step: 3.693 GB read + 1.487 GB written
    # against 4.998 GB algorithmic
    ('plane_step', 288): dict(ratio=(3.693 + 1.487) / 4.998, sha='08708691caeb2555', capture='4-vector launch',
                              operands=(3,), line_forms=(0, 1, 2, 3),
                              source=('kernels_cluster.cu', 'kb_unit.cuh', 'warp_fft.cuh', 'grid_common.cuh')),
}


def load_peaks():
    p = os.path.join(ROOT, 'MEASURED_PEAKS.json')
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return dict(hbm_gbs=float(d['hbm_gbs']), bf16_tflops=float(d['bf16_tflops']), source='measured')
    return dict(hbm_gbs=6800.0, bf16_tflops=1900.0, source='fallback')


def source_sha(names):
    """sha256 prefix of the concatenated kernel sources (a file name or a tuple of them)."""
    h = hashlib.sha256()
    for name in ((names,) if isinstance(names, str) else names):
        with open(os.path.join(ROOT, 'paper_2601_21005_gb300', 'csrc', name), 'rb') as f:
            h.update(f.read())
    return h.hexdigest()[:16]


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


def make_pipeline(cfg, sysd, ks, device, seed, fp64=True, graphs=False, autotune=False, zeta_group=None,
                  n_steps=None, xi=None):
    from paper_2601_21005_gb300.pipeline import Pipeline
    return Pipeline(cfg['n'], cfg['h'], sysd['vloc'], sysd['kb_atoms'], ks['phi'], ks['e_homo'], ks['e_lumo'],
                    n_eta=cfg['n_eta'], n_steps=cfg['n_steps'] if n_steps is None else n_steps, dt=cfg['dt'],
                    cheb_deg=cfg['cheb_deg'], n_cheb=cfg['n_cheb'], samples_per_batch=cfg['samples_per_batch'],
                    seed=seed, stream_id=1, device=device, spectrum=(ks['emin'], ks['emax']), fp64=fp64,
                    graphs=graphs, autotune=autotune,
                    zeta_group=cfg['zeta_group'] if zeta_group is None else zeta_group, xi=xi)


def step_samples(cfg):
    """MC samples of one bench step (one pipeline run)."""
    return cfg['samples_per_batch'] * cfg['zeta_group']


def units_per_step(cfg):
    """grid points x TDH-propagated orbitals x time steps of one bench step."""
    steps = cfg['step_time_steps'] if 'step_time_steps' in cfg else cfg['n_steps']
    return cfg['n'] ** 3 * 2 * cfg['n_eta'] * step_samples(cfg) * steps


def roofline(prof, peaks, n, tuning=None):
    """Dominant kernel kind by device time; achieved = its algorithmic bytes / its event time."""
    kinds = {k: v for k, v in prof.items() if v['launches'] > 0 and v['alg_bytes'] > 0}
    total = sum(v['ms'] for v in prof.values())
    name = max(kinds, key=lambda k: kinds[k]['ms'])
    v = kinds[name]
    gbs = v['alg_bytes'] / (v['ms'] * 1e-3) / 1e9
    peak = peaks['hbm_gbs']
    shares = {k: round(x['ms'] / total, 4) for k, x in prof.items() if x['launches']}
    tr = TRAFFIC.get((name, n))
    ops, form = (tuning[0], tuning[4]) if tuning else (1, 0)
    if tr is not None and (form not in tr.get('line_forms', (form,)) or ops not in tr.get('operands', (ops,))):
        tr = None                        # another kernel or cache policy does this kind's work here
    traffic, tsrc = None, 'no ncu capture of the current kernel source'
    if tr is not None and tr['sha'] and tr['sha'] == source_sha(tr['source']):
        traffic = round(tr['ratio'] * v['alg_bytes'] / v['launches'])
        tsrc = ('ncu dram__bytes_read.sum + dram__bytes_write.sum of a %s of this kernel source (%s %s), '
                'scaled by algorithmic bytes to the average launch' % (tr['capture'], '+'.join(
                    (tr['source'],) if isinstance(tr['source'], str) else tr['source']), tr['sha']))
    return dict(bound='hbm', achieved=round(gbs, 1), peak=peak, unit='GB/s', frac=round(gbs / peak, 4),
                traffic=traffic, traffic_source=tsrc, kernel=name, launches=v['launches'],
                avg_launch_us=round(1e3 * v['ms'] / v['launches'], 2), alg_bytes_per_launch=round(v['alg_bytes'] /
                                                                                                v['launches']),
                peak_source=peaks['source'] + ' hbm_gbs (burst copy; the kernel is timed inside a long step)',
                time_shares=shares,
                other_kernels_gbs={k: round(x['alg_bytes'] / (x['ms'] * 1e-3) / 1e9, 1) for k, x in kinds.items()})


def nvtx_range(torch, name):
    """Open (name) or close (None) an NVTX push/pop range around the timed steps, so that a
    profiler's launch list can be limited to them (`ncu --nvtx --nvtx-include timed_steps/`)."""
    try:
        if name is None:
            torch.cuda.nvtx.range_pop()
        else:
            torch.cuda.nvtx.range_push(name)
    except Exception:
        pass


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
_ORC = {}


def _oracle_term(i):
    """One Chebyshev term of the oracle's propagator (one H application and the recurrence update,
    FP64) on a vector of its own; returns the seconds it took."""
    import numpy as np
    from oracle import chebyshev as cheb
    p = _ORC['prob']
    v = np.random.default_rng(1000 + i).normal(size=p.grid.shape()) + 0j
    t0 = time.perf_counter()
    cheb.propagate_step(p.h0, v, p.emin, p.emax, 0.05, 1)
    return time.perf_counter() - t0


def oracle_pool(cfg, processes):
    """Fork a pool of oracle workers sharing the workload's H0 (only in a process that has not
    touched a GPU)."""
    import multiprocessing as mp
    import numpy as np
    from oracle import hamiltonian as ham
    from oracle import sgw as osgw
    sysd = build_system(cfg)
    g = ham.Grid(cfg['n'], cfg['h'])
    kb = ham.KB(sysd['kb_atoms']) if sysd['kb_atoms'] else None
    emin, emax = float(sysd['vloc'].min()) - 1.0, 0.5 * 3 * (np.pi / cfg['h']) ** 2 + 1.0
    _ORC['prob'] = osgw.Problem(g, sysd['vloc'], kb, emin, emax, emin + 0.5, emin + 0.6, np.zeros(g.shape()))
    return mp.get_context('fork').Pool(processes)


def oracle_sample(cfg, pool, processes):
    """Time `processes` oracle Chebyshev terms run at once, one per process, and extrapolate to one
    bench step: terms per step = time steps x 16 x (64 TDH orbitals + 8 zeta vectors); the
    per-step density, Poisson, xi and Sigma(t) work (under 2% of the terms' FFTs) is not counted,
    which favours the CPU."""
    per = pool.map(_oracle_term, range(processes), chunksize=1)
    wall = max(per)                 # the terms run at once: the slowest one ends the round
    n_vec = 2 * cfg['n_eta'] * step_samples(cfg) + 2 * step_samples(cfg)
    terms = cfg['step_time_steps'] * cfg['cheb_deg'] * n_vec
    step_s = terms * wall / processes
    return dict(value=units_per_step(cfg) / step_s, step_seconds=step_s, wall=wall,
                term_seconds_mean=statistics.mean(per), terms_per_step=terms)


def run_reference(args, cfg):
    """--impl reference: the FP64 oracle on every host core (rank 0 only), K timed bounded samples."""
    rank = int(os.environ.get('RANK', '0'))
    if rank != 0:
        return
    if 'step_time_steps' not in cfg:
        raise SystemExit('the reference arm times the headline workload only')
    P = os.cpu_count() or 1
    pool = oracle_pool(cfg, P)
    try:
        for _ in range(args.warmup):
            oracle_sample(cfg, pool, P)
        rs = [oracle_sample(cfg, pool, P) for _ in range(args.steps)]
    finally:
        pool.close()
        pool.join()
    v = statistics.median([r['value'] for r in rs])
    sample = ('per step: %d FP64 oracle Chebyshev terms (one H application with the recurrence update on one '
              '288^3 vector each) run at once on %d host processes, extrapolated to the step\'s %d terms (%d time '
              'steps x degree %d x %d vectors)' % (P, P, rs[0]['terms_per_step'], cfg['step_time_steps'],
                                                  cfg['cheb_deg'], rs[0]['terms_per_step'] //
                                                  (cfg['step_time_steps'] * cfg['cheb_deg'])))
    line = dict(impl='reference', metric=METRIC, value=v, unit=UNIT, n_gpus=args.gpus, steps=args.steps,
                warmup=args.warmup, ms_per_step=1e3 * statistics.median([r['wall'] for r in rs]),
                higher_is_better=True, scaling='weak', vs_baseline=None, dtype='f64', data='synthetic',
                config=dict(workload=cfg['workload'], l2='inputs larger than L2'),
                cpu_baseline=dict(value=v, unit=UNIT, cores=P, kind='oracle', sample=sample,
                                  step_seconds_extrapolated=statistics.median([r['step_seconds'] for r in rs]),
                                  term_seconds_mean=statistics.median([r['term_seconds_mean'] for r in rs])),
                e2e=dict(value=v, unit=UNIT, h2d_bytes_per_step=0, d2h_bytes_per_step=0))
    print(json.dumps(line), flush=True)


def cpu_baseline_subprocess(args):
    """Run the reference arm once (one bounded sample) in a fresh process that never touches a GPU."""
    env = dict(os.environ)
    for k in ('RANK', 'WORLD_SIZE', 'LOCAL_RANK'):
        env.pop(k, None)
    for k in ('OMP_NUM_THREADS', 'OPENBLAS_NUM_THREADS', 'MKL_NUM_THREADS'):
        env[k] = '1'                    # one thread per process: the processes are the parallelism
    cmd = [sys.executable, os.path.join(ROOT, 'bench.py'), '--impl', 'reference', '--steps', '1', '--warmup', '0',
           '--config', args.config]
    r = subprocess.run(cmd, capture_output=True, text=True, env=env, timeout=1200)
    for line in r.stdout.splitlines()[::-1]:
        if line.startswith('{'):
            return json.loads(line)['cpu_baseline']
    return dict(value=None, unit=UNIT, cores=os.cpu_count(), kind='oracle', sample='failed: ' + r.stderr[-300:])


# ---------------------------------------------------------------- our arm: the large cluster
def measure_large(args, cfg, local, world, rank, dist, peaks):
    import numpy as np
    import torch
    from paper_2601_21005_gb300 import replicas, synth
    t_setup = time.perf_counter()
    sysd = build_system(cfg)
    n, h = cfg['n'], cfg['h']
    c = 0.5 * n * h
    phi = synth.smooth_orbital(n, h, (c, c, c), width=3.0)
    phi /= np.sqrt(h ** 3 * np.sum(phi ** 2))
    from paper_2601_21005_gb300 import sgw
    S = cfg['step_time_steps']
    ks = dict(e_homo=cfg['e_homo'], e_lumo=cfg['e_lumo'], phi=phi, emin=None, emax=None)
    # spectral interval by the library's shifted power iteration on the same H0
    kctx = sgw.Context(n, h, max_batch=1, device=local)
    kctx.set_potential(torch.as_tensor(sysd['vloc'].reshape(-1).astype(np.float32)).cuda(local), sysd['kb_atoms'])
    (ks['emin'], ks['emax']), _ = kctx.spectral_bounds(200, 1000, 0.05)
    kctx.close()
    seed = 1000 * 5
    base = replicas.sample_base(rank)
    pl = make_pipeline(cfg, sysd, ks, local, seed, graphs=args.graphs, autotune=args.autotune, n_steps=S,
                       xi=cfg['xi'])
    del sysd
    ns = step_samples(cfg)
    st = torch.cuda.current_stream()
    # the batch's noise and occupied filter, timed on their own
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    pl.filter_batch(base)
    e1.record(st)
    torch.cuda.synchronize()
    filt_ms = e0.elapsed_time(e1)
    nv_filter = ns * (cfg['n_eta'] + 1)
    filt = dict(vectors=nv_filter, degree=cfg['n_cheb'], ms=round(filt_ms, 1),
                vector_terms_per_s=nv_filter * cfg['n_cheb'] / (filt_ms * 1e-3),
                grid_pt_vector_terms_per_s=n ** 3 * nv_filter * cfg['n_cheb'] / (filt_ms * 1e-3))
    t_setup = time.perf_counter() - t_setup
    sig = torch.empty(ns, 2 * S + 1, dtype=torch.complex128, device='cuda')
    xs = torch.empty(ns, dtype=torch.float64, device='cuda')

    def step():
        pl.propagate_batch(base, sig, xs)
        pl.qp(sig, xs, cfg['e_homo'])               # host scalars: synchronises

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    n0 = pl.ctx.launch_count()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    nvtx_range(torch, 'timed_steps')
    e0.record(st)
    for _ in range(args.steps):
        step()
    e1.record(st)
    nvtx_range(torch, None)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    launches = pl.ctx.launch_count() - n0
    # kernel durations: one more step with per-launch events (while profiling, the library launches
    # directly instead of replaying its graphs)
    pl.ctx.profile(True)
    step()
    prof = pl.ctx.profile_read()
    pl.ctx.profile(False)
    ms = replicas.max_over_ranks(ms, dist, 'cuda')
    value = replicas.job_throughput(units_per_step(cfg), args.steps, world, ms)
    # end to end through the public API: per step the batch's noise and filtered vectors and the
    # target orbital come from pinned host memory, Sigma(t), X and the QP result go back
    noise_h = pl.noise.cpu().pin_memory()
    filt_h = pl.filt.cpu().pin_memory()
    phi_h = pl.phi.cpu().pin_memory()
    sig_h = torch.empty(ns, 2 * S + 1, dtype=torch.complex128).pin_memory()
    x_h = torch.empty(ns, dtype=torch.float64).pin_memory()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    e0.record(st)
    for _ in range(args.steps):
        pl.noise.copy_(noise_h, non_blocking=True)
        pl.filt.copy_(filt_h, non_blocking=True)
        pl.phi.copy_(phi_h, non_blocking=True)
        pl.propagate_batch(base, sig, xs)
        sig_h.copy_(sig, non_blocking=True)
        x_h.copy_(xs, non_blocking=True)
        pl.qp(sig, xs, cfg['e_homo'])
    e1.record(st)
    torch.cuda.synchronize()
    ms_e2e = replicas.max_over_ranks(e0.elapsed_time(e1), dist, 'cuda')
    h2d = noise_h.numel() * 8 + filt_h.numel() * 8 + phi_h.numel() * 4
    e2e = dict(value=replicas.job_throughput(units_per_step(cfg), args.steps, world, ms_e2e), unit=UNIT,
               h2d_bytes_per_step=int(h2d), d2h_bytes_per_step=int(sig_h.numel() * 16 + x_h.numel() * 8 + 32))
    rl = roofline(prof, peaks, n, pl.tuning)
    peak_gb = round(torch.cuda.max_memory_allocated(local) / 1e9, 1)
    pl.ctx.close()
    tuning = dict(zip(('plane_operand_prefetch', 'plane_lookahead', 'pencil_lookahead', 'plane_variant',
                       'line_form'), pl.tuning)) if pl.tuning else 'defaults'
    return dict(value=value, ms=ms, ms_per_step=ms / args.steps, launches=launches, clocks=clk, e2e=e2e,
                roofline=rl, filter=filt, setup_seconds=round(t_setup, 1), peak_device_gb=peak_gb,
                spectrum=[pl.emin, pl.emax], tuning=tuning)


# ---------------------------------------------------------------- our arm: the 64^3 whole path
def measure_whole_path(args, cfg, local, world, rank, dist, peaks, steps, warmup):
    import numpy as np
    import torch
    from paper_2601_21005_gb300 import replicas
    sysd = build_system(cfg)
    t_setup = time.perf_counter()
    ks = kohn_sham_inputs(cfg, sysd, local)
    pl = make_pipeline(cfg, sysd, ks, local, 1000 * 2, graphs=args.graphs, autotune=args.autotune)
    t_setup = time.perf_counter() - t_setup
    ns = step_samples(cfg)
    nb_total = warmup + steps
    sig = torch.empty(nb_total * ns, 2 * cfg['n_steps'] + 1, dtype=torch.complex128, device='cuda')
    xs = torch.empty(nb_total * ns, dtype=torch.float64, device='cuda')
    base = replicas.sample_base(rank)
    eps_ks = ks['e_homo']

    def step(b):
        s0 = b * ns
        pl.run_batch(base + s0, sig[s0:s0 + ns], xs[s0:s0 + ns])
        pl.qp(sig[:s0 + ns], xs[:s0 + ns], eps_ks) if s0 + ns >= 2 else None

    for b in range(warmup):
        step(b)
    torch.cuda.synchronize()
    st = torch.cuda.current_stream()
    if dist:
        dist.barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for b in range(warmup, nb_total):
        step(b)
    e1.record(st)
    torch.cuda.synchronize()
    ms = replicas.max_over_ranks(e0.elapsed_time(e1), dist, 'cuda')
    pl.ctx.profile(True)
    step(0)
    prof = pl.ctx.profile_read()
    pl.ctx.profile(False)
    ms_per_step = ms / steps
    value = replicas.job_throughput(units_per_step(cfg), steps, world, ms)
    sig_all, xs_all = replicas.gather_rows(sig, xs, dist)
    tt = time_to_target(pl, sig_all, xs_all, eps_ks, ms_per_step * 1e-3 / (ns * world))
    prec = precision_comparison(cfg, pl, ks, base)
    cvres = cv_study(args, cfg, pl, ks, base, ms_per_step * 1e-3 / ns) if args.cv > 0 else None
    chosen = None
    if cvres is not None:
        # the chosen form (mixed precision + control variate) against the plain FP32 form (no control
        # variate, FP32 reductions at their own measured speed)
        plain_s = cvres['time_to_target_plain_s'] * prec['ms_per_step_plain_fp32'] / prec['ms_per_step_mixed']
        chosen = dict(workload=cfg['workload'], plain_fp32_seconds=round(plain_s, 1),
                      chosen_seconds=cvres['time_to_target_cv_s'],
                      chosen_seconds_incl_training=cvres['time_to_target_cv_incl_training_s'],
                      speedup=round(plain_s / cvres['time_to_target_cv_s'], 3),
                      speedup_incl_training=round(plain_s / cvres['time_to_target_cv_incl_training_s'], 3))
    out = dict(workload=cfg['workload'], value=value, unit=UNIT, ms_per_step=round(ms_per_step, 1), steps=steps,
               warmup=warmup, roofline=roofline(prof, peaks, cfg['n']), time_to_0_03eV=tt,
               time_to_0_03eV_chosen_vs_plain=chosen, precision_forms=prec, control_variate=cvres,
               setup=dict(seconds=round(t_setup, 2), e_homo=ks['e_homo'], e_lumo=ks['e_lumo'],
                          gap_eV=round((ks['e_lumo'] - ks['e_homo']) * HA_EV, 4), emin=ks['emin'], emax=ks['emax'],
                          eig_residual=float(ks['eig_residual'])))
    if args.split_study:
        out['split_operator'] = split_study(cfg, pl)
    if args.xi_study:
        out['xi_compression'] = xi_study(args, cfg, sysd, ks, pl, base)
    pl.ctx.close()
    return out


def run_ours(args, cfg):
    import torch
    world = int(os.environ.get('WORLD_SIZE', '1'))
    rank = int(os.environ.get('RANK', '0'))
    local = int(os.environ.get('LOCAL_RANK', '0'))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group('nccl', device_id=torch.device('cuda', local))
    from paper_2601_21005_gb300 import build
    build.build()
    peaks = load_peaks()
    if 'step_time_steps' in cfg:
        big = measure_large(args, cfg, local, world, rank, dist, peaks)
        torch.cuda.empty_cache()
        sec = None
        if not args.no_secondary:
            sec = measure_whole_path(args, CONFIGS['si35h36_64'], local, world, rank, dist, peaks,
                                     args.secondary_steps, 2)
        line = dict(metric=METRIC, value=big['value'], unit=UNIT, n_gpus=world, steps=args.steps,
                    warmup=args.warmup, ms_per_step=big['ms_per_step'], higher_is_better=True, scaling='weak',
                    vs_baseline=None, dtype='c64/f32 + f64', data='synthetic',
                    config=dict(workload=cfg['workload'], step_time_steps=cfg['step_time_steps'],
                                n_cheb=cfg['n_cheb'], cheb_deg=cfg['cheb_deg'], dt=cfg['dt'],
                                samples_per_step=step_samples(cfg) * world,
                                tdh_orbitals_per_launch=2 * cfg['n_eta'] * cfg['samples_per_batch'],
                                zeta_vectors_per_launch=2 * step_samples(cfg), xi=cfg['xi'],
                                l2='inputs larger than L2 (the 64 TDH orbitals alone are 12 GB)',
                                precision='FP32 propagation, FP64 Sigma/transform/QP', parallelism='dp%d' % world,
                                cuda_graphs=bool(args.graphs), launch_tuning=big['tuning'],
                                roofline_timing='per-kernel CUDA events over one extra step with direct launches '
                                                '(graph replay is timed unprofiled)'),
                    e2e=big['e2e'], gpu_launches=int(big['launches']), roofline=big['roofline'], cpu_baseline=None,
                    clocks=big['clocks'], filter=big['filter'],
                    setup=dict(seconds=big['setup_seconds'], spectrum=big['spectrum'],
                               peak_device_gb=big['peak_device_gb'],
                               ks='stand-in orbital and the filter window of the config (cost does not depend on '
                                  'them)'),
                    time_to_0_03eV_chosen_vs_plain=sec['time_to_0_03eV_chosen_vs_plain'] if sec else None,
                    c2_64=sec)
    else:
        sec = measure_whole_path(args, cfg, local, world, rank, dist, peaks, args.steps, args.warmup)
        line = dict(metric=METRIC, value=sec['value'], unit=UNIT, n_gpus=world, steps=args.steps,
                    warmup=args.warmup, ms_per_step=sec['ms_per_step'], higher_is_better=True, scaling='weak',
                    vs_baseline=None, dtype='c64/f32 + f64', data='synthetic',
                    config=dict(workload=cfg['workload'], parallelism='dp%d' % world), **{
                        k: sec[k] for k in ('roofline', 'time_to_0_03eV', 'time_to_0_03eV_chosen_vs_plain',
                                            'precision_forms', 'control_variate', 'setup')})
    if rank == 0:
        if world == 1 and not args.no_cpu_baseline and 'step_time_steps' in cfg:
            line['cpu_baseline'] = cpu_baseline_subprocess(args)
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
    stochastic xi basis, each timed with CUDA events after a warm-up run: time per step, bytes of the
    stored u, and the spread the xi projection adds to the per-sample Re Sigma_i(eps_KS)."""
    import torch
    from paper_2601_21005_gb300.pipeline import Pipeline
    pxi = Pipeline(cfg['n'], cfg['h'], sysd['vloc'], sysd['kb_atoms'], ks['phi'], ks['e_homo'], ks['e_lumo'],
                   n_eta=cfg['n_eta'], n_steps=cfg['n_steps'], dt=cfg['dt'], cheb_deg=cfg['cheb_deg'],
                   n_cheb=cfg['n_cheb'], samples_per_batch=cfg['samples_per_batch'], seed=pl.seed, stream_id=1,
                   device=pl.dev.index, spectrum=(ks['emin'], ks['emax']), graphs=args.graphs,
                   zeta_group=cfg['zeta_group'], xi=dict(n_xi=n_xi, f_g=f_g, L=L))
    m = pl.run_samples
    N = cfg['n_steps']
    res = {}
    for name, p in (('full_grid', pl), ('xi', pxi)):
        sg = torch.empty(m, 2 * N + 1, dtype=torch.complex128, device='cuda')
        x = torch.empty(m, dtype=torch.float64, device='cuda')
        p.run_batch(base + 700000, sg, x)
        st = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        p.run_batch(base + 700000, sg, x)
        e1.record(st)
        e1.synchronize()
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
                added_variance_ratio=round(float(d.var(ddof=1)) / max(sd_full ** 2, 1e-300), 4))


def cv_study(args, cfg, pl, ks, base, plain_sample_s):
    """The control variate against the plain estimator at equal target error (control_variate.study)."""
    from paper_2601_21005_gb300.control_variate import study
    return study(pl, ks['e_homo'], args.cv, args.cv_paired_batches, args.cv_cheap, base, plain_sample_s)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument('--gpus', type=int, default=1)
    ap.add_argument('--steps', type=int, default=5)
    ap.add_argument('--warmup', type=int, default=3)
    ap.add_argument('--impl', default='ours', choices=['ours', 'reference'])
    ap.add_argument('--config', default='si7055h1596_288', choices=sorted(CONFIGS))
    ap.add_argument('--no-cpu-baseline', action='store_true')
    ap.add_argument('--no-secondary', action='store_true', help='skip the 64^3 whole-path measurement')
    ap.add_argument('--secondary-steps', type=int, default=3, help='timed steps of the 64^3 whole-path measurement')
    ap.add_argument('--no-graphs', dest='graphs', action='store_false',
                    help='launch every kernel directly instead of replaying the loops as CUDA graphs')
    ap.add_argument('--no-autotune', dest='autotune', action='store_false',
                    help='keep the default launch hints instead of timing the candidates at setup')
    ap.add_argument('--split-study', action='store_true', help='64^3: time the split-operator stepper as well')
    ap.add_argument('--xi-study', action='store_true', help='64^3: time the xi-compressed pipeline as well')
    ap.add_argument('--cv', type=int, default=128, help='control-variate training samples (0: skip the study)')
    ap.add_argument('--cv-cheap', type=int, default=4096, help='cheap (features-only) samples in the study')
    ap.add_argument('--cv-paired-batches', type=int, default=8,
                    help='runs of paired samples in the study (8 runs of 16: 128 paired corrections)')
    ap.add_argument('--scale', type=float, default=1.0,
                    help='64^3 / 16^3 configs: scale N_tau and N_chb together (profiling captures)')
    ap.add_argument('--step-time-steps', type=int, default=None,
                    help='288^3: time steps per bench step (smaller: profiling captures)')
    ap.add_argument('--batch-samples', type=int, default=None,
                    help='288^3: MC samples per batch (smaller: profiling captures)')
    ap.add_argument('--n-cheb', type=int, default=None,
                    help='288^3: degree of the occupied filter at setup (smaller: profiling captures)')
    args = ap.parse_args()
    cfg = dict(CONFIGS[args.config])
    if args.scale != 1.0 and 'n_steps' in cfg:
        cfg['n_steps'] = max(2, int(round(cfg['n_steps'] * args.scale)))
        cfg['n_cheb'] = max(2, int(round(cfg['n_cheb'] * args.scale)))
        cfg['workload'] += ' (scaled: N_tau=%d, N_chb=%d)' % (cfg['n_steps'], cfg['n_cheb'])
    if args.step_time_steps is not None and 'step_time_steps' in cfg:
        cfg['step_time_steps'] = args.step_time_steps
        cfg['workload'] += ' (reduced: %d time steps per step)' % args.step_time_steps
    if args.n_cheb is not None and 'step_time_steps' in cfg:
        cfg['n_cheb'] = args.n_cheb
        cfg['workload'] += ' (reduced: filter degree %d)' % args.n_cheb
    if args.batch_samples is not None and 'step_time_steps' in cfg:
        cfg['samples_per_batch'] = args.batch_samples
        cfg['workload'] += ' (reduced: %d samples per batch)' % args.batch_samples
    if args.impl == 'reference':
        run_reference(args, cfg)
    else:
        run_ours(args, cfg)


if __name__ == '__main__':
    main()
