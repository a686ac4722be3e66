"""Stochastic-GW QP energy through the C ABI (the product path).

The steps of Sec. 2.1 (Fig. 1) for batches of Monte-Carlo samples, each one call into
libsgw; torch only allocates the device buffers and streams:

  white noise -> gapped filter (Eq. 3) -> split into eta / zeta pair / source ->
  exchange X (Eq. 6) -> linear-response TDH u^R(t) -> time ordering u(t) ->
  zeta propagation with Sigma(t) accumulation (Eq. 4, 5) -> ... over batches ... ->
  Sigma(omega) (Eq. 7) and the QP root (Eq. 6) on the sample means.

With xi=dict(n_xi=.., f_g=.., L=..) u^R(t) is carried as its overlaps U_m(t) = <xi_m|u^R(t)> with
n_xi sparse random functions on fragmented segments (Sec. 2.1, Sec. 2.3): u is stored as
[samples][N+1][n_xi] instead of [samples][N+1][N_g], the time ordering acts on U_m, and Sigma(t)
is accumulated in the xi basis.  The xi draws of sample i use the pipeline's seed, the counter
stream xi['stream'] (default stream_id + 2^16) and the global sample index i.
"""
import contextlib

import numpy as np

from . import sgw as _sgw


class Pipeline:
    def __init__(self, n, h, vloc, kb_atoms, phi, e_homo, e_lumo, n_eta=8, n_steps=200, dt=0.05,
                 cheb_deg=16, n_cheb=128, samples_per_batch=1, seed=1000, stream_id=1, device=0, ecut=0.0,
                 spectrum=None, coeffs=None, bounds_iter=100, margin=0.05, fp64=True, stream=None, graphs=False,
                 autotune=False, zeta_group=1, propagator='chebyshev', xi=None):
        import torch
        self.torch = torch
        # CUDA graphs need a non-default stream: the pipeline then owns one, and its buffers are
        # allocated and used on it
        self.stream = torch.cuda.Stream(device) if (graphs and stream is None) else None
        if self.stream is not None:
            stream = self.stream.cuda_stream
        self.n, self.h, self.ng = n, h, n ** 3
        if propagator not in ('chebyshev', 'split'):
            raise ValueError('propagator must be chebyshev or split')
        # the time steps of the TDH and zeta phases: degree-cheb_deg Chebyshev, or the split operator
        # (the library selects it with degree 0); the occupied filter is a Chebyshev series either way
        self.propagator = propagator
        self.n_eta, self.n_steps, self.dt = n_eta, n_steps, dt
        self.cheb_deg = 0 if propagator == 'split' else cheb_deg
        # a run is zeta_group chunks of samples_per_batch samples: white noise and the occupied filter
        # for all the run's samples at once ((N_eta + 1) samples_per_batch zeta_group vectors per
        # launch), exchange, TDH and time ordering chunk by chunk (2 N_eta samples_per_batch TDH
        # orbitals per launch), then the zeta pairs of all the run's samples in one propagation
        # (2 samples_per_batch zeta_group vectors per launch), with u of every sample of the run kept
        # in HBM
        self.ns = samples_per_batch
        self.group = int(zeta_group)
        if self.group < 1:
            raise ValueError('zeta_group must be >= 1')
        self.run_samples = self.ns * self.group
        self.seed, self.stream_id = seed, stream_id
        self.fp64 = 1 if fp64 else 0
        self.dev = torch.device('cuda', device)
        mb = max(self.run_samples * (n_eta + 1), 2 * self.ns * n_eta, 2 * self.run_samples)
        self.ctx = _sgw.Context(n, h, ecut=ecut, max_batch=mb, device=device, stream=stream)
        if graphs:
            self.ctx.set_graph_mode(True)
        vl = torch.as_tensor(np.asarray(vloc, dtype=np.float32).reshape(-1)).to(self.dev)
        self.ctx.set_potential(vl, kb_atoms)
        if spectrum is None:
            (self.emin, self.emax), self.raw_bounds = self.ctx.spectral_bounds(bounds_iter, seed, margin)
        else:
            self.emin, self.emax = spectrum
            self.ctx.set_spectrum(self.emin, self.emax)
        self.e_homo, self.e_lumo = e_homo, e_lumo
        # launch hints timed on this GPU with the TDH batch size (results do not depend on them)
        self.tuning = self.ctx.autotune(min(mb, 2 * self.ns * n_eta)) if autotune else None
        if coeffs is None:
            coeffs = _sgw.sgw_gapped_filter_coeffs(e_homo, e_lumo, self.emin, self.emax, n_cheb)
        self.coeffs = np.asarray(coeffs, dtype=np.float64)
        self.phi = torch.as_tensor(np.asarray(phi, dtype=np.float32).reshape(-1)).to(self.dev)
        ng, ns, N = self.ng, self.ns, n_steps
        c64, f32 = torch.complex64, torch.float32
        self.noise = torch.empty(self.run_samples * (n_eta + 1), ng, dtype=c64, device=self.dev)
        self.filt = torch.empty_like(self.noise)
        self.eta = torch.empty(ns * n_eta, ng, dtype=c64, device=self.dev)
        self.zeta = torch.empty(2 * self.run_samples, ng, dtype=c64, device=self.dev)
        self.source = torch.empty(ns, ng, dtype=f32, device=self.dev)
        if xi is not None:
            self.xi = dict(n_xi=int(xi['n_xi']), f_g=float(xi['f_g']), L=int(xi.get('L', 32)),
                           stream=int(xi.get('stream', stream_id + (1 << 16))))
            npts = self.xi['n_xi']
        else:
            self.xi = None
            npts = ng
        self.uR = torch.empty(ns, N + 1, npts, dtype=f32, device=self.dev)
        self.u = torch.empty(self.run_samples, N + 1, npts, dtype=c64, device=self.dev)

    def _xi_args(self, sample0):
        x = self.xi
        return (self.seed, x['stream'], sample0, x['n_xi'], x['f_g'], x['L'])

    @contextlib.contextmanager
    def on_stream(self):
        """Run the enclosed torch and libsgw work on the pipeline's stream, ordered after the
        caller's pending work and before the caller's later work."""
        if self.stream is None:
            yield
            return
        cur = self.torch.cuda.current_stream(self.dev)
        self.stream.wait_stream(cur)
        with self.torch.cuda.stream(self.stream):
            yield
        cur.wait_stream(self.stream)

    @property
    def gamma(self):
        """Damping gamma = 3 / (N_tau dt) (Sec. 3: N_tau ~ 3 / (gamma dt))."""
        return 3.0 / (self.n_steps * self.dt)

    def run_batch(self, sample0, sigma_out, x_out):
        """Samples sample0 .. sample0 + run_samples - 1; writes Sigma_i(t) [run_samples][2N+1]
        (complex128) and X_i [run_samples]."""
        with self.on_stream():
            self._run_batch(sample0, sigma_out, x_out)

    def filter_batch(self, sample0):
        """White noise and the occupied filter (Eq. 3) of samples sample0 .. sample0 + run_samples - 1,
        kept in the pipeline for `propagate_batch`."""
        with self.on_stream():
            self._filter_batch(sample0)

    def propagate_batch(self, sample0, sigma_out, x_out):
        """Everything after the filter for the batch `filter_batch` left (sample0 must be the same):
        exchange, TDH, time ordering, zeta propagation and Sigma(t)."""
        with self.on_stream():
            self._propagate_batch(sample0, sigma_out, x_out)

    def _filter_batch(self, sample0):
        c, ne = self.ctx, self.n_eta
        c.white_noise(self.seed, self.stream_id, sample0, self.run_samples, ne + 1, self.noise)
        c.filter_occupied(self.coeffs, self.noise, self.filt)

    def _run_batch(self, sample0, sigma_out, x_out):
        self._filter_batch(sample0)
        self._propagate_batch(sample0, sigma_out, x_out)

    def _propagate_batch(self, sample0, sigma_out, x_out):
        c, ns, ne, N = self.ctx, self.ns, self.n_eta, self.n_steps
        for g in range(self.group):
            s0 = g * ns
            rows = slice(s0 * (ne + 1), (s0 + ns) * (ne + 1))
            c.prepare_sample(self.noise[rows], self.filt[rows], self.phi, ns, ne, self.eta,
                             self.zeta[2 * s0:2 * (s0 + ns)], self.source)
            c.exchange(self.eta, self.phi, ns, ne, x_out[s0:s0 + ns])
            if self.xi is None:
                c.tdh_response(self.eta, self.source, ns, ne, N, self.dt, self.cheb_deg, self.uR)
                c.time_order(self.uR, self.u[s0:s0 + ns], ns, N)
            else:
                c.tdh_response_xi(self.eta, self.source, ns, ne, N, self.dt, self.cheb_deg,
                                  self._xi_args(sample0 + s0), self.uR)
                c.time_order_points(self.uR, self.u[s0:s0 + ns], ns, N, self.xi['n_xi'])
        if self.xi is None:
            c.sigma_c(self.zeta, self.phi, self.u, self.run_samples, N, self.dt, self.cheb_deg, sigma_out, self.fp64)
        else:
            c.sigma_c_xi(self.zeta, self.phi, self.u, self.run_samples, N, self.dt, self.cheb_deg,
                         self._xi_args(sample0), sigma_out, self.fp64)

    def run(self, n_samples, sample0=0):
        """Run n_samples (rounded up to whole runs); returns device Sigma [n][2N+1] and X [n]."""
        t = self.torch
        rs = self.run_samples
        nb = (n_samples + rs - 1) // rs
        sig = t.empty(nb * rs, 2 * self.n_steps + 1, dtype=t.complex128, device=self.dev)
        xs = t.empty(nb * rs, dtype=t.float64, device=self.dev)
        for b in range(nb):
            s0 = b * rs
            self.run_batch(sample0 + s0, sig[s0:s0 + rs], xs[s0:s0 + rs])
        return sig[:n_samples], xs[:n_samples]

    def qp(self, sigma, x, eps_ks, vxc=0.0, window=2.0, step=1e-3, fp64=None):
        f = self.fp64 if fp64 is None else (1 if fp64 else 0)
        with self.on_stream():
            return self.ctx.qp_energy(sigma.contiguous(), x.contiguous(), sigma.shape[0], self.n_steps, self.dt,
                                      self.gamma, eps_ks, vxc, window, step, f)
