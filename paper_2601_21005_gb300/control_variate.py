"""Learned control variate for the stochastic Sigma_c(t) and X (the product path, through the C ABI).

A sample's Sigma_i(t) (Eq. 5) and its sROI exchange X_i (Eq. 6) are quadratic forms in the
sample's random vectors (zeta-bar_i and the eta-bar_il), so cheap features of those vectors --
the Coulomb-weighted low-k power of zeta-bar_i phi and of eta-bar_il phi, summed per |k| shell --
predict part of them.  The predictor is f = (FP64 ridge-linear part on the per-|k|-shell sums of the
features) + (network on the per-k features, fitted to what the linear part leaves).
The steps:

  collect : run plain samples (Pipeline.run_batch); targets Y_i = [Sigma_i(t) (2 (2N + 1) reals),
            X_i], per-k features x_i of the same samples;
  train   : fit the linear part on the training samples (FP64 normal equations), then the
            network on the standardised residuals Y - f_lin(x) (GPU forward, backward, Adam),
            keeping the epoch with the lowest held-out loss -- and the network only if that
            loss beats predicting zero residual;
  estimate: with n new paired samples (Y_i, x_i) and M cheap samples (features only: the same
            Philox vectors of sample indices never run through the plain path), form the rows
            z_i = mean_j f(x_j) + Y_i - f(x_i) (FP64) and solve the QP equation on them.  The
            estimate is unbiased for any f; with no cheap samples it is the plain one.
"""
import time

import numpy as np

from . import sgw as _sgw

HA_EV = 27.211386245988


class ControlVariate:
    # ridge 0.1 (on standardised inputs): the best held-out variance ratio of the linear part for
    # 128 and 256 training samples on the 64^3 cluster (2.52 / 2.69 against 2.42 / 2.66 at 1e-3)
    def __init__(self, pipeline, m2max=10, width=256, seed=77, max_batch=256, ridge=0.1, linear=True):
        import torch
        self.torch = torch
        self.pl = pipeline
        self.m2max = m2max
        self.n_kfeat = _sgw.sgw_cv_feature_count(m2max)      # per-k features: the network's inputs
        self.n_feat = _sgw.sgw_cv_shell_count(m2max)         # their shell sums: the linear part's inputs
        self.n_sig = 2 * (2 * pipeline.n_steps + 1)
        self.n_out = self.n_sig + 1
        self.max_batch = max_batch
        self.ridge = ridge
        self.linear = linear        # False: no linear part (f_lin = 0), the network alone on Y
        self.linear_used = linear   # False when the fitted linear part failed its hold-out test
        self.lin = torch.zeros(_sgw.sgw_cv_linear_size(self.n_feat, self.n_out), dtype=torch.float64,
                               device=pipeline.dev)
        self.use_net = True
        self.mlp = _sgw.MLP(self.n_kfeat, width, self.n_out, max_batch, seed=seed, device=pipeline.dev.index or 0,
                            stream=pipeline.stream.cuda_stream if pipeline.stream is not None else None)
        # X is one output against 2 (2N + 1) for Sigma(t) but carries a comparable share of the
        # QP variance: give it half the weight of the whole Sigma block.
        w = np.ones(self.n_out, dtype=np.float32)
        w[-1] = 0.5 * self.n_sig
        self.mlp.set_loss_weights(w)
        dev = pipeline.dev
        f64 = torch.float64
        self.mu = torch.zeros(self.n_out, dtype=f64, device=dev)
        self.sd = torch.ones(self.n_out, dtype=f64, device=dev)
        self.mu_x = torch.zeros(self.n_kfeat, dtype=f64, device=dev)
        self.sd_x = torch.ones(self.n_kfeat, dtype=f64, device=dev)
        self._noise = None

    # -------------------------------------------------------------- data
    def collect(self, n_samples, sample0):
        with self.pl.on_stream():
            return self._collect(n_samples, sample0)

    def _collect(self, n_samples, sample0):
        """Plain samples sample0.. : (Y [n][n_out] f64 = [Sigma(t) interleaved, X], F [n][n_kfeat] f32)."""
        t, pl = self.torch, self.pl
        ns = pl.run_samples
        nb = (n_samples + ns - 1) // ns
        S = t.empty(nb * ns, 2 * pl.n_steps + 1, dtype=t.complex128, device=pl.dev)
        X = t.empty(nb * ns, dtype=t.float64, device=pl.dev)
        for b in range(nb):
            s0 = b * ns
            pl._run_batch(sample0 + s0, S[s0:s0 + ns], X[s0:s0 + ns])
        # the features of the same samples, from their white noise (regenerated: counter-based)
        F = self._cheap_features(n_samples, sample0)
        Y = t.cat([t.view_as_real(S).reshape(nb * ns, -1), X[:, None]], dim=1)[:n_samples].contiguous()
        return Y, F

    def cheap_features(self, n_samples, sample0):
        with self.pl.on_stream():
            return self._cheap_features(n_samples, sample0)

    def _cheap_features(self, n_samples, sample0):
        """Per-k features of samples sample0.. from their white noise alone (no filter, no propagation)."""
        t, pl = self.torch, self.pl
        nv = pl.n_eta + 1
        chunk = max(1, pl.ctx.max_batch // nv)
        if self._noise is None:
            self._noise = t.empty(chunk * nv, pl.ng, dtype=t.complex64, device=pl.dev)
        Fk = t.empty(n_samples, self.n_kfeat, dtype=t.float32, device=pl.dev)
        for s0 in range(0, n_samples, chunk):
            m = min(chunk, n_samples - s0)
            pl.ctx.white_noise(pl.seed, pl.stream_id, sample0 + s0, m, nv, self._noise)
            pl.ctx.cv_features(self._noise, m, nv, pl.phi, self.m2max, Fk[s0:s0 + m])
        return Fk

    def _shells(self, F):
        """Per-shell sums of per-k features (the linear part's inputs)."""
        out = self.torch.empty(F.shape[0], self.n_feat, dtype=self.torch.float32, device=F.device)
        self.pl.ctx.cv_shell_sums(F.contiguous(), self.m2max, out)
        return out

    # -------------------------------------------------------------- network
    def train(self, F, Y, epochs=300, batch=64, lr=1e-3, holdout=0.2, eps_ks=None):
        with self.pl.on_stream():
            return self._train(F, Y, epochs, batch, lr, holdout, eps_ks)

    def _train(self, F, Y, epochs, batch, lr, holdout, eps_ks=None):
        """Fit the linear part, then the network on its residuals; the network parameters of the
        epoch with the lowest held-out loss are kept.  With eps_ks (the target's KS energy) the
        linear part is held out too: the QP standard error of the held-out samples' rows with it
        (the training samples standing in for the cheap set) must be 2% below that of their plain
        rows, else it is dropped (f_lin = 0).  Returns (training losses, held-out losses)."""
        t, ctx = self.torch, self.pl.ctx
        n = F.shape[0]
        nv = max(1, int(round(holdout * n))) if n > 4 else 0
        ntr = n - nv
        self.linear_used = self.linear
        if self.linear:
            Fs = self._shells(F)
            ctx.cv_linear_fit(Fs[:ntr].contiguous(), Y[:ntr].contiguous(), self.ridge, self.lin)
            if eps_ks is not None and nv >= 4:
                Yv = Y[ntr:].clone()                 # fresh (aligned) buffers for the row slices
                rows = t.empty_like(Yv)
                ctx.cv_linear_rows(self.lin, Fs[:ntr].clone(), Fs[ntr:].clone(), Yv, rows)
                try:
                    se_lin = self.pl.qp(*self.plain_rows(rows), eps_ks)['se']
                    se_plain = self.pl.qp(*self.plain_rows(Yv), eps_ks)['se']
                    self.linear_used = bool(se_lin < 0.98 * se_plain)
                except _sgw.SgwError as e:
                    if e.status != 6:            # SGW_ENOCONV: no QP root for the held-out rows
                        raise                    # (no verdict: the linear part stays); anything else is an error
        if self.linear_used:
            R = t.empty_like(Y)
            ctx.cv_linear_apply(self.lin, Fs, self.n_out, R, y=Y)     # residuals Y - f_lin(x)
            Y = R
        Fs = F.clone()
        ctx.cv_standardize_f32(Fs[:ntr], self.mu_x, self.sd_x, True)
        if nv:
            ctx.cv_standardize_f32(Fs[ntr:], self.mu_x, self.sd_x, False)
        T = t.empty(Y.shape, dtype=t.float32, device=Y.device)
        ctx.cv_standardize(Y[:ntr].contiguous(), self.mu, self.sd, T[:ntr], True)
        if nv:
            ctx.cv_standardize(Y[ntr:].contiguous(), self.mu, self.sd, T[ntr:], False)
        bs = min(batch, self.max_batch)
        tr_l, va_l = [], []
        best, best_p = float('inf'), None
        for _ in range(epochs):
            tr_l.append(self.mlp.train_epoch(Fs[:ntr], T[:ntr], bs, lr))
            if nv:
                vl, _ = self.mlp.gradients(Fs[ntr:ntr + min(nv, self.max_batch)],
                                           T[ntr:ntr + min(nv, self.max_batch)])
                va_l.append(vl)
                if vl < best:
                    best, best_p = vl, self.mlp.get_params()
        if best_p is not None:
            self.mlp.set_params(best_p)
        self.use_net = True
        if nv:
            # the network is kept only if it beats predicting zero residual on the held-out part by
            # a clear margin (2%): a network that has learnt nothing adds its own noise to the rows
            p_keep = self.mlp.get_params()
            self.mlp.set_params(np.zeros_like(p_keep))
            zero_l, _ = self.mlp.gradients(Fs[ntr:ntr + min(nv, self.max_batch)], T[ntr:ntr + min(nv, self.max_batch)])
            self.mlp.set_params(p_keep)
            self.use_net = best < 0.98 * zero_l
        return tr_l, va_l

    def predict(self, F):
        with self.pl.on_stream():
            return self._predict(F)

    def _predict(self, F):
        """Network outputs (standardised units) for raw features F."""
        t = self.torch
        Fs = F.clone()
        self.pl.ctx.cv_standardize_f32(Fs, self.mu_x, self.sd_x, False)
        out = t.empty(F.shape[0], self.n_out, dtype=t.float32, device=F.device)
        for s0 in range(0, F.shape[0], self.max_batch):
            m = min(self.max_batch, F.shape[0] - s0)
            self.mlp.forward(Fs[s0:s0 + m].contiguous(), out[s0:s0 + m])
        return out

    # -------------------------------------------------------------- estimator
    def rows(self, F_cheap, F_paired, Y_paired):
        with self.pl.on_stream():
            return self._rows(F_cheap, F_paired, Y_paired)

    def _rows(self, F_cheap, F_paired, Y_paired):
        """Control-variate rows: (Sigma rows [n][2N+1] complex128, X rows [n] f64)."""
        t = self.torch
        rows = t.empty_like(Y_paired)
        if F_cheap is None:
            self.pl.ctx.cv_rows(None, None, Y_paired, None, None, rows)
        else:
            if self.linear_used:                 # Y - f_lin(x_paired) + mean f_lin(x_cheap)
                Yl = t.empty_like(Y_paired)
                self.pl.ctx.cv_linear_rows(self.lin, self._shells(F_cheap), self._shells(F_paired), Y_paired, Yl)
            else:                                # no linear part: f_lin = 0 (an unfitted buffer holds no scales)
                Yl = Y_paired
            if self.use_net:
                self.pl.ctx.cv_rows(self._predict(F_cheap), self._predict(F_paired), Yl, self.mu, self.sd, rows)
            else:
                rows = Yl
        n = rows.shape[0]
        sig = t.view_as_complex(rows[:, :self.n_sig].contiguous().reshape(n, -1, 2)).contiguous()
        return sig, rows[:, self.n_sig].contiguous()

    def cheap_mean_rows(self, F_cheap, sigma_rows, x_rows):
        """Rows whose QP standard error is the part the paired rows cannot show: the spread of the
        cheap-sample mean (1/M) sum_j f(x_j).  Every row z_i = mean_j f(x_j) + Y_i - f(x_i) shares
        that mean, so its fluctuation is missing from the spread of the z_i; its variance is
        Var_j f(x_j) / M.  The returned M rows are mean(z) + mean_j f(x_j) - f(x_k) (k over the cheap
        samples): their mean is the estimate's, so the QP solve finds the same root and Z, and their
        spread is that of f over the cheap samples.  Total standard error: the two added in
        quadrature."""
        with self.pl.on_stream():
            t = self.torch
            n = sigma_rows.shape[0]
            z = t.cat([t.view_as_real(sigma_rows).reshape(n, -1), x_rows[:, None]], dim=1)
            Y = z.mean(dim=0, keepdim=True).expand(F_cheap.shape[0], -1).contiguous()
            return self._rows(F_cheap, F_cheap, Y)

    def plain_rows(self, Y_paired):
        n = Y_paired.shape[0]
        t = self.torch
        return (t.view_as_complex(Y_paired[:, :self.n_sig].contiguous().reshape(n, -1, 2)).contiguous(),
                Y_paired[:, self.n_sig].contiguous())


def study(pl, eps_ks, n_train, paired_batches, n_cheap, sample0, plain_sample_s, target_ev=0.03, epochs=200):
    """Train the control variate on n_train plain samples, then compare, at equal target error
    (target_ev on the QP energy), the plain estimator charged its own per-sample time
    (plain_sample_s) with the control-variate estimator charged for its paired samples (the plain
    work plus their features) and for r = M/n cheap samples per paired one.  The control variate's
    variance is that of its rows over n plus that of the cheap-sample mean over M (the rows share
    that mean, so their spread cannot show it).  Samples: training from sample0 + 300000, paired
    from sample0 + 400000, cheap from sample0 + 500000.  Returns a dict of the measured figures."""
    import torch
    ns = pl.run_samples
    cv = ControlVariate(pl, m2max=10, width=256, max_batch=256, seed=11)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    Yt, Ft = cv.collect(n_train, sample0 + 300000)
    tr, va = cv.train(Ft, Yt, epochs=epochs, batch=64, lr=1e-3, eps_ks=eps_ks)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    st = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    Ys, Fs = [], []
    e0.record(st)
    for b in range(paired_batches):
        Y, F = cv.collect(ns, sample0 + 400000 + b * ns)
        Ys.append(Y)
        Fs.append(F)
    e1.record(st)
    torch.cuda.synchronize()
    n = ns * paired_batches
    paired_s = e0.elapsed_time(e1) * 1e-3 / n           # plain pipeline + the sample's features
    if plain_sample_s is None:                           # the plain form charged the paired time
        plain_sample_s = paired_s
    e0.record(st)
    Fc = cv.cheap_features(n_cheap, sample0 + 500000)
    e1.record(st)
    torch.cuda.synchronize()
    cheap_s = e0.elapsed_time(e1) * 1e-3 / n_cheap
    Yp, Fp = torch.cat(Ys), torch.cat(Fs)
    S1, X1 = cv.rows(Fc, Fp, Yp)
    r_cv = pl.qp(S1, X1, eps_ks)
    Sc, Xc = cv.cheap_mean_rows(Fc, S1, X1)
    r_cheap = pl.qp(Sc, Xc, eps_ks)
    S0, X0 = cv.plain_rows(Yp)
    r_pl = pl.qp(S0, X0, eps_ks)
    net_kept = cv.use_net
    cv.use_net = False
    S2, X2 = cv.rows(Fc, Fp, Yp)
    Sc2, Xc2 = cv.cheap_mean_rows(Fc, S2, X2)
    r_lin = pl.qp(S2, X2, eps_ks)
    r_lin_c = pl.qp(Sc2, Xc2, eps_ks)
    # the linear part with the network on its residual whether or not the hold-out test kept it
    cv.use_net = True
    S4, X4 = cv.rows(Fc, Fp, Yp)
    Sc4, Xc4 = cv.cheap_mean_rows(Fc, S4, X4)
    r_both, r_both_c = pl.qp(S4, X4, eps_ks), pl.qp(Sc4, Xc4, eps_ks)
    cv.use_net = net_kept
    # the network alone (no linear part), trained on the same samples and used as trained
    t1 = time.perf_counter()
    cvn = ControlVariate(pl, m2max=10, width=256, max_batch=256, seed=11, linear=False)
    cvn.train(Ft, Yt, epochs=epochs, batch=64, lr=1e-3)
    net_alone_kept = cvn.use_net
    cvn.use_net = True
    S3, X3 = cvn.rows(Fc, Fp, Yp)
    Sc3, Xc3 = cvn.cheap_mean_rows(Fc, S3, X3)
    r_net, r_net_c = pl.qp(S3, X3, eps_ks), pl.qp(Sc3, Xc3, eps_ks)
    cvn.mlp.close()
    torch.cuda.synchronize()
    t_net_alone = time.perf_counter() - t1
    se_cv = (r_cv['se'] ** 2 + r_cheap['se'] ** 2) ** 0.5
    se_lin = (r_lin['se'] ** 2 + r_lin_c['se'] ** 2) ** 0.5
    se_both = (r_both['se'] ** 2 + r_both_c['se'] ** 2) ** 0.5
    se_net = (r_net['se'] ** 2 + r_net_c['se'] ** 2) ** 0.5
    target = target_ev / HA_EV
    r = n_cheap / n
    # per paired sample, the variance at ratio r: n se_rows^2 + (M se_cheap^2) / r
    var_cv = n * r_cv['se'] ** 2 + n_cheap * r_cheap['se'] ** 2 / r
    need_pl, need_cv = n * r_pl['se'] ** 2 / target ** 2, var_cv / target ** 2
    t_plain = need_pl * plain_sample_s
    t_cv = need_cv * (paired_s + r * cheap_s)
    return dict(n_train=n_train, n_paired=n, n_cheap=n_cheap, train_seconds=round(t_train, 2),
                heldout_loss_first_best=[round(va[0], 4), round(min(va), 4)] if va else None,
                qp_eV_plain=round(r_pl['eps_qp'] * HA_EV, 5), se_eV_plain=round(r_pl['se'] * HA_EV, 5),
                qp_eV_cv=round(r_cv['eps_qp'] * HA_EV, 5), se_eV_cv=round(se_cv * HA_EV, 5),
                se_eV_cv_rows=round(r_cv['se'] * HA_EV, 5), se_eV_cv_cheap_mean=round(r_cheap['se'] * HA_EV, 5),
                variance_gain=round((r_pl['se'] / se_cv) ** 2, 3),
                variance_gain_linear_part_alone=round((r_pl['se'] / se_lin) ** 2, 3), network_kept=bool(net_kept),
                linear_part_kept=bool(cv.linear_used),
                variance_gain_linear_plus_network=round((r_pl['se'] / se_both) ** 2, 3),
                variance_gain_network_alone=round((r_pl['se'] / se_net) ** 2, 3),
                network_alone_passed_holdout=bool(net_alone_kept), network_alone_train_seconds=round(t_net_alone, 2),
                seconds_per_sample=dict(plain=round(plain_sample_s, 4), paired=round(paired_s, 4),
                                        cheap=round(cheap_s, 6)),
                time_to_target_plain_s=round(t_plain, 1), time_to_target_cv_s=round(t_cv, 1),
                time_to_target_cv_incl_training_s=round(t_cv + t_train, 1), target_eV=target_ev,
                speedup=round(t_plain / t_cv, 3), speedup_incl_training=round(t_plain / (t_cv + t_train), 3))
