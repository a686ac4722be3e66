"""Lowest Kohn-Sham states of H0 on the GPU (setup only, outside the timed path).

The paper takes E_HOMO, E_LUMO and the target orbital from a preliminary DFT run (Sec. 2.1,
items 4-5 of the inputs; Sec. 3).  For the synthetic systems here they come from a
Chebyshev-filtered subspace iteration (Zhou & Saad, 2007): the block is filtered with
T_m(H~) on the interval [cut, E_max] (which damps everything above `cut` and amplifies
the states below it), orthonormalised, and rotated by a Rayleigh-Ritz step; `cut` follows
the largest Ritz value.  The H applications and the filter run in libsgw; the block
products run as torch matmuls, and the m x m factorisations (Cholesky, eigh) on the host.
"""
import numpy as np


def _orth_rows(A, torch):
    """Rows of A orthonormalised by Cholesky QR, done twice, with FP64 Gram matrices."""
    for _ in range(2):
        A64 = A.to(torch.complex128)
        G = (A64.conj() @ A64.transpose(0, 1)).cpu().numpy()      # G_ij = <a_i|a_j>
        G = 0.5 * (G + G.conj().T)
        L = np.linalg.cholesky(G.T)                               # G^T = L L^H
        Li = np.linalg.inv(L)
        A = (torch.from_numpy(Li).to(A64.device) @ A64).to(torch.complex64)
    return A.contiguous()


def lowest_states(ctx, n_want, emin, emax, extra=24, degree=60, max_iter=40, tol=1e-5, seed=4242):
    """Return (eigenvalues [n_want] ascending, orbitals [n_want, N_g] real float64 normalised
    to dV sum phi^2 = 1, max residual).  ctx needs max_batch >= n_want + extra."""
    import torch
    m = n_want + extra
    ng = ctx.ng
    dev = torch.device('cuda', ctx.device)
    X = torch.empty(m, ng, dtype=torch.complex64, device=dev)
    ctx.white_noise(seed, 0xE16E, 0, 1, m, X)
    Y = torch.empty_like(X)
    coeff = np.zeros(degree + 1)
    coeff[-1] = 1.0

    def rayleigh_ritz(Q):
        ctx.apply_h(Q, Y)
        Q64, Y64 = Q.to(torch.complex128), Y.to(torch.complex128)
        Hs = (Q64.conj() @ Y64.transpose(0, 1)).cpu().numpy()    # <q_i|H q_j>
        Hs = 0.5 * (Hs + Hs.conj().T)
        w, V = np.linalg.eigh(Hs)
        R = torch.from_numpy(V.T.copy()).to(Q64.device)        # new q_k = sum_i V_ik q_i
        Qn = (R @ Q64)
        HQ = (R @ Y64)
        res = torch.sqrt(torch.sum(torch.abs(HQ - torch.from_numpy(w).to(Q64.device)[:, None] * Qn) ** 2, dim=1))
        return w, Qn.to(torch.complex64).contiguous(), res.cpu().numpy()

    Q = _orth_rows(X, torch)
    w, Q, res = rayleigh_ritz(Q)
    for _ in range(max_iter):
        if np.max(res[:n_want + 1]) < tol * max(1.0, np.max(np.abs(w[:n_want + 1]))):
            break
        cut = float(w[-1])
        ctx.set_spectrum(cut, emax)
        ctx.filter_occupied(coeff, Q, X)
        Q = _orth_rows(X, torch)
        w, Q, res = rayleigh_ritz(Q)
    ctx.set_spectrum(emin, emax)
    phis = []
    for i in range(n_want):
        q = Q[i].cpu().numpy().astype(np.complex128)
        k = np.argmax(np.abs(q))
        q = q * np.exp(-1j * np.angle(q[k]))
        r = q.real
        r /= np.sqrt(ctx.dV * np.sum(r * r))
        if r.sum() < 0:
            r = -r
        phis.append(r)
    return w[:n_want], np.array(phis), float(np.max(res[:n_want]))


# ---------------------------------------------------------------- states near the gap
# For large systems (the 288^3 cluster has ~15 000 occupied states) the block above cannot hold every
# occupied state.  The states next to the gap are found instead by (1) the kernel polynomial method
# (Weisse et al., Rev. Mod. Phys. 78, 275 (2006)): Chebyshev moments mu_k = dV <v|T_k(H~)|v> of
# Rademacher probes v (E[dV v v^T] = 1), from which the state count N(E) = Tr Theta(E - H) and the
# density of states follow for every E as Jackson-damped series.  With fixed probes the estimated
# N(E) changes only at eigenvalues, so a gap shows as a minimum of the estimated density of states
# even though N itself is uncertain by ~sqrt(2 n_occ / n_probe) states: the gap taken is the density
# minimum among the energies whose count is compatible with n_occ.  (2) A subspace iteration whose
# filter is a Gaussian of H centred in that gap, which amplifies the states nearest to it most, so
# the block converges to the m states closest to it.  (3) HOMO and LUMO are the converged Ritz values
# just below and just above the gap centre.


def jackson_kernel(degree):
    """Jackson damping factors g_k, k = 0..degree (removes the Gibbs oscillations of a truncated
    Chebyshev series; KPM review, Eq. 71)."""
    n1 = degree + 1
    k = np.arange(n1)
    a = np.pi / n1
    return ((n1 - k) * np.cos(a * k) + np.sin(a * k) / np.tan(a)) / n1


def step_coeffs(e, emin, emax, degree):
    """Jackson-damped Chebyshev coefficients of Theta(e - H) for H mapped from [emin, emax] to
    [-1, 1] (e scalar or array, coefficients along the last axis): the indicator of [-1, x_e] has,
    with x = cos(theta), c_0 = (pi - theta_e)/pi and c_k = -2 sin(k theta_e) / (k pi)."""
    c, h = 0.5 * (emax + emin), 0.5 * (emax - emin)
    te = np.arccos(np.clip((np.atleast_1d(np.asarray(e, dtype=np.float64)) - c) / h, -1.0, 1.0))[..., None]
    k = np.arange(1, degree + 1)
    out = np.concatenate([(np.pi - te) / np.pi, -2.0 * np.sin(k * te) / (k * np.pi)], axis=-1)
    out = out * jackson_kernel(degree)
    return out[0] if np.ndim(e) == 0 else out


def gaussian_coeffs(center, sigma, emin, emax, degree, damped=False):
    """Chebyshev coefficients of exp(-(H - center)^2 / (2 sigma^2)) on [emin, emax] by Chebyshev-Gauss
    quadrature at 4 (degree + 1) nodes (discrete orthogonality of the T_k there).  damped=True
    multiplies them by the Jackson factors: the truncated series then has no Gibbs oscillations
    (it stays positive and small far from the centre) at the price of a width broadened by about
    pi (emax - emin) / (2 degree)."""
    M = 4 * (degree + 1)
    th = np.pi * (np.arange(M) + 0.5) / M
    c, h = 0.5 * (emax + emin), 0.5 * (emax - emin)
    f = np.exp(-((c + h * np.cos(th)) - center) ** 2 / (2.0 * sigma * sigma))
    k = np.arange(degree + 1)
    out = (2.0 / M) * (np.cos(np.outer(k, th)) @ f)
    out[0] *= 0.5
    return out * jackson_kernel(degree) if damped else out


def cheb_moments(ctx, emin, emax, n_probe=16, degree=1000, seed=777, device=None):
    """Per-probe Chebyshev moments mu[p][k] = dV Re <v_p|T_k(H~)|v_p>, k = 0..degree, H~ = H mapped
    from [emin, emax] to [-1, 1], by the three-term recurrence (one H application per k through the
    library; the recurrence and the products in FP32 on the device, the moments in FP64)."""
    import torch
    dev = device if device is not None else torch.device('cuda', ctx.device)
    c, h = 0.5 * (emax + emin), 0.5 * (emax - emin)
    V = torch.empty(n_probe, ctx.ng, dtype=torch.complex64, device=dev)
    ctx.white_noise(seed, 0xC0DE, 0, 1, n_probe, V)
    Y = torch.empty_like(V)
    mu = np.zeros((n_probe, degree + 1))

    def mom(T):
        return (ctx.dV * torch.sum((V.conj() * T).real.to(torch.float64), dim=1)).cpu().numpy()

    t0 = V.clone()
    mu[:, 0] = mom(t0)
    if degree == 0:
        return mu
    ctx.apply_h(t0, Y)
    t1 = (Y - c * t0) / h
    mu[:, 1] = mom(t1)
    for k in range(2, degree + 1):
        ctx.apply_h(t1.contiguous(), Y)
        t2 = 2.0 * (Y - c * t1) / h - t0
        mu[:, k] = mom(t2)
        t0, t1 = t1, t2
    return mu


def count_and_dos(mu, energies, emin, emax):
    """From per-probe moments: the estimated N(E) (mean over probes), its standard error, and the
    estimated density of states dN/dE, at each energy."""
    degree = mu.shape[1] - 1
    C = step_coeffs(np.asarray(energies), emin, emax, degree)          # [n_e][degree + 1]
    Np = C @ mu.T                                                      # [n_e][n_probe]
    n = Np.mean(axis=1)
    se = Np.std(axis=1, ddof=1) / np.sqrt(mu.shape[0])
    # d/dE of the Jackson-damped step series: the KPM density g_k mu_k T_k(x) (2 - delta_k0) / (pi h sqrt(1-x^2))
    c, h = 0.5 * (emax + emin), 0.5 * (emax - emin)
    x = np.clip((np.asarray(energies) - c) / h, -1 + 1e-12, 1 - 1e-12)
    k = np.arange(degree + 1)
    w = jackson_kernel(degree) * np.where(k == 0, 1.0, 2.0)
    T = np.cos(np.outer(np.arccos(x), k))
    dos = (T @ (w * mu.mean(axis=0))) / (np.pi * h * np.sqrt(1.0 - x * x))
    return n, se, dos


def find_gap(mu, n_occ, emin, emax, n_grid=4000):
    """Centre of the gap above state n_occ: the minimum of the estimated density of states among the
    energies whose estimated count is within 3 standard errors + 1 of n_occ.  Returns
    (energy, count there, its standard error)."""
    e = np.linspace(emin, emax, n_grid)
    n, se, dos = count_and_dos(mu, e, emin, emax)
    ok = np.abs(n - n_occ) <= 3.0 * se + 1.0
    if not ok.any():
        raise RuntimeError('no energy with a state count compatible with n_occ')
    i = np.where(ok)[0][np.argmin(dos[ok])]
    return float(e[i]), float(n[i]), float(se[i])


def states_near_gap(ctx, n_occ, emin, emax, m=16, sigma=None, n_probe=16, count_degree=1000,
                    window_degree=2000, max_iter=60, tol=2e-4, seed=4243, device=None, log=None):
    """E_HOMO, E_LUMO and the HOMO orbital of an n_occ-occupied system without computing every
    occupied state.  Returns (e_homo, e_lumo, phi_homo [N_g] real float64 normalised to
    dV sum phi^2 = 1, info): info holds the gap centre, the estimated state count there and its
    standard error, the Ritz values and residuals, and the LUMO orbital (phi_lumo, same normalisation).
    When the HOMO or LUMO level is degenerate, the orbital is one vector of that level.  ctx needs max_batch >= max(m, n_probe).  log: optional callable
    taking a progress line (the gap search, then each iteration's HOMO/LUMO Ritz values).

    The window is the Jackson-damped Gaussian of degree window_degree; its default width sigma is
    1.5 pi (emax - emin) / (2 window_degree), the smallest the damped series resolves, so that the
    states next to the gap are amplified most against their neighbours.  tol is the relative
    residual at which the HOMO and LUMO Ritz pairs count as converged; FP32 H applications floor
    the residual near 1e-4 of |H|, hence the default 2e-4."""
    import torch
    dev = device if device is not None else torch.device('cuda', ctx.device)
    ctx.set_spectrum(emin, emax)
    mu = cheb_moments(ctx, emin, emax, n_probe, count_degree, device=dev)
    ef, n_ef, se_ef = find_gap(mu, n_occ, emin, emax)
    if log:
        log('gap search: centre %.6f Ha, estimated count %.1f +- %.1f (n_occ %d)' % (ef, n_ef, se_ef, n_occ))
    sig = sigma if sigma is not None else 1.5 * np.pi * 0.5 * (emax - emin) / window_degree
    coeff = gaussian_coeffs(ef, sig, emin, emax, window_degree, damped=True)
    X = torch.empty(m, ctx.ng, dtype=torch.complex64, device=dev)
    ctx.white_noise(seed, 0xE16F, 0, 1, m, X)
    Y = torch.empty_like(X)

    def orth(A):
        # dV-orthonormal rows (Cholesky QR twice, FP64 Gram matrices)
        for _ in range(2):
            A64 = A.to(torch.complex128)
            G = (A64.conj() @ A64.transpose(0, 1)).cpu().numpy() * ctx.dV
            G = 0.5 * (G + G.conj().T)
            Li = np.linalg.inv(np.linalg.cholesky(G.T))
            A = (torch.from_numpy(Li).to(A64.device) @ A64).to(torch.complex64)
        return A.contiguous()

    def rayleigh_ritz(Q):
        ctx.apply_h(Q, Y)
        Q64, Y64 = Q.to(torch.complex128), Y.to(torch.complex128)
        Hs = (Q64.conj() @ Y64.transpose(0, 1)).cpu().numpy() * ctx.dV
        Hs = 0.5 * (Hs + Hs.conj().T)
        w, V = np.linalg.eigh(Hs)
        R = torch.from_numpy(V.T.copy()).to(Q64.device)
        Qn, HQ = R @ Q64, R @ Y64
        res = torch.sqrt(ctx.dV * torch.sum(torch.abs(HQ - torch.from_numpy(w).to(Q64.device)[:, None] * Qn) ** 2,
                                            dim=1))
        return w, Qn.to(torch.complex64).contiguous(), res.cpu().numpy()

    def pair(w):
        below, above = np.where(w < ef)[0], np.where(w > ef)[0]
        return (below[-1] if len(below) else None), (above[0] if len(above) else None)

    Q = orth(X)
    w, Q, res = rayleigh_ritz(Q)
    for it in range(max_iter):
        ih, il = pair(w)
        if log and ih is not None and il is not None:
            log('iteration %d: HOMO %.8f (res %.1e), LUMO %.8f (res %.1e)' % (it, w[ih], res[ih], w[il], res[il]))
        if ih is not None and il is not None and max(res[ih], res[il]) < tol * max(1.0, abs(w[ih]), abs(w[il])):
            break
        ctx.filter_occupied(coeff, Q, X)
        Q = orth(X)
        w, Q, res = rayleigh_ritz(Q)
    ih, il = pair(w)
    if ih is None or il is None:
        raise RuntimeError('no Ritz value on one side of the gap centre')
    def real_orbital(i):
        q = Q[i].cpu().numpy().astype(np.complex128)
        k = np.argmax(np.abs(q))
        r = (q * np.exp(-1j * np.angle(q[k]))).real
        r /= np.sqrt(ctx.dV * np.sum(r * r))
        return -r if r.sum() < 0 else r

    info = dict(gap_centre=ef, count_at_gap=n_ef, count_se=se_ef, ritz=w.tolist(), residuals=res.tolist(),
                max_residual=float(max(res[ih], res[il])), phi_lumo=real_orbital(il))
    return float(w[ih]), float(w[il]), real_orbital(ih), info
