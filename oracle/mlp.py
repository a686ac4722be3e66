"""FP64 oracle: the learned control variate for the stochastic Sigma_c(t).

TEST INFRASTRUCTURE: part of the CPU oracle; only tests, the smoke check and the
CPU-baseline leg of the benchmark may use it.

The paper has no learned part; this is the control variate the hot path adds around the
plain sROI estimator (a sample's Sigma_i(t) is a quadratic form in its random vector
zeta-bar_i, Eq. 4-5, so cheap functions of zeta-bar predict part of it):

* features of a sample: for a random vector v and the orbital phi, F_v(k) = dV sum_r
  v(r) phi(r) e^{-i k.r} on the shells 0 < |m|^2 <= m2max (k = 2 pi m / L, one of each +-k
  pair: the first non-zero component of m positive) weighted by sqrt(4 pi)/|k|; the features
  are |F_zeta(k)|^2 for each k and F_zeta(0)^2 for zeta-bar, then sum_l |F_eta_l(k)|^2 and
  sum_l F_eta_l(0)^2 over the sample's eta-bar_l (these drive the fluctuations of the
  Coulomb-weighted quadratic forms behind Sigma_i and the exchange X_i);
* network: layers h_1 = tanh(x W1 + b1), h_2 = tanh(h_1 W2 + b2), h_3 = tanh(h_2 W3 + b3),
  y = h_3 W4 + b4; loss = mean over samples and outputs of (y - t)^2; Adam;
* linear part: an FP64 ridge regression of the targets on the per-shell sums of the features
  (the network then fits what the linear part leaves); its normal equations are solved directly;
* estimator: with M cheap samples (features only) and n paired samples (features and the
  plain Sigma_i), the rows z_i = mean_j f(x_j) + Y_i - f(x_i) have mean
  mean_j f(x_j) + mean_i (Y_i - f(x_i)), which is unbiased for E[Y] whatever f is, and
  their spread gives the standard error; with f = 0 they are the plain samples.
"""
import numpy as np


def kset(m2max):
    """Integer wave vectors m, 0 < |m|^2 <= m2max, one of each +-m pair (first non-zero > 0)."""
    r = int(np.floor(np.sqrt(m2max)))
    out = []
    for a in range(-r, r + 1):
        for b in range(-r, r + 1):
            for c in range(-r, r + 1):
                m = (a, b, c)
                n2 = a * a + b * b + c * c
                if 0 < n2 <= m2max:
                    first = next(x for x in m if x != 0)
                    if first > 0:
                        out.append(m)
    return np.array(sorted(out, key=lambda m: (m[0] ** 2 + m[1] ** 2 + m[2] ** 2, m)), dtype=np.int64)


def coeffs(v, phi, n, h, m2max):
    """Coulomb-weighted coefficients sqrt(4 pi)/|k| F_v(k) on the k list, and F_v(0), by FFT.

    F_v(m) = dV sum_r v phi exp(-2 pi i (mx x + my y + mz z) / n); arrays indexed [z, y, x].
    """
    F = np.fft.fftn(v * phi) * h ** 3          # F[mz, my, mx]
    L = n * h
    ks = kset(m2max)
    c = np.array([F[mz % n, my % n, mx % n] * np.sqrt(4 * np.pi) / (2 * np.pi / L * np.sqrt(mx * mx + my * my + mz * mz))
                  for mx, my, mz in ks])
    return c, F[0, 0, 0].real


def coeffs_direct(v, phi, n, h, m2max):
    """Same coefficients by the plain DFT sum (no FFT), for pinning `coeffs` on tiny grids."""
    s = v * phi
    L = n * h
    idx = np.arange(n)
    Z, Y, X = np.meshgrid(idx, idx, idx, indexing='ij')
    c = []
    for mx, my, mz in kset(m2max):
        ph = np.exp(-2j * np.pi * (mx * X + my * Y + mz * Z) / n)
        c.append(h ** 3 * np.sum(s * ph) * np.sqrt(4 * np.pi) / (2 * np.pi / L * np.sqrt(mx * mx + my * my + mz * mz)))
    return np.array(c), h ** 3 * np.sum(s)


def features(zbar, etabars, phi, n, h, m2max):
    """[|F_zeta(k)|^2 ..., F_zeta(0)^2, sum_l |F_eta_l(k)|^2 ..., sum_l F_eta_l(0)^2]."""
    cz, z0 = coeffs(zbar, phi, n, h, m2max)
    ce = [coeffs(e, phi, n, h, m2max) for e in etabars]
    se = np.sum([np.abs(c) ** 2 for c, _ in ce], axis=0)
    s0 = np.sum([e0 ** 2 for _, e0 in ce])
    return np.concatenate([np.abs(cz) ** 2, [z0 ** 2], se, [s0]])


def feature_count(m2max):
    return 2 * (len(kset(m2max)) + 1)


# ---------------------------------------------------------------- network
def init_params(n_in, width, n_out, seed):
    """Uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) weights, zero biases (numpy generator)."""
    rng = np.random.default_rng(seed)
    dims = [n_in, width, width, width, n_out]
    p = []
    for i in range(4):
        a = 1.0 / np.sqrt(dims[i])
        p.append(rng.uniform(-a, a, size=(dims[i], dims[i + 1])))
        p.append(np.zeros(dims[i + 1]))
    return p


def forward(p, x):
    """Returns the output and the cache of pre-activations and activations."""
    acts = [x]
    pre = []
    a = x
    for i in range(4):
        z = a @ p[2 * i] + p[2 * i + 1]
        pre.append(z)
        a = np.tanh(z) if i < 3 else z
        acts.append(a)
    return a, (acts, pre)


def loss_and_grads(p, x, t, w=None):
    """Loss sum_o w_o (y - t)^2 / (M n_out) (w = 1 by default) and its gradients (backpropagation)."""
    y, (acts, pre) = forward(p, x)
    M, O = y.shape
    w = np.ones(O) if w is None else np.asarray(w, dtype=np.float64)
    loss = np.mean(w * (y - t) ** 2)
    d = 2.0 * w * (y - t) / (M * O)
    g = [None] * 8
    for i in reversed(range(4)):
        if i < 3:
            d = d * (1.0 - np.tanh(pre[i]) ** 2)
        g[2 * i] = acts[i].T @ d
        g[2 * i + 1] = d.sum(axis=0)
        d = d @ p[2 * i].T
    return loss, g


def adam_step(p, g, m, v, step, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba) in place; `step` counts from 1."""
    for i in range(len(p)):
        m[i] = b1 * m[i] + (1 - b1) * g[i]
        v[i] = b2 * v[i] + (1 - b2) * g[i] ** 2
        mh = m[i] / (1 - b1 ** step)
        vh = v[i] / (1 - b2 ** step)
        p[i] = p[i] - lr * mh / (np.sqrt(vh) + eps)


# ---------------------------------------------------------------- estimator
def standardize(a, mu=None, sd=None):
    """Column statistics (sample standard deviation; 1 where it is zero) and (a - mu) / sd."""
    if mu is None:
        mu = a.mean(axis=0)
        sd = a.std(axis=0, ddof=1) if a.shape[0] > 1 else np.zeros(a.shape[1])
        sd = np.where(sd > 0, sd, 1.0)
    return (a - mu) / sd, mu, sd


def cv_rows(f_cheap, f_paired, y_paired):
    """Rows z_i = mean_j f(x_j) + Y_i - f(x_i) (their mean is the control-variate estimate)."""
    return np.mean(f_cheap, axis=0)[None, :] + y_paired - f_paired


# ---------------------------------------------------------------- shell sums and the linear part
def shells(m2max):
    """Distinct |m|^2 values of the k list, increasing (the shells of the feature wave vectors)."""
    return sorted(set(int(v) for v in (kset(m2max) ** 2).sum(axis=1)))


def shell_count(m2max):
    return 2 * (len(shells(m2max)) + 1)


def shell_sums(feat, m2max):
    """Per-shell sums of the per-k features: [zeta shells..., zeta k=0, eta shells..., eta k=0]."""
    feat = np.atleast_2d(np.asarray(feat, dtype=np.float64))
    ks = kset(m2max)
    nk = len(ks)
    sh = (ks ** 2).sum(axis=1)
    out = []
    for base in (0, nk + 1):
        for s in shells(m2max):
            out.append(feat[:, base:base + nk][:, sh == s].sum(axis=1))
        out.append(feat[:, base + nk])
    return np.stack(out, axis=1)


def linear_fit(x, y, ridge):
    """Ridge regression of y on standardised x: returns (mu_x, sd_x, ybar, B) with
    (Xs^T Xs + ridge n I) B = Xs^T (y - ybar), Xs = (x - mu_x) / sd_x (sample sd; 1 where it is 0)."""
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    n, p = x.shape
    mu = x.mean(axis=0)
    sd = x.std(axis=0, ddof=1) if n > 1 else np.zeros(p)
    sd = np.where(sd > 0, sd, 1.0)
    xs = (x - mu) / sd
    ybar = y.mean(axis=0)
    B = np.linalg.solve(xs.T @ xs + ridge * n * np.eye(p), xs.T @ (y - ybar))
    return mu, sd, ybar, B


def linear_apply(model, x):
    mu, sd, ybar, B = model
    return ybar + ((np.asarray(x, dtype=np.float64) - mu) / sd) @ B
