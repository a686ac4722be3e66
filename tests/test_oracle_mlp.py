"""Pins of the oracle's control variate: features against the plain DFT definition,
backpropagation against central finite differences, Adam against its closed form on a
quadratic, and the estimator's identities (no GPU)."""
import numpy as np
import pytest

from oracle import mlp


def test_kset_half_space_and_shells():
    ks = mlp.kset(10)
    assert len(ks) == len({tuple(k) for k in ks})
    assert all(0 < (k ** 2).sum() <= 10 for k in ks)
    full = {tuple(k) for k in ks} | {tuple(-k) for k in ks}
    # every nonzero m with |m|^2 <= 10 appears exactly once up to sign
    r = 3
    cnt = sum(1 for a in range(-r, r + 1) for b in range(-r, r + 1) for c in range(-r, r + 1)
              if 0 < a * a + b * b + c * c <= 10)
    assert len(full) == cnt == 2 * len(ks)


def test_coefficients_match_direct_dft():
    n, h = 8, 0.7
    rng = np.random.default_rng(0)
    zb = rng.choice([-1.0, 1.0], size=(n, n, n)) / np.sqrt(h ** 3)
    phi = rng.normal(size=(n, n, n))
    a, a0 = mlp.coeffs(zb, phi, n, h, 5)
    b, b0 = mlp.coeffs_direct(zb, phi, n, h, 5)
    assert np.max(np.abs(a - b)) < 1e-10 * np.max(np.abs(b))
    assert abs(a0 - b0) < 1e-10 * abs(b0)


def test_features_layout():
    n, h = 8, 0.7
    rng = np.random.default_rng(1)
    v = [rng.choice([-1.0, 1.0], size=(n, n, n)) for _ in range(4)]
    phi = rng.normal(size=(n, n, n))
    f = mlp.features(v[0], v[1:], phi, n, h, 5)
    nk = len(mlp.kset(5))
    assert len(f) == mlp.feature_count(5) == 2 * (nk + 1)
    c0, z0 = mlp.coeffs_direct(v[0], phi, n, h, 5)
    assert np.allclose(f[:nk], np.abs(c0) ** 2) and np.isclose(f[nk], z0 ** 2)
    ce = [mlp.coeffs_direct(e, phi, n, h, 5) for e in v[1:]]
    assert np.allclose(f[nk + 1:2 * nk + 1], sum(np.abs(c) ** 2 for c, _ in ce))
    assert np.isclose(f[-1], sum(e0 ** 2 for _, e0 in ce))


def test_backprop_matches_finite_differences():
    rng = np.random.default_rng(1)
    p = mlp.init_params(7, 9, 5, seed=2)
    x = rng.normal(size=(6, 7))
    t = rng.normal(size=(6, 5))
    wts = rng.uniform(0.5, 3.0, size=5)
    loss, g = mlp.loss_and_grads(p, x, t, wts)
    eps = 1e-6
    for i in range(8):
        flat = p[i].reshape(-1)
        for j in rng.choice(flat.size, size=min(5, flat.size), replace=False):
            old = flat[j]
            flat[j] = old + eps
            lp, _ = mlp.loss_and_grads(p, x, t, wts)
            flat[j] = old - eps
            lm, _ = mlp.loss_and_grads(p, x, t, wts)
            flat[j] = old
            fd = (lp - lm) / (2 * eps)
            assert abs(g[i].reshape(-1)[j] - fd) < 1e-6 * max(1.0, abs(fd)) + 1e-9


def test_adam_first_step_is_signed_lr():
    """Bias correction makes the first Adam step -lr * g / (|g| + eps') elementwise."""
    p = [np.array([1.0, -2.0, 3.0])]
    g = [np.array([0.5, -4.0, 1e-3])]
    m = [np.zeros(3)]
    v = [np.zeros(3)]
    mlp.adam_step(p, g, m, v, 1, lr=0.01)
    want = np.array([1.0, -2.0, 3.0]) - 0.01 * g[0] / (np.abs(g[0]) + 1e-8)
    assert np.allclose(p[0], want, atol=1e-12)


def test_adam_minimises_a_quadratic():
    p = [np.array([3.0, -1.0])]
    m, v = [np.zeros(2)], [np.zeros(2)]
    for s in range(1, 3001):
        mlp.adam_step(p, [2 * (p[0] - np.array([0.5, 0.25]))], m, v, s, lr=0.01)
    assert np.allclose(p[0], [0.5, 0.25], atol=1e-3)


def test_cv_rows_identities():
    rng = np.random.default_rng(3)
    Y = rng.normal(size=(20, 4))
    assert np.array_equal(mlp.cv_rows(np.zeros((50, 4)), np.zeros((20, 4)), Y), Y)
    # with a perfect predictor the rows are the mean of the cheap predictions
    f = Y.copy()
    rows = mlp.cv_rows(Y, f, Y)
    assert np.allclose(rows, Y.mean(axis=0))


def test_cv_estimator_unbiased_and_variance_reduced():
    """Y = q(x) + e with a predictor f ~ q: the CV mean equals E[Y] within its SE and its
    per-row spread is that of Y - f."""
    rng = np.random.default_rng(4)
    q = lambda x: (x ** 2).sum(axis=1, keepdims=True)
    est, ses, plain_se = [], [], []
    for rep in range(200):
        xc = rng.normal(size=(400, 3))
        xp = rng.normal(size=(20, 3))
        y = q(xp) + 0.3 * rng.normal(size=(20, 1))
        f = lambda x: 0.9 * q(x)
        rows = mlp.cv_rows(f(xc), f(xp), y)
        est.append(rows.mean())
        ses.append(rows.std(ddof=1) / np.sqrt(20))
        plain_se.append(y.std(ddof=1) / np.sqrt(20))
    est = np.array(est)
    # E[Y] = 3; the spread of the estimates matches the SE of Y - f plus Var(f)/M
    assert abs(est.mean() - 3.0) < 4 * est.std() / np.sqrt(len(est))
    assert np.mean(ses) < 0.5 * np.mean(plain_se)


def test_shell_sums_by_hand():
    # m2max = 3: shells 1 (3 vectors), 2 (6), 3 (4) -> 13 wave vectors, 8 shell features
    assert mlp.shells(3) == [1, 2, 3]
    assert mlp.shell_count(3) == 8
    nk = len(mlp.kset(3))
    assert nk == 13
    f = np.arange(2 * (nk + 1), dtype=np.float64)[None, :] + 1.0
    s = mlp.shell_sums(f, 3)[0]
    # zeta block: entries 1..13 in shell order 3 x |m|^2=1, 6 x 2, 4 x 3, then k=0 entry 14
    assert s[0] == 1 + 2 + 3 and s[1] == sum(range(4, 10)) and s[2] == sum(range(10, 14)) and s[3] == 14
    assert s[4] == 15 + 16 + 17 and s[7] == 28
    assert np.isclose(s.sum(), f.sum())                # every feature lands in exactly one sum


def test_linear_fit_recovers_an_exact_linear_map():
    rng = np.random.default_rng(5)
    x = rng.normal(size=(40, 3)) * np.array([1.0, 10.0, 0.1]) + np.array([2.0, -1.0, 5.0])
    A = rng.normal(size=(3, 4))
    a0 = rng.normal(size=4)
    y = a0 + x @ A
    model = mlp.linear_fit(x, y, 0.0)
    xt = rng.normal(size=(7, 3))
    assert np.allclose(mlp.linear_apply(model, xt), a0 + xt @ A, atol=1e-10)


def test_linear_fit_normal_equations_and_shrinkage():
    rng = np.random.default_rng(6)
    x = rng.normal(size=(30, 4))
    y = rng.normal(size=(30, 2))
    lam = 0.3
    mu, sd, ybar, B = mlp.linear_fit(x, y, lam)
    xs = (x - mu) / sd
    # stationarity of sum |y - ybar - xs B|^2 + lam n |B|^2, written out independently
    grad = -2 * xs.T @ (y - ybar - xs @ B) + 2 * lam * len(x) * B
    assert np.max(np.abs(grad)) < 1e-10
    assert np.allclose(xs.mean(0), 0, atol=1e-12) and np.allclose(xs.std(0, ddof=1), 1)
    # stronger ridge shrinks the coefficients
    assert np.linalg.norm(mlp.linear_fit(x, y, 10 * lam)[3]) < np.linalg.norm(B)
