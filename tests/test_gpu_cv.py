"""GPU control variate against the oracle: network forward/backward/Adam (BF16 tensor-core
GEMMs with FP32 accumulation vs FP64), features, and the estimator's identities.

Tolerances: each GEMM rounds its operands to BF16 (unit roundoff 2^-8).  Outputs and gradients
are compared norm-wise per tensor (2e-2 / 5e-2) and element by element against a first-order
rounding bound computed from the oracle's FP64 pass; Adam and the FP64 estimator, given identical
inputs, at 1e-6."""
import numpy as np
import pytest

from oracle import hamiltonian as ham
from oracle import mlp as omlp
from oracle import sgw as osgw
from paper_2601_21005_gb300 import build, synth

import gpu_common as gc

torch = pytest.importorskip('torch')
pytestmark = pytest.mark.gpu


@pytest.fixture(scope='module', autouse=True)
def _built():
    assert torch.cuda.is_available()
    build.build()


def _sgw():
    from paper_2601_21005_gb300 import sgw
    return sgw


def _flat(p):
    return np.concatenate([a.reshape(-1) for a in p]).astype(np.float32)


def _unflat(flat, like):
    out, o = [], 0
    for a in like:
        out.append(flat[o:o + a.size].reshape(a.shape).astype(np.float64))
        o += a.size
    return out


def _nrel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / max(np.linalg.norm(np.ravel(b)), 1e-30))


def test_mlp_forward_and_gradients_match_oracle():
    n_in, H, O, M = 37, 72, 50, 45          # not multiples of the 64 x 64 x 32 GEMM tiles
    p = omlp.init_params(n_in, H, O, seed=3)
    for i in range(1, 8, 2):
        p[i] = 0.1 * np.random.default_rng(i).normal(size=p[i].shape)
    flat = _flat(p)
    p32 = _unflat(flat, p)
    net = _sgw().MLP(n_in, H, O, 64)
    net.set_params(flat)
    rng = np.random.default_rng(4)
    x = rng.normal(size=(M, n_in)).astype(np.float32)
    t = rng.normal(size=(M, O)).astype(np.float32)
    xd, td = gc.to_dev(x, torch, torch.float32), gc.to_dev(t, torch, torch.float32)
    y = torch.empty(M, O, dtype=torch.float32, device='cuda')
    net.forward(xd, y)
    yo, _ = omlp.forward(p32, x.astype(np.float64))
    assert _nrel(y.cpu().numpy(), yo) < 2e-2
    wts = rng.uniform(0.5, 3.0, size=O).astype(np.float32)
    net.set_loss_weights(wts)
    loss, g = net.gradients(xd, td, want_grads=True)
    lo, go = omlp.loss_and_grads(p32, x.astype(np.float64), t.astype(np.float64), wts.astype(np.float64))
    assert abs(loss - lo) < 2e-2 * lo
    gg = _unflat(g, p)
    for i in range(8):
        assert _nrel(gg[i], go[i]) < 5e-2, i
    assert np.array_equal(net.get_params(), flat)


def _bf16_error_bounds(p, x, t, w, u=2.0 ** -8):
    """First-order bounds, element by element, on the difference between the GPU network (every
    GEMM operand rounded to BF16, unit roundoff u = 2^-8; FP32 accumulation, biases, pre-activations,
    tanh and the output kept in FP32) and the FP64 oracle at the same parameters.

    A product C = A B of perturbed operands |A^ - A| <= E_A, |B^ - B| <= E_B is off by at most
    E_A |B| + |A| E_B (first order); rounding an operand to BF16 adds u |operand| to its E.  The
    rules run through the forward pass and backpropagation exactly as the oracle's layers do.
    Returns (bound on y, bounds on the 8 gradient tensors)."""
    _, (acts, pre) = omlp.forward(p, x)
    M = x.shape[0]
    O = p[-1].shape[0]
    W = [np.abs(p[2 * i]) for i in range(4)]
    E_a = [u * np.abs(x)]                         # x rounded to BF16 for the first GEMM
    E_z = []
    for i in range(4):
        a = np.abs(acts[i])
        ez = E_a[i] @ W[i] + u * a @ W[i]           # operand errors, plus rounding of W_i
        E_z.append(ez)
        if i < 3:
            sech2 = 1.0 - np.tanh(pre[i]) ** 2
            E_a.append(sech2 * ez + u * np.abs(acts[i + 1]))     # tanh stored as BF16
    E_y = E_z[3]
    y = acts[4]
    d = 2.0 * w * (y - t) / (M * O)
    E_d = 2.0 * w * E_y / (M * O) + u * np.abs(d)                # dY rounded to BF16
    G = [None] * 8
    for i in reversed(range(4)):
        a = np.abs(acts[i])
        G[2 * i] = E_a[i].T @ np.abs(d) + a.T @ E_d
        G[2 * i + 1] = E_d.sum(axis=0)
        if i == 0:
            break
        da = np.abs(d) @ W[i].T
        E_da = E_d @ W[i].T + u * np.abs(d) @ W[i].T
        th = np.tanh(pre[i - 1])
        sech2 = 1.0 - th ** 2
        E_dz = E_da * sech2 + da * 2.0 * np.abs(th) * sech2 * E_z[i - 1]
        d = (d @ p[2 * i].T) * sech2
        E_d = E_dz + u * np.abs(d)                               # dZ rounded to BF16
    return E_y, G


def test_mlp_outputs_and_gradients_elementwise_within_bf16_bound():
    """Every output and every gradient element within twice its first-order BF16 rounding bound
    (the bound is computed from the oracle's own FP64 pass: see _bf16_error_bounds)."""
    n_in, H, O, M = 37, 72, 50, 45
    p = omlp.init_params(n_in, H, O, seed=13)
    for i in range(1, 8, 2):
        p[i] = 0.1 * np.random.default_rng(20 + i).normal(size=p[i].shape)
    flat = _flat(p)
    p32 = _unflat(flat, p)
    net = _sgw().MLP(n_in, H, O, 64)
    net.set_params(flat)
    rng = np.random.default_rng(14)
    x = rng.normal(size=(M, n_in)).astype(np.float32)
    t = rng.normal(size=(M, O)).astype(np.float32)
    wts = rng.uniform(0.5, 3.0, size=O).astype(np.float32)
    xd, td = gc.to_dev(x, torch, torch.float32), gc.to_dev(t, torch, torch.float32)
    y = torch.empty(M, O, dtype=torch.float32, device='cuda')
    net.forward(xd, y)
    net.set_loss_weights(wts)
    _, g = net.gradients(xd, td, want_grads=True)
    x64, t64, w64 = x.astype(np.float64), t.astype(np.float64), wts.astype(np.float64)
    yo, _ = omlp.forward(p32, x64)
    _, go = omlp.loss_and_grads(p32, x64, t64, w64)
    E_y, E_g = _bf16_error_bounds(p32, x64, t64, w64)
    tiny = 1e-7                                   # FP32 rounding of the outputs themselves
    err_y = np.abs(y.cpu().numpy() - yo)
    assert np.all(err_y <= 2.0 * E_y + tiny * np.abs(yo) + 1e-12), np.max(err_y / (E_y + 1e-30))
    gg = _unflat(g, p)
    ratios = []
    for i in range(8):
        err = np.abs(gg[i] - go[i])
        bound = 2.0 * E_g[i] + tiny * np.abs(go[i]) + 1e-12
        assert np.all(err <= bound), (i, float(np.max(err / bound)))
        ratios.append(float(np.max(err / bound)))
    print('largest error / bound: outputs %.3f, gradients %s' % (float(np.max(err_y / (2 * E_y + 1e-30))),
                                                                   ['%.3f' % r for r in ratios]))


def test_adam_step_matches_oracle_update():
    n_in, H, O, M = 20, 64, 30, 33
    p = omlp.init_params(n_in, H, O, seed=5)
    flat = _flat(p)
    net = _sgw().MLP(n_in, H, O, 64)
    net.set_params(flat)
    rng = np.random.default_rng(6)
    x = gc.to_dev(rng.normal(size=(M, n_in)), torch, torch.float32)
    t = gc.to_dev(rng.normal(size=(M, O)), torch, torch.float32)
    pp = _unflat(flat, p)
    m = [np.zeros_like(a) for a in pp]
    v = [np.zeros_like(a) for a in pp]
    for step in (1, 2):
        _, g = net.gradients(x, t, want_grads=True)
        net.adam_step(1e-3)
        omlp.adam_step(pp, _unflat(g, p), m, v, step, 1e-3)
        got = _unflat(net.get_params(), p)
        for i in range(8):
            assert np.max(np.abs(got[i] - pp[i])) < 1e-6 + 1e-5 * np.max(np.abs(pp[i]))


def test_training_fits_a_quadratic_form():
    rng = np.random.default_rng(7)
    n_in, O, M = 16, 8, 512
    A = rng.normal(size=(O, n_in, n_in)) / n_in
    x = rng.normal(size=(M, n_in))
    t = np.einsum('mi,oij,mj->mo', x, A, x)
    t = (t - t.mean(0)) / t.std(0)
    net = _sgw().MLP(n_in, 128, O, 64, seed=1)
    xd, td = gc.to_dev(x, torch, torch.float32), gc.to_dev(t, torch, torch.float32)
    l0 = net.train_epoch(xd, td, 64, 2e-3)
    for _ in range(150):
        l1 = net.train_epoch(xd, td, 64, 2e-3)
    assert l1 < 0.15 * l0


def test_cv_features_match_oracle():
    s = synth.wells()
    g = ham.Grid(s['n'], s['h'])
    sg = _sgw()
    ctx = sg.Context(s['n'], s['h'], max_batch=8)
    n_eta, ns = 3, 3                      # 3 samples x 4 vectors: two chunks of max_batch 8 (ragged)
    noise = torch.empty(ns * (n_eta + 1), g.ng, dtype=torch.complex64, device='cuda')
    ctx.white_noise(11, 1, 4, ns, n_eta + 1, noise)
    phi = synth.smooth_orbital(g.n, g.h, (4.8, 4.8, 4.8)).astype(np.float32)
    nf = sg.sgw_cv_feature_count(10)
    assert nf == omlp.feature_count(10)
    feat = torch.empty(ns, nf, dtype=torch.float32, device='cuda')
    ctx.cv_features(noise, ns, n_eta + 1, gc.to_dev(phi.ravel(), torch, torch.float32), 10, feat)
    for i in range(ns):
        v = osgw.white_noise(g, 11, 1, 4 + i, n_eta + 1)
        ref = omlp.features(v[0], v[1:], phi.astype(np.float64), g.n, g.h, 10)
        assert gc.rel_err(feat[i].cpu().numpy(), ref) < 1e-5


def test_cv_rows_identities_and_formula():
    sg = _sgw()
    s = synth.wells()
    ctx = sg.Context(s['n'], s['h'], max_batch=2)
    rng = np.random.default_rng(8)
    n, Mc, O = 7, 11, 12
    Y = gc.to_dev(rng.normal(size=(n, O)), torch, torch.float64)
    rows = torch.empty_like(Y)
    ctx.cv_rows(None, None, Y, None, None, rows)
    assert torch.equal(rows, Y)                                   # f = 0: the plain samples
    fc = rng.normal(size=(Mc, O)).astype(np.float32)
    fp = rng.normal(size=(n, O)).astype(np.float32)
    mu, sd = rng.normal(size=O), 1 + rng.random(O)
    ctx.cv_rows(gc.to_dev(fc, torch, torch.float32), gc.to_dev(fp, torch, torch.float32), Y,
                gc.to_dev(mu, torch, torch.float64), gc.to_dev(sd, torch, torch.float64), rows)
    ref = omlp.cv_rows(mu + sd * fc.astype(np.float64), mu + sd * fp.astype(np.float64), Y.cpu().numpy())
    assert np.max(np.abs(rows.cpu().numpy() - ref)) < 1e-12 * np.max(np.abs(ref))
    # standardisation
    T = torch.empty(n, O, dtype=torch.float32, device='cuda')
    mud = torch.empty(O, dtype=torch.float64, device='cuda')
    sdd = torch.empty(O, dtype=torch.float64, device='cuda')
    ctx.cv_standardize(Y, mud, sdd, T, True)
    yn = Y.cpu().numpy()
    assert np.allclose(mud.cpu().numpy(), yn.mean(0), atol=1e-14)
    assert np.allclose(sdd.cpu().numpy(), yn.std(0, ddof=1), atol=1e-14)
    assert np.allclose(T.cpu().numpy(), (yn - yn.mean(0)) / yn.std(0, ddof=1), atol=1e-6)
    # float columns, in place, with given statistics
    Xf = gc.to_dev(rng.normal(size=(n, O)), torch, torch.float32)
    x0 = Xf.cpu().numpy().astype(np.float64)
    ctx.cv_standardize_f32(Xf, mud, sdd, False)
    assert np.allclose(Xf.cpu().numpy(), (x0 - yn.mean(0)) / yn.std(0, ddof=1), atol=1e-5)


def test_control_variate_gain_tiny():
    """16^3 wells, 8 eta pairs, 200 steps: train on 1024 plain samples, then compare the plain
    and the control-variate QP energies on 256 paired samples (+ 8192 cheap ones)."""
    from paper_2601_21005_gb300.control_variate import ControlVariate
    from paper_2601_21005_gb300.pipeline import Pipeline
    s = synth.wells()
    g, kb, w, phis = gc.oracle_eigs(s, 8)
    pl = Pipeline(s['n'], s['h'], s['vloc'], [], phis[3], w[3], w[4], n_eta=8, n_steps=200, dt=0.05,
                  cheb_deg=16, n_cheb=128, samples_per_batch=8, seed=3000, stream_id=1)
    cv = ControlVariate(pl, m2max=10, width=256, max_batch=256, seed=5)
    Yt, Ft = cv.collect(1024, 0)
    tr, va = cv.train(Ft, Yt, epochs=200, batch=64, lr=1e-3, eps_ks=w[3])
    assert min(va) < va[0]
    assert cv.linear_used                    # the linear part passes its hold-out test here
    Yp, Fp = cv.collect(256, 100000)
    Fc = cv.cheap_features(8192, 200000)
    S0, X0 = cv.plain_rows(Yp)
    S1, X1 = cv.rows(Fc, Fp, Yp)
    plain = pl.qp(S0, X0, w[3])
    cvr = pl.qp(S1, X1, w[3])
    gain = (plain['se'] / cvr['se']) ** 2
    # the same rows with the linear part alone: what the trained network adds on top of it
    net_kept = cv.use_net
    cv.use_net = False
    S2, X2 = cv.rows(Fc, Fp, Yp)
    cv.use_net = net_kept
    lin = pl.qp(S2, X2, w[3])
    gain_lin = (plain['se'] / lin['se']) ** 2
    print('control-variate gain (variance ratio) %.2f (linear part alone %.2f, network kept: %s), '
          'QP plain %.4f +- %.4f eV, CV %.4f +- %.4f eV' % (
              gain, gain_lin, net_kept, plain['eps_qp'] * 27.2114, plain['se'] * 27.2114,
              cvr['eps_qp'] * 27.2114, cvr['se'] * 27.2114))
    assert abs(cvr['eps_qp'] - plain['eps_qp']) < 4 * plain['se']
    assert gain > 1.5
    # what the trained network adds on top of the linear part: when it is dropped the rows are
    # those of the linear part, bit for bit; when it is kept it must not lose against it (the
    # gain measured here is about 2.15 either way: the predictable part is linear in the features)
    if net_kept:
        assert gain >= 0.95 * gain_lin
    else:
        assert gain == gain_lin
    # no cheap samples: the rows are the plain samples, bit for bit
    S2, X2 = cv.rows(None, None, Yp)
    assert torch.equal(S2, S0) and torch.equal(X2, X0)


def test_cv_shell_sums_and_linear_part_match_oracle():
    sg = _sgw()
    s = synth.wells()
    ctx = sg.Context(s['n'], s['h'], max_batch=2)
    rng = np.random.default_rng(12)
    m2 = 10
    nk, ns = sg.sgw_cv_feature_count(m2), sg.sgw_cv_shell_count(m2)
    assert ns == omlp.shell_count(m2)
    fk = rng.random(size=(9, nk)).astype(np.float32)
    out = torch.empty(9, ns, dtype=torch.float32, device='cuda')
    ctx.cv_shell_sums(gc.to_dev(fk, torch, torch.float32), m2, out)
    assert np.allclose(out.cpu().numpy(), omlp.shell_sums(fk.astype(np.float64), m2), rtol=1e-6)
    # ridge fit, prediction, residuals and rows against the FP64 oracle on the same float inputs
    n, p, o, mc = 57, ns, 13, 40
    x = (rng.normal(size=(n, p)) * rng.uniform(0.1, 10, size=p) + rng.normal(size=p)).astype(np.float32)
    y = x.astype(np.float64) @ rng.normal(size=(p, o)) + 0.3 * rng.normal(size=(n, o))
    xd, yd = gc.to_dev(x, torch, torch.float32), gc.to_dev(y, torch, torch.float64)
    model = torch.zeros(sg.sgw_cv_linear_size(p, o), dtype=torch.float64, device='cuda')
    ctx.cv_linear_fit(xd, yd, 1e-3, model)
    mu, sd, ybar, B = omlp.linear_fit(x.astype(np.float64), y, 1e-3)
    m = model.cpu().numpy()
    assert np.allclose(m[:p], mu, rtol=1e-12) and np.allclose(m[p:2 * p], sd, rtol=1e-12)
    assert np.allclose(m[2 * p:2 * p + o], ybar, rtol=1e-12)
    assert np.max(np.abs(m[2 * p + o:].reshape(p, o) - B)) < 1e-9 * np.max(np.abs(B))
    f = torch.empty(n, o, dtype=torch.float64, device='cuda')
    ctx.cv_linear_apply(model, xd, o, f)
    ref = omlp.linear_apply((mu, sd, ybar, B), x.astype(np.float64))
    assert np.max(np.abs(f.cpu().numpy() - ref)) < 1e-9 * np.max(np.abs(ref))
    r = torch.empty_like(f)
    ctx.cv_linear_apply(model, xd, o, r, y=yd)
    assert np.max(np.abs(r.cpu().numpy() - (y - ref))) < 1e-9 * np.max(np.abs(ref))
    xc = rng.normal(size=(mc, p)).astype(np.float32) * x.std(0) + x.mean(0)
    rows = torch.empty_like(yd)
    ctx.cv_linear_rows(model, gc.to_dev(xc, torch, torch.float32), xd, yd, rows)
    model_np = (mu, sd, ybar, B)
    want = omlp.cv_rows(omlp.linear_apply(model_np, xc.astype(np.float64)), ref, y)
    assert np.max(np.abs(rows.cpu().numpy() - want)) < 1e-9 * np.max(np.abs(want))
    # a fit needs at least two samples
    with pytest.raises(RuntimeError):
        ctx.cv_linear_fit(xd[:1], yd[:1], 1e-3, model)
