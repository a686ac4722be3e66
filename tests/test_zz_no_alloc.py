"""The QP solve that allocates nothing (sgw_qp_energy_noalloc), for callers that cannot let the
library allocate device memory, against the context-based sgw_qp_energy on the same inputs.
Collected last on purpose: it must pass both alone in a fresh process and after every other
test, and the static scratch it uses keeps the previous call's contents."""
import numpy as np
import pytest

from paper_2601_21005_gb300 import build, synth

torch = pytest.importorskip('torch')
pytestmark = pytest.mark.gpu


def _sigma(n_s, N, dt, seed):
    r = np.random.default_rng(seed)
    t = dt * np.arange(-N, N + 1)
    rows = []
    for _ in range(n_s):
        a = 0.02 * (1 + 0.3 * r.normal())
        e1, e2 = -0.4 + 0.02 * r.normal(), 0.3 + 0.02 * r.normal()
        rows.append(-1j * a * np.exp(-1j * e2 * t) * (t > 0) + 1j * a * np.exp(-1j * e1 * t) * (t < 0))
    return np.array(rows), -0.05 + 0.01 * r.normal(size=n_s)


def test_noalloc_qp_matches_context_qp_twice():
    assert torch.cuda.is_available()
    build.build()
    from paper_2601_21005_gb300 import sgw
    s = synth.wells()
    ctx = sgw.Context(s['n'], s['h'], max_batch=2)
    dt, N = 0.05, 200
    gamma = 3.0 / (N * dt)
    for call, (n_s, seed) in enumerate(((6, 31), (9, 32))):          # two calls in a row
        S, X = _sigma(n_s, N, dt, seed)
        sd = torch.from_numpy(S).cuda()
        xd = torch.from_numpy(X).cuda()
        ref = ctx.qp_energy(sd, xd, n_s, N, dt, gamma, -0.25)
        got = sgw.sgw_qp_energy_noalloc(sd, xd, n_s, N, dt, gamma, -0.25)
        for k in ('eps_qp', 'se', 're_sigma', 'z'):
            assert abs(got[k] - ref[k]) <= 1e-10 * max(1.0, abs(ref[k])), (call, k)
    # the largest request that fits: n_scan = 2 w/s + 1 = 130265 (130266 rounded to even) +
    # 2 (2 N + 1) + 4 = 131072 doubles, exactly the scratch size
    w_max = 65.132
    ref = ctx.qp_energy(sd, xd, n_s, N, dt, gamma, -0.25, window=w_max)
    got = sgw.sgw_qp_energy_noalloc(sd, xd, n_s, N, dt, gamma, -0.25, window=w_max)
    for k in ('eps_qp', 'se', 're_sigma', 'z'):
        assert abs(got[k] - ref[k]) <= 1e-10 * max(1.0, abs(ref[k])), k
    # sizes beyond the static scratch are rejected with a clear error, before any launch: one
    # scan point too many, a large window, and a window/step ratio that overflows any integer
    for window, step in ((65.133, 1e-3), (200.0, 1e-3), (1e300, 1e-300)):
        with pytest.raises(sgw.SgwError) as ei:
            sgw.sgw_qp_energy_noalloc(sd, xd, n_s, N, dt, gamma, -0.25, window=window, step=step)
        assert 'static' in str(ei.value), (window, step)
    # the array is still usable afterwards
    got = sgw.sgw_qp_energy_noalloc(sd, xd, n_s, N, dt, gamma, -0.25)
    ref = ctx.qp_energy(sd, xd, n_s, N, dt, gamma, -0.25)
    assert abs(got['eps_qp'] - ref['eps_qp']) <= 1e-10 * max(1.0, abs(ref['eps_qp']))
