"""Launch tuning: the L2 prefetch hints and the autotuner change no result (bit-identical
propagation and TDH response under every setting), and bad keys or values are rejected."""
import numpy as np
import pytest

from paper_2601_21005_gb300 import build, synth

import gpu_common as gc

torch = pytest.importorskip('torch')
pytestmark = pytest.mark.gpu


def _ctx(s, mb):
    from paper_2601_21005_gb300 import sgw
    c = sgw.Context(s['n'], s['h'], max_batch=mb)
    c.set_potential(gc.to_dev(s['vloc'].ravel(), torch, torch.float32), s['kb_atoms'])
    c.set_spectrum(float(s['vloc'].min()) - 2.0, 0.5 * 3 * (np.pi / s['h']) ** 2 + 2.0)
    return c


def _run(c, s):
    ng = s['n'] ** 3
    x = torch.empty(8, ng, dtype=torch.complex64, device='cuda')
    c.white_noise(5, 2, 0, 1, 8, x)
    c.propagate(x, 2, 0.05, 16, np.array([1, -1] * 4, dtype=np.int8))
    phi = gc.to_dev(synth.smooth_orbital(s['n'], s['h'], (8.0, 8.0, 8.0)).ravel(), torch, torch.float32)
    src = (x[:2].real.contiguous() * phi).contiguous()
    uR = torch.empty(2, 4, ng, dtype=torch.float32, device='cuda')
    c.tdh_response(x[:4].contiguous(), src, 2, 2, 3, 0.05, 16, uR)
    torch.cuda.synchronize()
    return x, uR


def test_tuning_is_only_a_hint():
    assert torch.cuda.is_available()
    build.build()
    s = gc.small_cluster()
    c = _ctx(s, 16)
    assert [c.get_tuning(k) for k in range(c.TUNE_KEYS)] == [1, 0, 0, 0, 0]
    ref = _run(c, s)
    for setting in ((0, 0, 0, 0), (1, 7, 0, 1), (0, 0, 13, 0), (1, 100000, 100000, 1), (1, 0, 0, 2),
                    (0, 5, 9, 2)):
        for k, v in enumerate(setting):
            c.set_tuning(k, v)
        got = _run(c, s)
        assert torch.equal(got[0], ref[0]) and torch.equal(got[1], ref[1]), setting
    chosen = c.autotune(8, reps=1)
    assert len(chosen) == c.TUNE_KEYS and chosen[0] in (0, 1) and chosen[3] in (0, 1, 2) and min(chosen) >= 0
    assert chosen[4] == 0                    # the line form is tuned on the 288 grid only
    assert [c.get_tuning(k) for k in range(c.TUNE_KEYS)] == chosen
    got = _run(c, s)
    assert torch.equal(got[0], ref[0]) and torch.equal(got[1], ref[1])


def test_tuning_rejects_bad_keys_and_values():
    build.build()
    s = gc.small_cluster()
    c = _ctx(s, 4)
    for key, val in ((5, 0), (-1, 0), (0, 4), (1, -5), (2, -1), (3, 3), (4, 5), (4, -1)):
        with pytest.raises(RuntimeError):
            c.set_tuning(key, val)
    with pytest.raises(RuntimeError):
        c.autotune(5)                        # above max_batch
    # a buffer that is not 16-byte aligned is refused before any launch
    ng = s['n'] ** 3
    raw = torch.empty(ng * 4 + 1, dtype=torch.complex64, device='cuda')
    bad = raw[1:1 + ng]                       # 8-byte offset
    with pytest.raises(RuntimeError):
        c.propagate(bad, 1, 0.05, 4)
