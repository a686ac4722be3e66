"""The literal twiddle constants of the register DFTs used by the 288-point two-stage transforms
(fft288_2s.cuh: 16-point, 9-point and 18-point DFTs) against cos and sin of the angles they stand
for.  A mistyped digit would shift a twiddle by more than FP32 rounding; the GPU parity tests would
see it only as a larger error of the 288^3 transforms."""
import math
import os
import re

import pytest

SRC = os.path.join(os.path.dirname(__file__), '..', 'paper_2601_21005_gb300', 'csrc', 'fft288_2s.cuh')


def _body(src, name, nxt):
    # a definition is the name directly followed by its parameter list (calls carry <DIR>)
    return src[src.index(' %s(' % name):src.index(' %s(' % nxt) if nxt else None]


def _consts(body):
    return {m.group(1): float(m.group(2)) for m in re.finditer(r'\b([A-Z][0-9A-Z]*) = (-?[0-9.]+)f', body)}


@pytest.fixture(scope='module')
def src():
    with open(SRC) as f:
        return f.read()


def test_dft16_constants(src):
    c = _consts(_body(src, 'dft16', 'dft9'))
    assert c['C1'] == pytest.approx(math.cos(math.pi / 8), abs=1e-15)
    assert c['S1'] == pytest.approx(math.sin(math.pi / 8), abs=1e-15)
    assert c['R'] == pytest.approx(math.sqrt(0.5), abs=1e-15)


def test_dft9_constants(src):
    c = _consts(_body(src, 'dft9', 'dft18'))
    for k, (cn, sn) in {1: ('C1', 'S1'), 2: ('C2', 'S2'), 4: ('C4', 'S4')}.items():
        assert c[cn] == pytest.approx(math.cos(2 * math.pi * k / 9), abs=1e-15), cn
        assert c[sn] == pytest.approx(math.sin(2 * math.pi * k / 9), abs=1e-15), sn


def test_dft18_twiddles(src):
    body = _body(src, 'dft18', 'tw288')
    cb = [float(x) for x in re.findall(r'-?[0-9.]+(?=f)', body[body.index('CB[8]'):body.index('SB[8]')])]
    sb = [float(x) for x in re.findall(r'-?[0-9.]+(?=f)', body[body.index('SB[8]'):body.index('float2 e[9]')])]
    assert len(cb) == 8 and len(sb) == 8
    for b in range(1, 9):
        assert cb[b - 1] == pytest.approx(math.cos(2 * math.pi * b / 18), abs=1e-15), b
        assert sb[b - 1] == pytest.approx(math.sin(2 * math.pi * b / 18), abs=1e-15), b
