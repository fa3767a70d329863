"""Pins of oracle.formats: rounding against torch's casts and Table 1's unit roundoffs."""
import numpy as np
import pytest
import torch

from oracle.formats import round_to, UNIT_ROUNDOFF, XMAX
from conftest import read_golden


def _all_patterns(dtype):
    bits = torch.arange(0, 1 << 16, dtype=torch.int32).to(torch.int16)
    vals = bits.view(dtype).double().numpy()
    return vals[np.isfinite(vals)]


@pytest.mark.parametrize("fmt,dtype", [("fp16", torch.float16), ("bf16", torch.bfloat16)])
def test_every_pattern_and_midpoint(fmt, dtype):
    v = np.unique(_all_patterns(dtype))
    # representable values are fixed points
    assert np.array_equal(round_to(v, fmt), v)
    # midpoints between neighbours: ties to even, compared with torch's direct FP64 -> fmt cast
    mid = (v[:-1] + v[1:]) / 2
    ref = torch.from_numpy(mid).to(dtype).double().numpy()
    assert np.array_equal(round_to(mid, fmt), ref)
    # points a quarter of the way between neighbours
    q = v[:-1] + (v[1:] - v[:-1]) / 4
    assert np.array_equal(round_to(q, fmt), torch.from_numpy(q).to(dtype).double().numpy())


def test_random_doubles():
    """Single rounding from FP64: numpy's float16 cast is direct (torch's goes through fp32,
    a double rounding that differs at fp16 midpoints); bf16 is checked on FP32-representable
    inputs, where torch's cast is a single rounding."""
    rng = np.random.default_rng(1)
    x = rng.standard_normal(200000) * np.exp(rng.uniform(-30, 30, 200000))
    with np.errstate(over="ignore"):
        assert np.array_equal(round_to(x, "fp16"), x.astype(np.float16).astype(np.float64))
    assert np.array_equal(round_to(x, "fp32"), torch.from_numpy(x).float().double().numpy())
    x32 = x.astype(np.float32).astype(np.float64)
    assert np.array_equal(round_to(x32, "bf16"), torch.from_numpy(x32).to(torch.bfloat16).double().numpy())


def test_e4m3_in_range():
    rng = np.random.default_rng(2)
    x = rng.uniform(-463.9, 463.9, 100000)
    x = np.concatenate([x, rng.standard_normal(10000) * 1e-3, [0.0, 448.0, -448.0, 464.0, 2.0 ** -9, 2.0 ** -10]])
    ref = torch.from_numpy(x).to(torch.float8_e4m3fn).double().numpy()
    assert np.array_equal(round_to(x, "e4m3"), ref)
    # beyond the largest finite value the oracle saturates (torch gives NaN there)
    assert round_to(np.array([500.0, -1e6]), "e4m3").tolist() == [448.0, -448.0]


def test_overflow_and_subnormals():
    assert np.isinf(round_to(np.array([65520.0]), "fp16"))[0]
    assert round_to(np.array([65519.0]), "fp16")[0] == 65504.0
    assert round_to(np.array([2.0 ** -24]), "fp16")[0] == 2.0 ** -24       # smallest subnormal
    assert round_to(np.array([2.0 ** -26]), "fp16")[0] == 0.0
    assert XMAX["fp16"] == 65504.0


def test_table1_unit_roundoffs():
    for name, val in read_golden("table1_unit_roundoff.txt"):
        assert abs(UNIT_ROUNDOFF[name] - float(val)) <= 0.005 * float(val), name
    # unit roundoff is half the gap from 1 to the next number: fl(1 + u) rounds to 1 (tie to even)
    for fmt in ("fp16", "bf16", "fp32"):
        u = UNIT_ROUNDOFF[fmt]
        assert round_to(np.array([1.0 + u]), fmt)[0] == 1.0
        assert round_to(np.array([1.0 + 3 * u]), fmt)[0] == 1.0 + 4 * u
