"""Rounding of FP64 values to the low-precision formats used by the method.

Section 3 simulates half precision by rounding every result to fp16
("chop"); Table 1 lists the unit roundoffs of the IEEE formats. The function
``round_to`` implements round-to-nearest-even into a binary format with t
significand bits (including the implicit bit), minimum normal exponent emin and
largest finite value xmax, with gradual underflow. Overflow gives +-inf for the
IEEE formats and saturates to +-xmax for fp8-e4m3 (OCP E4M3FN has no infinity;
the saturating conversion is the one the GPU uses).

Pinned by tests/test_oracle_formats.py against torch's casts (every fp16/bf16
bit pattern and its midpoints, random doubles, e4m3 below the overflow point).
"""
from __future__ import annotations

import numpy as np

# name: (t, emin, xmax, saturate)
FORMATS = {
    "fp32": (24, -126, (2.0 - 2.0 ** -23) * 2.0 ** 127, False),
    "fp16": (11, -14, 65504.0, False),
    "bf16": (8, -126, (2.0 - 2.0 ** -7) * 2.0 ** 127, False),
    "e4m3": (4, -6, 448.0, True),
}

# Unit roundoff u = 2^-t of each format (Table 1 lists fp16, fp32, fp64 and fp128).
UNIT_ROUNDOFF = {
    "fp16": 2.0 ** -11,
    "bf16": 2.0 ** -8,
    "e4m3": 2.0 ** -4,
    "fp32": 2.0 ** -24,
    "fp64": 2.0 ** -53,
    "dd": 2.0 ** -106,
    "fp128": 2.0 ** -113,
}

XMAX = {k: v[2] for k, v in FORMATS.items()}
XMAX["fp64"] = np.finfo(np.float64).max


def round_to(x, fmt: str) -> np.ndarray:
    """Round FP64 values to ``fmt`` (round to nearest, ties to even), returned as FP64."""
    x = np.asarray(x, dtype=np.float64)
    if fmt in ("fp64", "dd"):
        return x.copy()
    t, emin, xmax, sat = FORMATS[fmt]
    with np.errstate(invalid="ignore", over="ignore"):
        _, e = np.frexp(np.abs(x))          # |x| = f * 2^e, f in [0.5, 1)
        expo = np.maximum(e - 1, emin)      # exponent of the binade (emin in the subnormal range)
        quantum = np.ldexp(1.0, expo - (t - 1))
        r = np.rint(x / quantum) * quantum  # x/quantum is exact: quantum is a power of two
        big = np.abs(r) > xmax
        if sat:
            r = np.where(big, np.sign(x) * xmax, r)
        else:
            r = np.where(big, np.sign(x) * np.inf, r)
        r = np.where(np.isnan(x), np.nan, r)
    return r


def unit_roundoff(fmt: str) -> float:
    return UNIT_ROUNDOFF[fmt]
