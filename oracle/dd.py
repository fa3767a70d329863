"""Double-double arithmetic (a value is an unevaluated sum hi + lo of two FP64 numbers).

The paper simulates quad precision with a multiprecision toolbox (Section 3); the
oracle uses double-double instead (unit roundoff about 2^-106, which is still below
u^2 for u = FP64). Error-free transformations: Knuth's TwoSum and Dekker's TwoProduct
with Veltkamp splitting (numpy has no fused multiply-add).

Pinned by tests/test_oracle_dd.py against exact rational arithmetic (fractions.Fraction).
"""
from __future__ import annotations

import numpy as np

_SPLITTER = 134217729.0  # 2^27 + 1


def two_sum(a, b):
    s = a + b
    bb = s - a
    e = (a - (s - bb)) + (b - bb)
    return s, e


def fast_two_sum(a, b):
    s = a + b
    e = b - (s - a)
    return s, e


def split(a):
    c = _SPLITTER * a
    hi = c - (c - a)
    return hi, a - hi


def two_prod(a, b):
    p = a * b
    ah, al = split(a)
    bh, bl = split(b)
    e = ((ah * bh - p) + ah * bl + al * bh) + al * bl
    return p, e


def dd_add(ah, al, bh, bl):
    s, e = two_sum(ah, bh)
    t, f = two_sum(al, bl)
    e = e + t
    s, e = fast_two_sum(s, e)
    e = e + f
    return fast_two_sum(s, e)


def dd_add_d(ah, al, b):
    s, e = two_sum(ah, b)
    e = e + al
    return fast_two_sum(s, e)


def dd_mul_d(ah, al, b):
    p, e = two_prod(ah, b)
    e = e + al * b
    return fast_two_sum(p, e)


def dd_div_d(ah, al, b):
    """(ah + al) / b for an FP64 b, to double-double accuracy."""
    q1 = ah / b
    ph, pl = two_prod(q1, b)
    rh, rl = dd_add(ah, al, -ph, -pl)
    q2 = rh / b
    ph, pl = two_prod(q2, b)
    rh, rl = dd_add(rh, rl, -ph, -pl)
    q3 = rh / b
    s, e = fast_two_sum(q1, q2)
    return dd_add_d(s, e, q3)


def dd_residual(A, x, b):
    """r = b - A x accumulated in double-double (exact products), returned as (hi, lo)."""
    A = np.asarray(A, dtype=np.float64)
    x = np.asarray(x, dtype=np.float64)
    hi = np.array(b, dtype=np.float64, copy=True)
    lo = np.zeros_like(hi)
    for j in range(A.shape[1]):
        ph, pl = two_prod(A[:, j], x[j])
        hi, lo = dd_add(hi, lo, -ph, -pl)
    return hi, lo


def dd_matvec(A, vh, vl=None):
    """y = A v in double-double for a double-double vector v (vl may be None)."""
    A = np.asarray(A, dtype=np.float64)
    n = A.shape[0]
    hi = np.zeros(n)
    lo = np.zeros(n)
    for j in range(A.shape[1]):
        ph, pl = two_prod(A[:, j], vh[j])
        if vl is not None:
            pl = pl + A[:, j] * vl[j]
        hi, lo = dd_add(hi, lo, ph, pl)
    return hi, lo


def dd_lower_solve(L, zh, zl, unit: bool):
    """Forward substitution L y = z in double-double (column-oriented)."""
    n = L.shape[0]
    sh = np.array(zh, dtype=np.float64, copy=True)
    sl = np.array(zl, dtype=np.float64, copy=True)
    yh = np.zeros(n)
    yl = np.zeros(n)
    for j in range(n):
        if unit:
            yh[j], yl[j] = sh[j], sl[j]
        else:
            yh[j], yl[j] = dd_div_d(sh[j], sl[j], L[j, j])
        if j + 1 < n:
            col = L[j + 1:, j]
            ph, pl = two_prod(col, yh[j])
            pl = pl + col * yl[j]
            sh[j + 1:], sl[j + 1:] = dd_add(sh[j + 1:], sl[j + 1:], -ph, -pl)
    return yh, yl


def dd_upper_solve(U, zh, zl):
    """Back substitution U y = z in double-double (column-oriented)."""
    n = U.shape[0]
    sh = np.array(zh, dtype=np.float64, copy=True)
    sl = np.array(zl, dtype=np.float64, copy=True)
    yh = np.zeros(n)
    yl = np.zeros(n)
    for j in range(n - 1, -1, -1):
        yh[j], yl[j] = dd_div_d(sh[j], sl[j], U[j, j])
        if j > 0:
            col = U[:j, j]
            ph, pl = two_prod(col, yh[j])
            pl = pl + col * yl[j]
            sh[:j], sl[:j] = dd_add(sh[:j], sl[:j], -ph, -pl)
    return yh, yl
