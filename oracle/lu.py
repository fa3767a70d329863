"""LU factorization with partial pivoting in precision u_f, and the preconditioner it defines.

Algorithm 4 (and Algorithms 1-2) start with "compute the LU factorization A ~ LU in
precision u_f" and "solve A x0 = b by substitution in precision u_f". The paper runs
this with every arithmetic operation rounded to u_f (Section 3, chop); ``lu_chop`` is
that, written out: Gaussian elimination with partial pivoting (GEPP, Section 1; the
pivot is the first entry of largest magnitude in the column) where each quotient,
product and difference is rounded to u_f.

``lu_block`` is the precision-u_f factorization as tensor cores compute it (block
fused multiply-add model): the Schur complement is held in FP32, each block column of
width w is factored by GEPP in FP32 arithmetic, and the trailing update takes its
operands L21 and U12 rounded to u_f with exact products and FP32-or-better
accumulation. The stored factors are the u_f-rounded values. For fp16 the matrix is
first equilibrated by powers of two and scaled by mu (diagonal scaling against
overflow); for fp8-e4m3 each 128 x 128 tile of an operand gets its own power-of-two
scale. These are readings of "LU in precision u_f" for hardware formats;
``lu_block`` with fmt='fp64' is plain GEPP and is pinned against LAPACK.

The factors define M^-1 = mu S U^-1 L^-1 P R, the left preconditioner of the
correction equation (Algorithm 4); ``apply_minv`` applies it in a chosen
precision and ``apply_minv_t`` applies its transpose (used by the adjoint solve).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.linalg as sla

from .formats import round_to, UNIT_ROUNDOFF
from . import dd as ddm

FP8_TILE = 128
FP8_MAX = 448.0
FP16_THETA = 0.1


class SingularError(ArithmeticError):
    """A zero pivot was met."""


class NonFiniteError(ArithmeticError):
    """An infinity or NaN appeared (overflow of the factorization format)."""


@dataclass
class Factors:
    n: int
    fmt: str
    L: np.ndarray            # unit lower triangular, entries are u_f values (FP64 storage)
    U: np.ndarray            # upper triangular, u_f values
    perm: np.ndarray         # (P v)[i] = v[perm[i]]
    ipiv: np.ndarray         # sequential row interchanges: at step k rows k and ipiv[k] swapped
    R: np.ndarray = field(default=None)   # row scaling (powers of two)
    S: np.ndarray = field(default=None)   # column scaling (powers of two)
    mu: float = 1.0
    mode: str = "block"


def pow2_floor_scale(m):
    """2^-E with m = f 2^E, f in [0.5, 1): maps m into [0.5, 1). m == 0 gives 1."""
    m = np.asarray(m, dtype=np.float64)
    _, e = np.frexp(m)
    return np.where(m > 0, np.ldexp(1.0, -e), 1.0)


def equilibrate_pow2(A):
    """Two-sided power-of-two equilibration: R = diag(row scales), S = diag(column scales of RA).

    After scaling every row and then every column of R A S has largest magnitude in [0.5, 1).
    """
    R = pow2_floor_scale(np.max(np.abs(A), axis=1))
    RA = A * R[:, None]
    S = pow2_floor_scale(np.max(np.abs(RA), axis=0))
    return R, S


def fp16_mu(n=1):
    """mu = largest power of two not above theta * xmax(fp16) / sqrt(n), theta = 0.1.

    The 1/sqrt(n) leaves room for the element growth of partial pivoting, which grows with
    the dimension, so the factors do not overflow fp16 (a reading: the paper does not scale).
    """
    return float(2.0 ** np.floor(np.log2(FP16_THETA * 65504.0 / np.sqrt(n))))


def scale_for(A, fmt):
    """(R, S, mu) of the input scaling step for format ``fmt``."""
    n = A.shape[0]
    if fmt == "fp16":
        R, S = equilibrate_pow2(A)
        return R, S, fp16_mu(n)
    return np.ones(n), np.ones(n), 1.0


def fp8_tile_scale(tile_max):
    """Power-of-two s with tile_max * s in (224, 448]; 1 for an all-zero tile."""
    tile_max = np.asarray(tile_max, dtype=np.float64)
    with np.errstate(divide="ignore"):
        e = np.floor(np.log2(FP8_MAX / np.where(tile_max > 0, tile_max, 1.0)))
    return np.where(tile_max > 0, np.ldexp(1.0, e.astype(np.int64)), 1.0)


def quantize_operand(X, fmt, row0=0, col0=0):
    """Round an operand block to the factorization format.

    For fp8-e4m3 every 128 x 128 tile of the global tile grid (X[0, 0] sits at global
    position (row0, col0)) is multiplied by its power-of-two scale, rounded with
    saturation, and divided by the scale again.
    """
    if fmt != "e4m3":
        return round_to(X, fmt)
    out = np.empty_like(X)
    m, n = X.shape
    t = FP8_TILE
    r = 0
    while r < m:
        r_end = min(m, (r + row0) // t * t + t - row0)
        c = 0
        while c < n:
            c_end = min(n, (c + col0) // t * t + t - col0)
            blk = X[r:r_end, c:c_end]
            s = fp8_tile_scale(np.max(np.abs(blk)) if blk.size else 0.0)
            out[r:r_end, c:c_end] = round_to(blk * s, "e4m3") / s
            c = c_end
        r = r_end
    return out


def _check_pivot(v):
    if not np.isfinite(v):
        raise NonFiniteError("non-finite pivot")
    if v == 0.0:
        raise SingularError("zero pivot")


def lu_chop(A, fmt):
    """GEPP with every quotient, product and difference rounded to ``fmt`` (paper's chop form).

    Computing each operation in FP64 and rounding once gives the correctly rounded
    result for fp32 and narrower formats (53 >= 2t + 2, so the double rounding is innocuous).
    """
    W = round_to(np.array(A, dtype=np.float64), fmt)
    n = W.shape[0]
    perm = np.arange(n)
    ipiv = np.zeros(n, dtype=np.int64)
    for k in range(n):
        p = k + int(np.argmax(np.abs(W[k:, k])))
        ipiv[k] = p
        _check_pivot(W[p, k])
        if p != k:
            W[[k, p]] = W[[p, k]]
            perm[[k, p]] = perm[[p, k]]
        if k + 1 < n:
            l = round_to(W[k + 1:, k] / W[k, k], fmt)
            W[k + 1:, k] = l
            prod = round_to(np.outer(l, W[k, k + 1:]), fmt)
            W[k + 1:, k + 1:] = round_to(W[k + 1:, k + 1:] - prod, fmt)
        if not np.all(np.isfinite(W[k:, k:])):
            raise NonFiniteError("overflow in the factorization format")
    L = np.tril(W, -1) + np.eye(n)
    U = np.triu(W)
    return Factors(n, fmt, L, U, perm, ipiv, np.ones(n), np.ones(n), 1.0, mode="chop")


def lu_block(A, fmt, w=64, scale=True, order="dot"):
    """Block-FMA LU in precision ``fmt`` with block-column width ``w`` (the tensor-core model).

    Steps per block column [c0, c1):
      1. GEPP on the panel W[c0:, c0:c1] in FP32 arithmetic (each l is an FP32 quotient and
         each update an FP32 fused multiply-add), whole rows interchanged.
      2. Stored factors: L21/L11 and U11 rounded to ``fmt``.
      3. U12 = L11^-1 W[c0:c1, c1:] by FP32 substitution with the stored (rounded) L11, then
         rounded to ``fmt``.
      4. W[c1:, c1:] = fl32(W[c1:, c1:] - L21 U12) with the rounded operands.
    ``order`` is the FP32 summation order of steps 3 and 4, which the paper leaves open:
    'dot' rounds each entry once after its whole sum of products (the reference reading);
    'fma' subtracts the products one at a time in column order, rounding to FP32 after each
    (an FP32 fused multiply-add chain over the w columns). The products are exact in both.
    ``scale`` applies the fp16 equilibration (R, S, mu). fmt='fp64' gives plain GEPP in FP64.
    """
    if order not in ("dot", "fma"):
        raise ValueError(order)
    A = np.array(A, dtype=np.float64)
    n = A.shape[0]
    if scale:
        R, S, mu = scale_for(A, fmt)
    else:
        R, S, mu = np.ones(n), np.ones(n), 1.0
    As = mu * (A * R[:, None]) * S[None, :]
    work = "fp64" if fmt == "fp64" else "fp32"
    f32 = (lambda z: np.array(z, dtype=np.float64)) if work == "fp64" else (lambda z: round_to(z, "fp32"))
    W = f32(As)
    if not np.all(np.isfinite(W)):
        raise NonFiniteError("input does not fit the working format")
    Lst = np.zeros((n, n))
    Ust = np.zeros((n, n))
    perm = np.arange(n)
    ipiv = np.zeros(n, dtype=np.int64)
    if fmt == "e4m3":
        w = FP8_TILE
    for c0 in range(0, n, w):
        c1 = min(c0 + w, n)
        for k in range(c0, c1):
            p = k + int(np.argmax(np.abs(W[k:, k])))
            ipiv[k] = p
            _check_pivot(W[p, k])
            if p != k:
                W[[k, p]] = W[[p, k]]
                Lst[[k, p]] = Lst[[p, k]]
                perm[[k, p]] = perm[[p, k]]
            if k + 1 < n:
                l = f32(W[k + 1:, k] / W[k, k])
                W[k + 1:, k] = l
                if k + 1 < c1:
                    W[k + 1:, k + 1:c1] = f32(W[k + 1:, k + 1:c1] - np.outer(l, W[k, k + 1:c1]))
        panel = W[c0:, c0:c1].copy()
        wd = c1 - c0
        top = panel[:wd]
        lower = panel.copy()
        lower[:wd] = np.tril(top, -1)
        Lst[c0:, c0:c1] = quantize_operand(lower, fmt, c0, c0)
        Ust[c0:c1, c0:c1] = quantize_operand(np.triu(top), fmt, c0, c0)
        if c1 < n:
            L11 = Lst[c0:c1, c0:c1] + np.eye(wd)
            X = W[c0:c1, c1:].copy()
            for r in range(1, wd):
                if order == "dot":
                    X[r] = f32(X[r] - L11[r, :r] @ X[:r])
                else:
                    for q in range(r):
                        X[r] = f32(X[r] - L11[r, q] * X[q])
            U12 = quantize_operand(X, fmt, c0, c1)
            Ust[c0:c1, c1:] = U12
            W[c0:c1, c1:] = X
            if order == "dot":
                W[c1:, c1:] = f32(W[c1:, c1:] - Lst[c1:, c0:c1] @ U12)
            elif work == "fp32":
                # products of two u_f values are exact in FP32, so each FP32 subtraction below is
                # one correctly rounded fused multiply-add
                Wt = W[c1:, c1:].astype(np.float32)
                L32 = Lst[c1:, c0:c1].astype(np.float32)
                U32 = U12.astype(np.float32)
                for q in range(wd):
                    Wt -= np.outer(L32[:, q], U32[q])
                W[c1:, c1:] = Wt.astype(np.float64)
            else:
                for q in range(wd):
                    W[c1:, c1:] = W[c1:, c1:] - np.outer(Lst[c1:, c0 + q], U12[q])
            if not np.all(np.isfinite(W[c1:, c1:])):
                raise NonFiniteError("overflow in the Schur complement")
    L = Lst + np.eye(n)
    return Factors(n, fmt, L, Ust, perm, ipiv, R, S, mu, mode="block")


# --------------------------------------------------------------------------- applying M^-1

def _chop_lower(L, z, fmt, unit=True):
    s = np.array(z, dtype=np.float64, copy=True)
    n = len(s)
    y = np.zeros(n)
    for j in range(n):
        y[j] = s[j] if unit else round_to(s[j] / L[j, j], fmt)
        if j + 1 < n:
            s[j + 1:] = round_to(s[j + 1:] - round_to(L[j + 1:, j] * y[j], fmt), fmt)
    return y


def _chop_upper(U, z, fmt):
    s = np.array(z, dtype=np.float64, copy=True)
    n = len(s)
    y = np.zeros(n)
    for j in range(n - 1, -1, -1):
        y[j] = round_to(s[j] / U[j, j], fmt)
        if j > 0:
            s[:j] = round_to(s[:j] - round_to(U[:j, j] * y[j], fmt), fmt)
    return y


def apply_minv(F: Factors, v, prec="fp64", out_fmt=None):
    """M^-1 v = mu S U^-1 L^-1 P R v with the triangular solves in precision ``prec``.

    prec: 'fp64' (LAPACK substitution), 'fp32', 'dd' (double-double substitution) or a
    factorization format name for substitution with every operation rounded to it.
    The result is rounded to ``out_fmt`` when given.
    """
    z = (F.R * np.asarray(v, dtype=np.float64))[F.perm]
    if prec == "fp64":
        y = sla.solve_triangular(F.L, z, lower=True, unit_diagonal=True, check_finite=False)
        y = sla.solve_triangular(F.U, y, lower=False, check_finite=False)
    elif prec == "fp32":
        y = sla.solve_triangular(F.L.astype(np.float32), z.astype(np.float32), lower=True,
                                 unit_diagonal=True, check_finite=False)
        y = sla.solve_triangular(F.U.astype(np.float32), y, lower=False, check_finite=False)
        y = y.astype(np.float64)
    elif prec == "dd":
        yh, yl = ddm.dd_lower_solve(F.L, z, np.zeros_like(z), unit=True)
        yh, yl = ddm.dd_upper_solve(F.U, yh, yl)
        y = yh + yl
    else:
        y = _chop_lower(F.L, round_to(z, prec), prec)
        y = _chop_upper(F.U, y, prec)
    y = F.mu * F.S * y
    return round_to(y, out_fmt) if out_fmt else y


def apply_minv_t(F: Factors, v, prec="fp64", out_fmt=None):
    """M^-T v = mu R P^T L^-T U^-T S v (the adjoint preconditioner)."""
    z = F.S * np.asarray(v, dtype=np.float64)
    if prec == "fp64":
        y = sla.solve_triangular(F.U, z, lower=False, trans="T", check_finite=False)
        y = sla.solve_triangular(F.L, y, lower=True, trans="T", unit_diagonal=True, check_finite=False)
    elif prec == "dd":
        yh, yl = ddm.dd_lower_solve(F.U.T.copy(), z, np.zeros_like(z), unit=False)
        yh, yl = ddm.dd_upper_solve(F.L.T.copy(), yh, yl)
        y = yh + yl
    else:
        raise ValueError(prec)
    w = np.empty_like(y)
    w[F.perm] = y
    w = F.mu * F.R * w
    return round_to(w, out_fmt) if out_fmt else w


def matvec(A, v, prec="fp64"):
    """A v in precision ``prec`` ('fp64', 'fp32', 'dd')."""
    if prec == "fp64":
        return A @ v
    if prec == "fp32":
        return (A.astype(np.float32) @ np.asarray(v, dtype=np.float32)).astype(np.float64)
    if prec == "dd":
        h, l = ddm.dd_matvec(A, np.asarray(v, dtype=np.float64))
        return h + l
    raise ValueError(prec)


def ipiv_to_perm(ipiv):
    n = len(ipiv)
    perm = np.arange(n)
    for k in range(n):
        p = ipiv[k]
        if p != k:
            perm[[k, p]] = perm[[p, k]]
    return perm


def unit_roundoff(fmt):
    return UNIT_ROUNDOFF[fmt]


def apply_atilde(A, F: Factors, v, prec="fp64", out_fmt=None):
    """A~ v = M^-1 (A v): the preconditioned operator of Algorithm 4's correction equation, in precision ``prec``.

    For 'dd' the product A v and both substitutions are carried in double-double
    without an intermediate rounding (the paper's u^2 = quad application for u = FP64).
    """
    v = np.asarray(v, dtype=np.float64)
    if prec != "dd":
        return apply_minv(F, matvec(A, v, prec), prec, out_fmt)
    wh, wl = ddm.dd_matvec(A, v)
    zh = (F.R * wh)[F.perm]
    zl = (F.R * wl)[F.perm]
    yh, yl = ddm.dd_lower_solve(F.L, zh, zl, unit=True)
    yh, yl = ddm.dd_upper_solve(F.U, yh, yl)
    y = F.mu * F.S * (yh + yl)
    return round_to(y, out_fmt) if out_fmt else y


def apply_atilde_t(A, F: Factors, v, prec="fp64", out_fmt=None):
    """M^-T (A^T v): the operator of the adjoint correction equation."""
    v = np.asarray(v, dtype=np.float64)
    if prec == "dd":
        wh, wl = ddm.dd_matvec(A.T.copy(), v)
        zh, zl = F.S * wh, F.S * wl
        yh, yl = ddm.dd_lower_solve(F.U.T.copy(), zh, zl, unit=False)
        yh, yl = ddm.dd_upper_solve(F.L.T.copy(), yh, yl)
        y = np.empty_like(yh)
        y[F.perm] = yh + yl
        y = F.mu * F.R * y
        return round_to(y, out_fmt) if out_fmt else y
    return apply_minv_t(F, matvec(A.T, v, prec), prec, out_fmt)
