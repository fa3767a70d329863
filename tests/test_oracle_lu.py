"""Pins of oracle.lu: LAPACK agreement, brute-force rational GEPP, scaling and operator identities."""
from fractions import Fraction

import numpy as np
import pytest
import scipy.linalg as sla

from oracle import lu as lum
from oracle.formats import UNIT_ROUNDOFF
from synth import randsvd, prolate

T_EMIN = {"fp16": (11, -14), "bf16": (8, -126), "fp32": (24, -126)}


def round_frac(q: Fraction, fmt):
    """Exact round-to-nearest-even of a rational into a binary format (independent of oracle.formats)."""
    t, emin = T_EMIN[fmt]
    if q == 0:
        return Fraction(0)
    a = abs(q)
    e = a.numerator.bit_length() - a.denominator.bit_length()
    while Fraction(2) ** e > a:
        e -= 1
    while Fraction(2) ** (e + 1) <= a:
        e += 1
    quantum = Fraction(2) ** (max(e, emin) - t + 1)
    v = q / quantum
    n = v.numerator // v.denominator
    rem = v - n
    if rem > Fraction(1, 2) or (rem == Fraction(1, 2) and n % 2 == 1):
        n += 1
    return n * quantum


def gepp_rational(A, fmt, fma):
    """Scalar GEPP on rationals with explicit rounding after every operation (or per FMA)."""
    n = len(A)
    W = [[Fraction(float(v)) for v in row] for row in A]
    W = [[round_frac(v, fmt) for v in row] for row in W]
    piv = []
    for k in range(n):
        p = max(range(k, n), key=lambda i: (abs(W[i][k]), -i))
        piv.append(p)
        W[k], W[p] = W[p], W[k]
        for i in range(k + 1, n):
            l = round_frac(W[i][k] / W[k][k], fmt)
            W[i][k] = l
            for j in range(k + 1, n):
                if fma:
                    W[i][j] = round_frac(W[i][j] - l * W[k][j], fmt)
                else:
                    W[i][j] = round_frac(W[i][j] - round_frac(l * W[k][j], fmt), fmt)
    return W, piv


@pytest.mark.parametrize("fmt", ["fp16", "bf16"])
def test_chop_matches_rational_gepp(fmt):
    rng = np.random.default_rng(7)
    for n in (3, 5, 7):
        A = rng.standard_normal((n, n))
        F = lum.lu_chop(A, fmt)
        W, piv = gepp_rational(A, fmt, fma=False)
        assert list(F.ipiv) == piv
        LU = np.tril(F.L, -1) + F.U
        assert np.array_equal(LU, np.array([[float(v) for v in row] for row in W]))


def test_block_panel_matches_rational_fp32_fma():
    """With w >= n the block model is GEPP in FP32 with fused updates; stored factors rounded."""
    rng = np.random.default_rng(8)
    n = 6
    A = rng.standard_normal((n, n))
    F = lum.lu_block(A, "bf16", w=64)
    W, piv = gepp_rational(A, "fp32", fma=True)
    assert list(F.ipiv) == piv
    ref = np.array([[float(round_frac(v, "bf16")) for v in row] for row in W])
    assert np.array_equal(np.tril(F.L, -1) + F.U, ref)


@pytest.mark.parametrize("mode", ["chop", "block"])
def test_fp64_matches_lapack(mode):
    rng = np.random.default_rng(9)
    n = 80
    A = rng.standard_normal((n, n))
    F = lum.lu_chop(A, "fp64") if mode == "chop" else lum.lu_block(A, "fp64", w=16)
    P, L, U = sla.lu(A)
    perm_lapack = np.argmax(P, axis=0)     # A = P L U  ->  A[perm] = L U
    assert np.array_equal(F.perm, perm_lapack)
    assert np.allclose(F.L, L, rtol=0, atol=1e-12)
    assert np.allclose(F.U, U, rtol=0, atol=1e-12 * np.abs(U).max())


@pytest.mark.parametrize("fmt", ["fp16", "bf16", "e4m3"])
def test_block_backward_error_and_pivots(fmt):
    n = 256
    A = randsvd(n, 1e4, seed=1)
    F = lum.lu_block(A, fmt, w=32)
    As = F.mu * (A * F.R[:, None]) * F.S[None, :]
    E = As[F.perm] - F.L @ F.U
    bound = (np.abs(F.L) @ np.abs(F.U)).max()
    assert np.abs(E).max() <= 8 * UNIT_ROUNDOFF[fmt] * bound
    assert np.abs(np.tril(F.L, -1)).max() <= 1.0
    # a block model that dropped the trailing update would fail this by O(1)
    assert np.abs(E).max() <= 0.5 * bound


def test_fp16_scaling():
    A = randsvd(64, 1e3, seed=2) * 1e9
    R, S = lum.equilibrate_pow2(A)
    for v in np.concatenate([R, S]):
        assert np.log2(v) == np.round(np.log2(v))
    RA = A * R[:, None]
    assert np.all((np.abs(RA).max(axis=1) >= 0.5) & (np.abs(RA).max(axis=1) < 1.0))
    RAS = RA * S[None, :]
    assert np.all((np.abs(RAS).max(axis=0) >= 0.5) & (np.abs(RAS).max(axis=0) < 1.0))
    assert lum.fp16_mu(1) == 4096.0 and lum.fp16_mu(64) == 512.0 and lum.fp16_mu(16384) == 32.0
    F = lum.lu_block(A, "fp16", w=16)
    # without the scaling the entries (~1e9) would overflow fp16; with it M^-1 A ~ I
    X = np.stack([lum.apply_minv(F, A[:, j]) for j in range(64)], axis=1)
    assert np.abs(X - np.eye(64)).max() < 0.5


def test_fp8_tiles():
    rng = np.random.default_rng(10)
    X = rng.standard_normal((300, 260)) * np.exp(rng.uniform(-5, 5, (300, 260)))
    Q = lum.quantize_operand(X, "e4m3", row0=50, col0=0)
    # tile grid is global: rows 50..127 form the first tile row
    for (r0, r1) in [(0, 78), (78, 206), (206, 300)]:
        for (c0, c1) in [(0, 128), (128, 256), (256, 260)]:
            blk, qb = X[r0:r1, c0:c1], Q[r0:r1, c0:c1]
            m = np.abs(blk).max()
            s = lum.fp8_tile_scale(m)
            assert 224 < m * s <= 448
            assert np.abs(qb - blk).max() <= 2.0 ** -4 * 448 / s


@pytest.mark.parametrize("fmt", ["fp64", "fp16", "bf16"])
def test_minv_transpose_identity(fmt):
    rng = np.random.default_rng(11)
    n = 60
    A = randsvd(n, 1e3, seed=3) * 7.0
    F = lum.lu_block(A, fmt, w=16)
    x = rng.standard_normal(n)
    y = rng.standard_normal(n)
    lhs = lum.apply_minv(F, x) @ y
    rhs = x @ lum.apply_minv_t(F, y)
    assert abs(lhs - rhs) <= 1e-10 * (abs(lhs) + 1)
    # the adjoint operator M^-T A^T is the transpose of A M^-1
    ax = (A @ lum.apply_minv(F, x)) @ y
    bx = x @ lum.apply_atilde_t(A, F, y)
    assert abs(ax - bx) <= 1e-10 * (abs(ax) + 1)


def test_minv_fp64_inverts():
    A = prolate(50, 0.47)
    F = lum.lu_block(A, "fp64", w=8)
    X = np.stack([lum.apply_atilde(A, F, e) for e in np.eye(50)], axis=1)
    assert np.abs(X - np.eye(50)).max() < 1e-6      # kappa ~ 1e7 at n = 50


def test_dd_apply_more_accurate():
    A = prolate(40, 0.455)
    F = lum.lu_block(A, "fp32", w=8)
    rng = np.random.default_rng(12)
    v = rng.standard_normal(40)
    a = lum.apply_atilde(A, F, v, "dd")
    b = lum.apply_atilde(A, F, v, "fp64")
    # both apply the same operator; they agree to the FP64 rounding of the operator
    assert np.abs(a - b).max() <= 1e-6 * np.abs(a).max()
