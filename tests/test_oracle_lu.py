"""Pins of oracle.lu: LAPACK agreement, brute-force rational GEPP, scaling and operator identities."""
from fractions import Fraction

import numpy as np
import pytest
import scipy.linalg as sla

from oracle import lu as lum
from oracle.formats import UNIT_ROUNDOFF
from synth import randsvd, prolate

T_EMIN = {"fp16": (11, -14), "bf16": (8, -126), "fp32": (24, -126), "e4m3": (4, -6)}


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


def _tile_scale_frac(vmax):
    """Largest power of two s with vmax * s <= 448 (1 for an all-zero tile), exactly."""
    if vmax == 0:
        return Fraction(1)
    e = 0
    while vmax * Fraction(2) ** e > 448:
        e -= 1
    while vmax * Fraction(2) ** (e + 1) <= 448:
        e += 1
    return Fraction(2) ** e


def _round_operand_frac(X, fmt, row0, col0, tile):
    """Round a block (list of rows of Fractions) to fmt; e4m3 per tile of the global grid."""
    if fmt != "e4m3":
        return [[round_frac(v, fmt) for v in row] for row in X]
    m, n = len(X), len(X[0]) if X else 0
    out = [[None] * n for _ in range(m)]
    for r0 in range(0, m):
        if (r0 + row0) % tile != 0 and r0 != 0:
            continue
        r1 = min(m, (r0 + row0) // tile * tile + tile - row0)
        for c0 in range(0, n):
            if (c0 + col0) % tile != 0 and c0 != 0:
                continue
            c1 = min(n, (c0 + col0) // tile * tile + tile - col0)
            vmax = max((abs(X[i][j]) for i in range(r0, r1) for j in range(c0, c1)), default=Fraction(0))
            sc = _tile_scale_frac(vmax)
            for i in range(r0, r1):
                for j in range(c0, c1):
                    out[i][j] = round_frac(X[i][j] * sc, "e4m3") / sc
    return out


def block_lu_rational(A, fmt, w, tile=None, round_l=True, round_u12=True, order="dot"):
    """The block-FMA LU model in exact rational arithmetic with explicit roundings, written
    from its definition independently of oracle.lu: per block column, GEPP of the panel with
    FP32 quotients and FP32 fused updates (ties to the lowest row), the panel's L and U11 rounded
    to fmt, U12 by FP32 substitution (exact dot, one rounding) with the rounded L11, then rounded
    to fmt, and the trailing matrix fl32(W - L21 U12) from the rounded operands (exact dot, one
    rounding). order='fma' rounds after every single product instead (in column order), in both
    the substitution and the trailing update. round_l / round_u12 switch off one rounding, to
    show the comparison sees it."""
    n = len(A)
    if fmt == "e4m3":
        w = tile
    f32 = lambda q: round_frac(q, "fp32")
    W = [[f32(Fraction(float(v))) for v in row] for row in A]
    Ls = [[Fraction(0)] * n for _ in range(n)]
    Us = [[Fraction(0)] * n for _ in range(n)]
    piv = []
    for c0 in range(0, n, w):
        c1 = min(c0 + w, n)
        for k in range(c0, c1):
            p = max(range(k, n), key=lambda i: (abs(W[i][k]), -i))
            piv.append(p)
            W[k], W[p] = W[p], W[k]
            Ls[k], Ls[p] = Ls[p], Ls[k]
            for i in range(k + 1, n):
                l = f32(W[i][k] / W[k][k])
                W[i][k] = l
                for j in range(k + 1, c1):
                    W[i][j] = f32(W[i][j] - l * W[k][j])
        wd = c1 - c0
        low = [[W[i][j] if (i - c0) > (j - c0) else Fraction(0) for j in range(c0, c1)] for i in range(c0, n)]
        lowq = _round_operand_frac(low, fmt, c0, c0, tile) if round_l else low
        for i in range(c0, n):
            for j in range(c0, c1):
                if i > j:
                    Ls[i][j] = lowq[i - c0][j - c0]
        top = [[W[i][j] if j >= i else Fraction(0) for j in range(c0, c1)] for i in range(c0, c1)]
        topq = _round_operand_frac(top, fmt, c0, c0, tile)
        for i in range(c0, c1):
            for j in range(c0, c1):
                if j >= i:
                    Us[i][j] = topq[i - c0][j - c0]
        if c1 < n:
            X = [list(W[i][c1:]) for i in range(c0, c1)]
            for r in range(1, wd):
                for j in range(n - c1):
                    if order == "dot":
                        X[r][j] = f32(X[r][j] - sum(Ls[c0 + r][c0 + q] * X[q][j] for q in range(r)))
                    else:
                        for q in range(r):
                            X[r][j] = f32(X[r][j] - Ls[c0 + r][c0 + q] * X[q][j])
            U12 = _round_operand_frac(X, fmt, c0, c1, tile) if round_u12 else X
            for i in range(wd):
                W[c0 + i][c1:] = X[i]
                Us[c0 + i][c1:] = U12[i]
            for i in range(c1, n):
                for j in range(c1, n):
                    if order == "dot":
                        W[i][j] = f32(W[i][j] - sum(Ls[i][c0 + q] * U12[q][j - c1] for q in range(wd)))
                    else:
                        for q in range(wd):
                            W[i][j] = f32(W[i][j] - Ls[i][c0 + q] * U12[q][j - c1])
    LU = [[float(Ls[i][j]) if i > j else float(Us[i][j]) for j in range(n)] for i in range(n)]
    return np.array(LU), piv


@pytest.mark.parametrize("fmt,n,w", [("bf16", 7, 2), ("bf16", 9, 3), ("fp16", 8, 3), ("fp16", 6, 2)])
def test_block_multipanel_matches_rational(fmt, n, w):
    """Several block columns: the oracle's block model equals the rational restatement bit for
    bit (pivots and every stored factor entry), and would not if it skipped the u_f rounding of
    L21 or of U12 before the trailing update."""
    rng = np.random.default_rng(100 * n + w)
    A = rng.standard_normal((n, n)) * np.exp(rng.uniform(-2, 2, (n, n)))
    F = lum.lu_block(A, fmt, w=w, scale=False)
    ref, piv = block_lu_rational(A, fmt, w)
    assert list(F.ipiv) == piv
    got = np.tril(F.L, -1) + F.U
    assert np.array_equal(got, ref)
    for kw in ({"round_l": False}, {"round_u12": False}):
        alt, _ = block_lu_rational(A, fmt, w, **kw)
        assert not np.array_equal(got, alt), kw


@pytest.mark.parametrize("fmt,n,w", [("bf16", 9, 3), ("fp16", 8, 3), ("bf16", 10, 4)])
def test_block_fma_order_matches_rational(fmt, n, w):
    """The 'fma' summation order (one FP32 rounding per product, in column order, in U12 and in the
    trailing update) equals its rational restatement bit for bit, and the rounding of U12 is seen."""
    rng = np.random.default_rng(300 + 10 * n + w)
    A = rng.standard_normal((n, n)) * np.exp(rng.uniform(-2, 2, (n, n)))
    F = lum.lu_block(A, fmt, w=w, scale=False, order="fma")
    ref, piv = block_lu_rational(A, fmt, w, order="fma")
    assert list(F.ipiv) == piv
    assert np.array_equal(np.tril(F.L, -1) + F.U, ref)
    alt, _ = block_lu_rational(A, fmt, w, order="fma", round_u12=False)
    assert not np.array_equal(np.tril(F.L, -1) + F.U, alt)


def test_block_orders_differ_and_both_factor():
    """The two summation orders give different u_f factors on a 96 x 96 randsvd matrix (the order
    reaches the stored factors through their rounding), and both satisfy the backward-error bound."""
    A = randsvd(96, 1e3, seed=5)
    Fd = lum.lu_block(A, "bf16", w=32, order="dot")
    Ff = lum.lu_block(A, "bf16", w=32, order="fma")
    assert not np.array_equal(Fd.U, Ff.U)
    for F in (Fd, Ff):
        E = A[F.perm] - F.L @ F.U
        assert np.abs(E).max() <= 8 * UNIT_ROUNDOFF["bf16"] * (np.abs(F.L) @ np.abs(F.U)).max()


def test_block_fp8_tiles_match_rational(monkeypatch):
    """FP8-E4M3 with power-of-two tile scales on a 4 x 4 tile grid (the tile size is the model's
    parameter; 128 in production): block columns of one tile width, panels crossing row-tile
    boundaries, a ragged last tile. Equal to the rational restatement bit for bit."""
    monkeypatch.setattr(lum, "FP8_TILE", 4)
    rng = np.random.default_rng(44)
    n = 10
    A = rng.standard_normal((n, n)) * np.exp(rng.uniform(-3, 3, (n, n)))
    F = lum.lu_block(A, "e4m3", w=32, scale=False)
    ref, piv = block_lu_rational(A, "e4m3", None, tile=4)
    assert list(F.ipiv) == piv
    got = np.tril(F.L, -1) + F.U
    assert np.array_equal(got, ref)
    for kw in ({"round_l": False}, {"round_u12": False}):
        alt, _ = block_lu_rational(A, "e4m3", None, tile=4, **kw)
        assert not np.array_equal(got, alt), kw


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
