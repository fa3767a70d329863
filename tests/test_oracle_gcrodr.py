"""Pins of oracle.gcrodr: Arnoldi relation, recycle invariants, least squares, harmonic Ritz,
and the k = 0 reduction to restarted GMRES(m)."""
import numpy as np
import scipy.linalg as sla

from oracle import gcrodr as G
from oracle import lu as lum
from synth import randsvd, prolate

U64 = 2.0 ** -53


def _system(n=120, kappa=1e6, fmt="fp16", seed=0):
    A = randsvd(n, kappa, seed=seed)
    F = lum.lu_block(A, fmt, w=16)
    op = lambda v: lum.apply_atilde(A, F, v, "fp64")
    Atil = np.stack([op(e) for e in np.eye(n)], axis=1)
    return A, F, op, Atil


def test_arnoldi_relation_and_orthogonality():
    n = 120
    _, _, op, At = _system(n)
    rng = np.random.default_rng(1)
    # a recycle space C with orthonormal columns (any will do for the relation)
    C, _ = np.linalg.qr(rng.standard_normal((n, 4)))
    r = rng.standard_normal(n)
    r = r - C @ (C.T @ r)
    V, H, B, j, _ = G.arnoldi(op, r, C, 20, 0.0, "fp64")
    assert j == 20
    lhs = np.stack([op(V[:, i]) for i in range(j)], axis=1)
    rel = np.linalg.norm(lhs - C @ B - V @ H) / (np.linalg.norm(At, 2) * np.sqrt(j))
    assert rel <= 10 * (4 + j) * U64
    W = np.hstack([C, V])
    assert np.abs(W.T @ W - np.eye(W.shape[1])).max() <= 10 * (4 + j) * U64
    # H is upper Hessenberg with a positive subdiagonal
    assert np.allclose(np.tril(H, -2), 0)
    assert np.all(np.diag(H, -1) > 0)


def test_recycle_invariants_after_every_solve():
    n = 150
    _, _, op, At = _system(n, kappa=1e4)
    rng = np.random.default_rng(2)
    Y = None
    for step in range(3):
        c = rng.standard_normal(n)
        d, U, C, info = G.gcrodr(op, c, 20, 6, 1e-10, Ytil=Y)
        assert U.shape[1] == C.shape[1] > 0
        kk = U.shape[1]
        assert np.abs(C.T @ C - np.eye(kk)).max() <= 10 * kk * U64 * 10
        AU = np.stack([op(U[:, i]) for i in range(kk)], axis=1)
        rel = np.linalg.norm(AU - C) / (np.linalg.norm(At, 2) * np.linalg.norm(U))
        # exact in exact arithmetic; rounding is amplified by ||R^-1|| of QR(G P)
        assert rel <= 1e4 * U64
        # the returned d solves the system to the tolerance (explicit residual)
        assert np.linalg.norm(c - At @ d) <= 1.01e-10 * np.linalg.norm(c) + 1e-14
        assert info.converged
        Y = U


def test_givens_estimate_matches_explicit_residual():
    n = 100
    _, _, op, At = _system(n, kappa=1e5)
    rng = np.random.default_rng(3)
    c = rng.standard_normal(n)
    d, U, C, info = G.gcrodr(op, c, 12, 4, 1e-9)
    assert info.cycles >= 2
    true = np.linalg.norm(c - At @ d)
    assert abs(info.resid[-1] - true) <= 1e-6 * np.linalg.norm(c) * 1e-3 + 1e-8 * true


def test_decoupled_least_squares():
    """The (k+j+1) x (k+j) problem with G = [[D, B], [0, H]] and rhs [0; beta e1] decouples:
    y2 solves the Hessenberg problem, y1 = -D^-1 B y2, and the residual is the Hessenberg one."""
    rng = np.random.default_rng(4)
    k, j = 5, 9
    D = np.diag(rng.uniform(0.5, 2, k))
    B = rng.standard_normal((k, j))
    H = np.triu(rng.standard_normal((j + 1, j)), -1)
    Gm = np.block([[D, B], [np.zeros((j + 1, k)), H]])
    rhs = np.zeros(k + j + 1)
    rhs[k] = 2.5
    y = G._lstsq(Gm, rhs)
    y2 = np.linalg.lstsq(H, rhs[k:], rcond=None)[0]
    assert np.allclose(y[k:], y2, rtol=1e-10, atol=1e-12)
    assert np.allclose(y[:k], -np.linalg.solve(D, B @ y2), rtol=1e-10, atol=1e-12)
    assert np.isclose(np.linalg.norm(rhs - Gm @ y), np.linalg.norm(rhs[k:] - H @ y2), rtol=1e-10)
    # Givens recurrence gives the same residual
    g = np.zeros(j + 1)
    g[0] = 2.5
    cs = np.zeros(j)
    sn = np.zeros(j)
    for i in range(j):
        e = G._givens_estimate(H, i, g, cs, sn)
    assert np.isclose(e, np.linalg.norm(rhs[k:] - H @ y2), rtol=1e-10)


def test_harmonic_ritz_whole_space_gives_eigenvalues():
    """When the Krylov space is the whole space (j = n) the harmonic Ritz values are the
    eigenvalues of A~ and the recycled U spans the invariant subspace of the k smallest."""
    n = 10
    A = randsvd(n, 1e3, seed=5)
    F = lum.lu_block(A, "bf16", w=4)
    op = lambda v: lum.apply_atilde(A, F, v, "fp64")
    At = np.stack([op(e) for e in np.eye(n)], axis=1)
    rng = np.random.default_rng(5)
    c = rng.standard_normal(n)
    d, U, C, info = G.gcrodr(op, c, n, 3, 1e-30, max_its=n)
    lam = np.linalg.eigvals(At)
    k_eff = U.shape[1]
    assert k_eff in (2, 3, 4)
    # U spans an invariant subspace of A~ ...
    T = np.linalg.lstsq(U, At @ U, rcond=None)[0]
    assert np.linalg.norm(At @ U - U @ T) <= 1e-8 * np.linalg.norm(At @ U)
    # ... whose eigenvalues are the smallest-magnitude eigenvalues of A~
    mu = np.sort(np.abs(np.linalg.eigvals(T)))
    assert np.allclose(mu, np.sort(np.abs(lam))[:k_eff], rtol=1e-6)


def test_select_harmonic_rules():
    theta = np.array([3.0, 0.5 + 1j, 0.5 - 1j, 0.2, 5.0, np.inf])
    Z = np.eye(6, dtype=complex)
    Z[:, 1] = Z[:, 1] + 1j * np.eye(6)[:, 2]
    Z[:, 2] = np.conj(Z[:, 1])
    P = G.select_harmonic(theta, Z, 2, 6, 10)          # 0.2 then the pair -> pair taken whole
    assert P.shape[1] == 3
    P = G.select_harmonic(theta, Z, 2, 6, 3)           # k + 1 = 3 is not < m: pair dropped
    assert P.shape[1] == 1
    P = G.select_harmonic(theta, Z, 1, 6, 10)
    assert P.shape[1] == 1 and P[3, 0] == 1.0
    P = G.select_harmonic(theta, Z, 5, 6, 10)          # inf sorts last
    assert P.shape[1] == 5 and np.all(P[5] == 0)


def plain_gmres(At, c, m, tol, max_its):
    """Independent textbook restarted GMRES(m) (modified Gram-Schmidt, lstsq per cycle)."""
    n = len(c)
    x = np.zeros(n)
    its = 0
    r = c.copy()
    while np.linalg.norm(r) > tol and its < max_its:
        beta = np.linalg.norm(r)
        V = [r / beta]
        H = np.zeros((m + 1, m))
        for j in range(m):
            w = At @ V[j]
            for i in range(j + 1):
                H[i, j] = w @ V[i]
                w = w - H[i, j] * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            V.append(w / H[j + 1, j])
            its += 1
            e1 = np.zeros(j + 2)
            e1[0] = beta
            y = np.linalg.lstsq(H[: j + 2, : j + 1], e1, rcond=None)[0]
            if np.linalg.norm(e1 - H[: j + 2, : j + 1] @ y) <= tol or its >= max_its:
                break
        x = x + np.stack(V[: len(y)], axis=1) @ y
        r = c - At @ x
    return x, its


def test_k0_is_restarted_gmres():
    n = 100
    _, _, op, At = _system(n, kappa=1e6, fmt="bf16")
    c = np.random.default_rng(6).standard_normal(n)
    tol = 1e-8 * np.linalg.norm(c)
    d, U, C, info = G.gcrodr(op, c, 10, 0, 1e-8, max_its=400)
    x, its = plain_gmres(At, c, 10, tol, 400)
    assert U.shape[1] == 0
    assert abs(info.its - its) <= 1
    assert np.linalg.norm(d - x) <= 1e-6 * np.linalg.norm(x)


def test_m_equals_n_solves_exactly():
    n = 30
    _, _, op, At = _system(n, kappa=1e4, fmt="bf16")
    c = np.random.default_rng(7).standard_normal(n)
    d, U, C, info = G.gcrodr(op, c, n, 5, 1e-13, max_its=n)
    assert info.its <= n
    assert np.linalg.norm(d - np.linalg.solve(At, c)) <= 1e-10 * np.linalg.norm(d)


def test_recycling_reduces_second_solve():
    A = prolate(100, 0.455)
    F = lum.lu_block(A, "fp32", w=16)
    op = lambda v: lum.apply_atilde(A, F, v, "fp64")
    rng = np.random.default_rng(8)
    c1, c2 = rng.standard_normal(100), rng.standard_normal(100)
    _, U, C, i1 = G.gcrodr(op, c1, 16, 4, 1e-8)
    _, _, _, i2 = G.gcrodr(op, c2, 16, 4, 1e-8, Ytil=U)
    _, _, _, i2n = G.gcrodr(op, c2, 16, 0, 1e-8)
    assert i2.its < i2n.its
    # carrying (U, C) instead of recomputing QR(A~ Y~) gives the same solve
    _, _, _, i2c = G.gcrodr(op, c2, 16, 4, 1e-8, carry=(U, C))
    assert abs(i2c.its - i2.its) <= 1 and i2c.carry_applies == 0 and i2.carry_applies == U.shape[1]


U32 = 2.0 ** -24


def test_fp32_basis_storage_relation_and_rounding():
    """Low-precision basis storage (Section 5's future work): with basis='fp32' every stored Arnoldi
    vector is an FP32 number and the Arnoldi relation and orthogonality hold at the FP32 level
    (and no better: the FP64-stored basis meets the same relation at the FP64 level, far below)."""
    n = 120
    _, _, op, At = _system(n)
    rng = np.random.default_rng(1)
    C, _ = np.linalg.qr(rng.standard_normal((n, 4)))
    C = C.astype(np.float32).astype(np.float64)
    r = rng.standard_normal(n)
    r = r - C @ (C.T @ r)
    V, H, B, j, _ = G.arnoldi(op, r, C, 20, 0.0, "fp64", store="fp32")
    assert j == 20
    assert np.array_equal(V, V.astype(np.float32).astype(np.float64))
    lhs = np.stack([op(V[:, i]) for i in range(j)], axis=1)
    rel = np.linalg.norm(lhs - C @ B - V @ H) / (np.linalg.norm(At, 2) * np.sqrt(j))
    assert rel <= 10 * (4 + j) * U32
    W = np.hstack([C, V])
    orth = np.abs(W.T @ W - np.eye(W.shape[1])).max()
    assert orth <= 10 * (4 + j) * U32
    V64, H64, B64, _, _ = G.arnoldi(op, r, C, 20, 0.0, "fp64")
    lhs64 = np.stack([op(V64[:, i]) for i in range(j)], axis=1)
    rel64 = np.linalg.norm(lhs64 - C @ B64 - V64 @ H64) / (np.linalg.norm(At, 2) * np.sqrt(j))
    assert rel > 100 * rel64


def test_fp32_basis_recycle_vectors_and_solve():
    """With basis='fp32' the recycle vectors U, C are FP32 numbers after every solve, C^T C = I and
    A~ U = C hold at the FP32 level, and GCRO-DR still reaches an inner tolerance of 1e-6; with
    basis='fp64' the solve is the default one, bit for bit."""
    n = 150
    _, _, op, At = _system(n, kappa=1e4)
    rng = np.random.default_rng(2)
    Y = None
    for step in range(3):
        c = rng.standard_normal(n)
        d, U, C, info = G.gcrodr(op, c, 20, 6, 1e-6, Ytil=Y, basis="fp32")
        kk = U.shape[1]
        assert kk > 0 and info.converged
        for X in (U, C):
            assert np.array_equal(X, X.astype(np.float32).astype(np.float64))
        assert np.abs(C.T @ C - np.eye(kk)).max() <= 10 * kk * U32 * 10
        AU = np.stack([op(U[:, i]) for i in range(kk)], axis=1)
        assert np.linalg.norm(AU - C) / (np.linalg.norm(At, 2) * np.linalg.norm(U)) <= 1e4 * U32
        assert np.linalg.norm(c - At @ d) <= 1.01e-6 * np.linalg.norm(c) + 1e-14
        Y = U
    c = rng.standard_normal(n)
    a = G.gcrodr(op, c, 20, 6, 1e-10, basis="fp64")
    b = G.gcrodr(op, c, 20, 6, 1e-10)
    assert np.array_equal(a[0], b[0]) and a[3].its == b[3].its
