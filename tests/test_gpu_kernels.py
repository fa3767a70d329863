"""GPU parity of the single steps of the hot path against the CPU oracle (through the C ABI)."""
import numpy as np
import pytest
import torch

from oracle import dd as odd
from oracle import lu as olu
from oracle.formats import round_to, UNIT_ROUNDOFF
from synth import randsvd, prolate

pytestmark = pytest.mark.gpu
U64 = 2.0 ** -53


@pytest.fixture(scope="module")
def G():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2201_09827_gb300 import gir
    gir.load()
    return gir


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("n", [1, 7, 128, 129, 1000, 1023])
def test_residual_fp64_and_dd(G, n):
    rng = np.random.default_rng(n)
    A = rng.standard_normal((n, n))
    x = rng.standard_normal(n)
    b = A @ x + 1e-12 * rng.standard_normal(n)        # heavy cancellation
    rh, rl = odd.dd_residual(A, x, b)
    exact = rh + rl
    scale = np.abs(A) @ np.abs(x) + np.abs(b)
    r64 = G.residual(cuda(A), cuda(x), cuda(b), "fp64").cpu().numpy()
    assert np.all(np.abs(r64 - exact) <= 1.01 * n * U64 * scale + 1e-300)
    rdd = G.residual(cuda(A), cuda(x), cuda(b), "dd").cpu().numpy()
    assert np.all(np.abs(rdd - exact) <= U64 * np.abs(exact) + 4 * n * 2.0 ** -106 * scale + 1e-300)


def test_residual_strided(G):
    n, lda = 300, 333
    rng = np.random.default_rng(5)
    Afull = rng.standard_normal((n, lda))
    A = Afull[:, :n]
    x = rng.standard_normal(n)
    b = rng.standard_normal(n)
    Ad = cuda(Afull)[:, :n]
    r = G.residual(Ad, cuda(x), cuda(b), "dd").cpu().numpy()
    rh, rl = odd.dd_residual(A, x, b)
    assert np.abs(r - (rh + rl)).max() <= 1e-13


@pytest.mark.parametrize("n", [1, 33, 512, 1000])
@pytest.mark.parametrize("trans", [False, True])
def test_gemv(G, n, trans):
    rng = np.random.default_rng(n + trans)
    A = rng.standard_normal((n, n))
    v = rng.standard_normal(n)
    w = G.gemv(cuda(A), cuda(v), trans=trans).cpu().numpy()
    ref = (A.T if trans else A) @ v
    assert np.abs(w - ref).max() <= 2 * n * U64 * (np.abs(A).max() * np.abs(v).sum() + 1)


def panel_oracle(W):
    """GEPP of an FP32 panel with correctly rounded FP32 quotients and fused updates."""
    W = W.astype(np.float64).copy()
    m, w = W.shape
    piv = []
    f32 = lambda z: round_to(z, "fp32")
    for k in range(w):
        p = k + int(np.argmax(np.abs(W[k:, k])))
        piv.append(p)
        W[[k, p]] = W[[p, k]]
        l = f32(W[k + 1:, k] / W[k, k])
        W[k + 1:, k] = l
        W[k + 1:, k + 1:] = f32(W[k + 1:, k + 1:] - np.outer(l, W[k, k + 1:]))
    return W, np.array(piv)


@pytest.mark.parametrize("m,w,cluster", [(32, 32, 1), (200, 32, 1), (2000, 32, 2), (2000, 32, 5), (3001, 17, 13),
                                         (1000, 16, 16), (77, 1, 3), (4096, 7, 8),
                                         (1500, 32, 1), (1400, 16, 1)])
def test_panel_bitexact(G, m, w, cluster):
    """Ties in the first column resolve to the lowest row; the last two cases put 1500 / 1400
    rows (three per thread) into one CTA."""
    rng = np.random.default_rng(m * 31 + w)
    W = rng.standard_normal((m, w)).astype(np.float32)
    W[rng.integers(0, m, 5), 0] = 3.0        # exact ties in the first column: lowest row wins
    Wd = cuda(W)
    ipiv = G.lu_panel(Wd, cluster=cluster).cpu().numpy()
    Wo, po = panel_oracle(W)
    assert np.array_equal(ipiv, po)
    assert np.array_equal(Wd.cpu().numpy().astype(np.float64), Wo)


def test_panel_singular_column(G):
    W = np.random.default_rng(1).standard_normal((100, 8)).astype(np.float32)
    W[:, 3] = W[:, 1] * 2.0
    W[:, 3] -= W[:, 1] * 2.0                 # exactly zero column
    with pytest.raises(G.GirError) as e:
        G.lu_panel(cuda(W))
    assert e.value.status == G.GIR_SINGULAR


@pytest.mark.parametrize("fmt,tdt", [("bf16", torch.bfloat16), ("fp16", torch.float16)])
@pytest.mark.parametrize("M,N,K", [(128, 256, 64), (300, 500, 256), (1000, 700, 32), (257, 129, 200), (4096, 2048, 512)])
@pytest.mark.parametrize("tc", [True, False])
def test_trailing_update(G, fmt, tdt, M, N, K, tc):
    g = torch.Generator(device="cuda").manual_seed(M + N + K)
    A = torch.randn(M, K, device="cuda", generator=g).to(tdt)
    B = torch.randn(K, N, device="cuda", generator=g).to(tdt)
    C0 = torch.randn(M, N, device="cuda", dtype=torch.float32, generator=g)
    ref = C0.double() - A.double() @ B.double()          # exact products, FP64 sums
    Cm = C0.clone()
    G.lu_update(Cm, A.view(torch.int16), B.view(torch.int16), fmt, use_tc=tc)
    bound = (K + 2) * 2.0 ** -24 * ((A.double().abs() @ B.double().abs()) + C0.double().abs())
    assert bool(((Cm.double() - ref).abs() <= bound).all())


def _gpu_factors(G, A, fmt, m=20, k=5, ua="fp64"):
    import paper_2201_09827_gb300 as pkg
    F = pkg.Factorization(cuda(A), pkg.Params(uf=fmt, m=m, k=k, ua=ua))
    LU, ipiv, R, S, mu = F.export_factors()
    LU = LU.double().cpu().numpy()
    n = A.shape[0]
    ipiv = ipiv.cpu().numpy()
    Fo = olu.Factors(n, fmt, np.tril(LU, -1) + np.eye(n), np.triu(LU), olu.ipiv_to_perm(ipiv), ipiv,
                     R.cpu().numpy(), S.cpu().numpy(), mu)
    return F, Fo


@pytest.mark.parametrize("n,fmt", [(32, "bf16"), (20, "fp16")])
def test_factor_single_panel_bitexact(G, n, fmt):
    """n <= panel width: the factorization is one FP32 GEPP panel, identical to the oracle's model."""
    A = randsvd(n, 1e3, seed=3)
    F, Fg = _gpu_factors(G, A, fmt)
    Fo = olu.lu_block(A, fmt, w=32)
    assert np.array_equal(Fg.ipiv, Fo.ipiv)
    assert np.array_equal(Fg.L, Fo.L) and np.array_equal(Fg.U, Fo.U)
    assert np.array_equal(Fg.R, Fo.R) and np.array_equal(Fg.S, Fo.S) and Fg.mu == Fo.mu
    F.close()


@pytest.mark.parametrize("n,fmt", [(100, "bf16"), (300, "bf16"), (300, "fp16"), (1000, "fp16"), (1537, "bf16")])
def test_factor_properties(G, n, fmt):
    """Beyond one panel the FP32 summation order differs from the oracle, so the factors are
    checked by what both must satisfy: partial pivoting and the u_f backward error bound."""
    A = randsvd(n, 1e3, seed=n)
    F, Fg = _gpu_factors(G, A, fmt)
    Fo = olu.lu_block(A, fmt, w=32)
    # identical input scaling (a plain definition: powers of two from row/column maxima)
    assert np.array_equal(Fg.R, Fo.R) and np.array_equal(Fg.S, Fo.S) and Fg.mu == Fo.mu
    As = Fg.mu * (A * Fg.R[:, None]) * Fg.S[None, :]
    E = np.abs(As[Fg.perm] - Fg.L @ Fg.U).max() / (np.abs(Fg.L) @ np.abs(Fg.U)).max()
    Eo = np.abs(As[Fo.perm] - Fo.L @ Fo.U).max() / (np.abs(Fo.L) @ np.abs(Fo.U)).max()
    assert E <= 8 * UNIT_ROUNDOFF[fmt] and E <= 4 * Eo + UNIT_ROUNDOFF[fmt]
    assert np.abs(np.tril(Fg.L, -1)).max() <= 1.0
    # the stored values are representable in u_f
    assert np.array_equal(round_to(Fg.U, fmt), Fg.U)
    F.close()


U_FF = 2.0 ** -46     # float-float unit roundoff (two FP32 significands)


def _ff_bound(Fg, A, v, trans, with_a):
    """Elementwise forward-error bound of the float-float application of M^-1 (or M^-T), and of
    A~ = M^-1 A (with_a), from the arithmetic: each substitution in float-float has the componentwise
    error |T^-1| |T| |y| u_ff (per step, times a small constant), the error of the first solve
    propagates through the second as |T2^-1| |delta|, and the float-float product A v adds
    |A| |v| u_ff at the input. Returned without the constant and u_ff."""
    import scipy.linalg as sla
    n = Fg.L.shape[0]
    Li = sla.solve_triangular(Fg.L, np.eye(n), lower=True, unit_diagonal=True)
    Ui = sla.solve_triangular(Fg.U, np.eye(n), lower=False)
    if not trans:
        x = A @ v if with_a else v
        z = (Fg.mu * Fg.R * x)[Fg.perm]
        zin = ((Fg.mu * Fg.R * (np.abs(A) @ np.abs(v)))[Fg.perm]) if with_a else np.zeros(n)
        y1 = Li @ z
        y = Ui @ y1
        b = np.abs(Ui) @ (np.abs(Li) @ (np.abs(Fg.L) @ np.abs(y1) + zin)) + np.abs(Ui) @ (np.abs(Fg.U) @ np.abs(y))
        return np.abs(Fg.S) * b
    x = A.T @ v if with_a else v
    z = Fg.S * x
    y1 = Ui.T @ z
    y = Li.T @ y1
    b = np.abs(Li.T) @ (np.abs(Ui.T) @ (np.abs(Fg.U.T) @ np.abs(y1))) + np.abs(Li.T) @ (np.abs(Fg.L.T) @ np.abs(y))
    out = np.empty(n)
    out[Fg.perm] = Fg.mu * Fg.R[Fg.perm] * b
    return out


@pytest.mark.parametrize("n,fmt", [(64, "bf16"), (300, "fp16"), (1000, "bf16"), (1031, "fp16"), (1537, "bf16"),
                                   (2600, "fp16"), (4096, "bf16")])
def test_apply_minv_and_atilde(G, n, fmt):
    """With the same (GPU) factors, M^-1 v, M^-1 A v and their transposes agree elementwise with the
    oracle's FP64 substitution within the forward-error bound of float-float substitution
    (_ff_bound, u_ff = 2^-46, constant 64 for the block order of the sums). The transposed product
    A^T v is FP64 and the oracle's own FP64 error sits 2^7 below u_ff. n = 1537, 2600 and 4096 span
    several 16-CTA clusters of 64-row blocks (1024 rows each), the first two with a ragged last
    block."""
    A = randsvd(n, 1e4, seed=7)
    F, Fg = _gpu_factors(G, A, fmt)
    rng = np.random.default_rng(8)
    for trans in (False, True):
        v = rng.standard_normal(n)
        w = F.apply_minv(cuda(v), trans=trans).cpu().numpy()
        wo = olu.apply_minv_t(Fg, v) if trans else olu.apply_minv(Fg, v)
        bound = 64 * U_FF * _ff_bound(Fg, A, v, trans, False)
        assert np.all(np.abs(w - wo) <= bound), (trans, np.max(np.abs(w - wo) / bound))
        w = F.apply_atilde(cuda(A), cuda(v), trans=trans).cpu().numpy()
        wo = olu.apply_atilde_t(A, Fg, v) if trans else olu.apply_atilde(A, Fg, v)
        bound = 64 * U_FF * _ff_bound(Fg, A, v, trans, True)
        assert np.all(np.abs(w - wo) <= bound), (trans, np.max(np.abs(w - wo) / bound))
    F.close()


@pytest.mark.parametrize("n,fmt", [(33, "bf16"), (300, "fp16"), (1001, "bf16")])
def test_apply_minv_and_atilde_dd(G, n, fmt):
    """u_a = double-double (the paper's u^2 for u = FP64): M^-1 v, M^-1 A v and their transposes
    against the oracle's double-double substitution on the same factors. Both carry about 106
    bits (times the conditioning of the factors, kappa_2(A) = 1e6 here), so the results, rounded
    to FP64, agree elementwise to a couple of ulps; n = 33 and 1001 leave ragged 32-row blocks."""
    A = randsvd(n, 1e6, seed=9)
    F, Fg = _gpu_factors(G, A, fmt, ua="dd")
    rng = np.random.default_rng(10)
    u = UNIT_ROUNDOFF["fp64"]
    for trans in (False, True):
        v = rng.standard_normal(n)
        w = F.apply_minv(cuda(v), trans=trans).cpu().numpy()
        wo = olu.apply_minv_t(Fg, v, "dd") if trans else olu.apply_minv(Fg, v, "dd")
        assert np.all(np.abs(w - wo) <= 4 * u * np.abs(wo)), np.abs((w - wo) / wo).max()
        w = F.apply_atilde(cuda(A), cuda(v), trans=trans).cpu().numpy()
        wo = olu.apply_atilde_t(A, Fg, v, "dd") if trans else olu.apply_atilde(A, Fg, v, "dd")
        assert np.all(np.abs(w - wo) <= 4 * u * np.abs(wo)), np.abs((w - wo) / wo).max()
    F.close()


@pytest.mark.parametrize("d", [1, 2, 5, 12, 30, 50, 112])
@pytest.mark.parametrize("largest", [0, 1])
@pytest.mark.parametrize("eig_prec", ["fp32", "fp64"])
def test_small_eig(G, d, largest, eig_prec):
    """The harmonic Ritz eigen-solver: eigenvalues from Hessenberg QR in FP32 (the default; they
    steer only the selection and the shifts) or FP64, eigenvectors by FP64 inverse iteration, so
    the eigenvalues match to the QR's precision times their condition and P spans an invariant
    subspace to FP64 accuracy either way."""
    from scipy.optimize import linear_sum_assignment
    rng = np.random.default_rng(d + 100 * largest)
    M = rng.standard_normal((d, d))
    k = min(10, max(1, d - 1))
    wr, wi, P, failed = G.small_eig(M, k, largest, 200, eig_prec=eig_prec)
    assert not failed
    lam = np.linalg.eigvals(M)
    got = wr + 1j * wi
    dist = np.abs(got[:, None] - lam[None, :])
    r, c = linear_sum_assignment(dist)
    tol = 1e-4 if eig_prec == "fp32" else 1e-10
    assert dist[r, c].max() <= tol * max(1.0, np.abs(lam).max())
    # P spans an invariant subspace whose eigenvalues are the selected ones
    T = np.linalg.lstsq(P, M @ P, rcond=None)[0]
    assert np.linalg.norm(M @ P - P @ T) <= 1e-9 * max(1.0, np.linalg.norm(M @ P))
    mags = np.sort(np.abs(np.linalg.eigvals(T)))
    allm = np.sort(np.abs(lam))
    want = allm[::-1][:P.shape[1]] if largest else allm[:P.shape[1]]
    assert np.allclose(np.sort(mags), np.sort(want), rtol=1e-8, atol=1e-12)
    assert abs(P.shape[1] - k) <= 1


def _near_tie_matrix(rng, d, k, gap, pair_at_boundary):
    """Real d x d matrix with well-conditioned eigenvectors whose eigenvalue magnitudes are
    distinct except for a near tie (relative gap ``gap``) straddling the k-th place: either two
    real eigenvalues of opposite sign, or a real eigenvalue and a conjugate pair."""
    mags = list(np.geomspace(0.5, 40.0, d))
    blocks, vals = [], []
    i = 0
    while len(vals) < d:
        if len(vals) == k - 1:
            # places k and k+1: the near tie
            base = mags[len(vals)]
            if pair_at_boundary and len(vals) + 3 <= d:
                vals += [base]
                blocks.append(np.array([[base]]))
                r = base * (1 + gap)
                a, b = r * np.cos(1.0), r * np.sin(1.0)
                vals += [complex(a, b), complex(a, -b)]
                blocks.append(np.array([[a, b], [-b, a]]))
            else:
                vals += [base, -base * (1 + gap)]
                blocks.append(np.array([[base]]))
                blocks.append(np.array([[-base * (1 + gap)]]))
            continue
        m = mags[len(vals)]
        sgn = 1.0 if rng.random() < 0.5 else -1.0
        vals.append(sgn * m)
        blocks.append(np.array([[sgn * m]]))
    D = np.zeros((d, d))
    o = 0
    for bl in blocks:
        q = bl.shape[0]
        D[o:o + q, o:o + q] = bl
        o += q
    D = D[:d, :d]
    Q = np.linalg.qr(rng.standard_normal((d, d)))[0]
    X = Q @ (np.eye(d) + 0.1 * np.triu(rng.standard_normal((d, d)), 1) / np.sqrt(d))
    return X @ D @ np.linalg.inv(X)


@pytest.mark.parametrize("eig_prec,gap", [("fp32", 1e-4), ("fp64", 1e-9)])
@pytest.mark.parametrize("pair_at_boundary", [False, True])
@pytest.mark.parametrize("largest", [0, 1])
def test_small_eig_near_ties_select_oracle_subspace(G, eig_prec, gap, pair_at_boundary, largest):
    """Near ties in |theta| at the k-th place: the eigenvalues that steer the selection (FP32 by
    default, FP64 with GIR_FLAG_EIG_FP64) pick the same eigenvectors as the oracle's FP64
    selection (numpy eig + the pair rule), so P spans the oracle's subspace. FP32 separates
    relative gaps of 1e-4 on well-conditioned eigenvalues; ties closer than FP32's accuracy need
    the FP64 iteration, shown here at 1e-9."""
    from oracle.gcrodr import select_harmonic
    import scipy.linalg as sla
    d, k = 30, 8
    for trial in range(4):
        rng = np.random.default_rng(1000 * trial + 10 * largest + pair_at_boundary)
        kk = (d - k) if largest else k          # the near tie straddles the k-th selected place
        M = _near_tie_matrix(rng, d, kk, gap, pair_at_boundary)
        wr, wi, P, failed = G.small_eig(M, k, largest, 50, eig_prec=eig_prec)
        assert not failed
        theta, Z = np.linalg.eig(M)
        Po = select_harmonic(1.0 / theta if largest else theta, Z, k, d, 50)
        assert P.shape[1] == Po.shape[1]
        ang = sla.subspace_angles(P, Po)
        assert ang.max() <= 1e-8, (trial, ang.max())


def _tile_scale(vmax):
    """Power-of-two s with vmax * s in (224, 448] (the block scale of the FP8 model)."""
    return 1.0 if vmax == 0 else 2.0 ** np.floor(np.log2(448.0 / vmax))


def _assert_e4m3_tiles(X, mask, row0=0, col0=0):
    """Every 128 x 128 tile (global grid) of X restricted to mask holds e4m3 values times the
    reciprocal of a power-of-two scale derived from the tile's largest stored magnitude."""
    m, n = X.shape
    for r in range(0, m, 128):
        for c in range(0, n, 128):
            blk = X[r:r + 128, c:c + 128][mask[r:r + 128, c:c + 128]]
            if blk.size == 0:
                continue
            s = _tile_scale(np.abs(blk).max())
            for ss in (s, 2 * s):        # a tile maximum that rounded down to 224 / s also fits 2 s
                if np.array_equal(round_to(blk * ss, "e4m3"), blk * ss):
                    break
            else:
                raise AssertionError(f"tile ({r}, {c}) is not e4m3 under scale {s}")


@pytest.mark.parametrize("n", [200, 300, 517])
def test_factor_properties_fp8(G, n):
    """FP8-E4M3 u_f with 128 x 128 power-of-two tile scales: the factors satisfy the u_f backward
    error bound of the oracle's block model (128-wide FP32 block columns), |L| <= 1, and every
    stored tile is an e4m3 tile under its scale."""
    A = randsvd(n, 1e2, seed=n)
    F, Fg = _gpu_factors(G, A, "e4m3")
    Fo = olu.lu_block(A, "e4m3", w=32)
    assert np.all(Fg.R == 1.0) and np.all(Fg.S == 1.0) and Fg.mu == 1.0
    E = np.abs(A[Fg.perm] - Fg.L @ Fg.U).max() / (np.abs(Fg.L) @ np.abs(Fg.U)).max()
    Eo = np.abs(A[Fo.perm] - Fo.L @ Fo.U).max() / (np.abs(Fo.L) @ np.abs(Fo.U)).max()
    u8 = UNIT_ROUNDOFF["e4m3"]
    assert E <= 8 * u8 and E <= 4 * Eo + u8
    assert np.abs(np.tril(Fg.L, -1)).max() <= 1.0
    strict = np.tril(np.ones((n, n), bool), -1)
    _assert_e4m3_tiles(np.tril(Fg.L, -1), strict)
    # U: the diagonal tiles (upper part) and the tiles right of them are rounded separately
    for c0 in range(0, n, 128):
        c1 = min(n, c0 + 128)
        top = Fg.U[c0:c1, c0:c1]
        _assert_e4m3_tiles(top, np.triu(np.ones_like(top, bool)))
        if c1 < n:
            _assert_e4m3_tiles(Fg.U[c0:c1, c1:], np.ones((c1 - c0, n - c1), bool))
    F.close()


@pytest.mark.parametrize("n,ld", [(1, 1), (7, 9), (300, 300), (1001, 1004)])
def test_adjoint_grad_a(G, n, ld):
    """dA = -lambda x^T: one FP64 product per entry, so bit-identical to numpy's outer product."""
    rng = np.random.default_rng(n)
    lam, x = rng.standard_normal(n), rng.standard_normal(n)
    dA = torch.full((n, ld), 7.0, dtype=torch.float64, device="cuda")
    lib = G.load()
    lam_d, x_d = cuda(lam), cuda(x)
    st = lib.gir_adjoint_grad_a(lam_d.data_ptr(), x_d.data_ptr(), n, dA.data_ptr(), ld, None)
    torch.cuda.synchronize()
    assert st == 0
    got = dA.cpu().numpy()
    assert np.array_equal(got[:, :n], -np.outer(lam, x))
    assert np.all(got[:, n:] == 7.0)
