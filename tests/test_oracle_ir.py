"""Pins of oracle.ir: the paper's tables and bounds, special cases, gradients and status paths."""
import numpy as np
import pytest

from oracle.ir import (Params, solve, exact_solution, adjoint_gradients, normwise_berr,
                       forward_err, batch_solve)
from oracle.formats import UNIT_ROUNDOFF
from oracle import lu as lum
from synth import prolate, randsvd, convdiff, rhs_uniform, normal_vector
from conftest import read_golden


def _steps(s):
    return None if s == "-" else [int(v) for v in s.split(",")]


def _paper_run(alpha, triple, k):
    A = prolate(100, alpha)
    b = np.ones(100)
    if triple == "sdq":
        p = Params(uf="fp32", u="fp64", ur="dd", ua="u2", m=16, k=k, tau=1e-8, imax=2,
                   target=0.0, lu_mode="chop", max_its=2000)
    else:
        p = Params(uf="fp16", u="fp32", ur="fp64", ua="u2", m=16, k=k, tau=1e-4, imax=2,
                   target=0.0, lu_mode="chop", max_its=2000)
    return solve(A, b, p)[1]


def test_table5_first_two_steps():
    """Table 5 (s,d,q), (m,k) = (16,4): per-step counts of the first two refinement steps
    within +-1 of the paper and recycling never worse; exact equality is unpinned (the
    paper's factorization used MATLAB's blocked single-precision LU)."""
    for alpha, g, r in read_golden("table5_prolate_sdq.txt"):
        g, r = _steps(g), _steps(r)
        ig = _paper_run(float(alpha), "sdq", 0)
        ir = _paper_run(float(alpha), "sdq", 4)
        assert ig.its[0] == ir.its[0]                     # step 1 has no recycle space yet
        for got, ref in ((ig.its[:2], g[:2]), (ir.its[:2], r[:2])):
            assert all(abs(a - b) <= 1 for a, b in zip(got, ref)), (alpha, got, ref)
        assert ir.its[1] <= ig.its[1]
        if r[1] < g[1]:
            assert ir.its[1] < ig.its[1]


def test_table6_first_two_steps():
    """Table 6 (h,s,d), (m,k) = (16,5): the three rows whose first step takes under 10
    iterations reproduce the paper exactly in the first two steps."""
    rows = read_golden("table6_prolate_hsd.txt")[:3]
    for alpha, g, r in rows:
        g, r = _steps(g), _steps(r)
        ig = _paper_run(float(alpha), "hsd", 0)
        ir = _paper_run(float(alpha), "hsd", 5)
        assert ig.its[:2] == g[:2]
        assert ir.its[:2] == r[:2]


def test_table4_prolate_condition_numbers():
    for alpha, kinf, k2 in read_golden("table4_prolate_kappa.txt")[:4]:
        A = prolate(100, float(alpha))
        ki = np.linalg.norm(A, np.inf) * np.linalg.norm(np.linalg.inv(A), np.inf)
        s = np.linalg.svd(A, compute_uv=False)
        assert abs(ki / float(kinf) - 1) < 0.006, alpha
        assert abs(s[0] / s[-1] / float(k2) - 1) < 0.006, alpha


def test_randsvd_singular_values():
    A = randsvd(120, 1e6, seed=4)
    s = np.linalg.svd(A, compute_uv=False)
    ref = 1e6 ** (-np.arange(120) / 119.0)
    assert np.allclose(s, ref, rtol=1e-8)


# Table 2: (u_f, u, u_r, kappa_inf limit).  (h,h,s) is skipped (u = half is not a working precision here).
TABLE2 = {
    ("fp16", "fp32", "fp64"): 1e8,
    ("fp16", "fp64", "dd"): 1e12,
    ("fp32", "fp32", "fp64"): 1e8,
    ("fp32", "fp64", "dd"): 1e16,
}


@pytest.mark.parametrize("triple", list(TABLE2))
def test_table2_limiting_accuracy(triple):
    """Below the kappa_inf limit of Table 2, unrestarted GMRES-IR (m = n, Section 1) reaches
    a normwise backward error and forward error at the level of u."""
    uf, u, ur = triple
    n = 60
    kappa2 = TABLE2[triple] / 1e3
    A = randsvd(n, kappa2, seed=7)
    kinf = np.linalg.norm(A, np.inf) * np.linalg.norm(np.linalg.inv(A), np.inf)
    assert kinf < TABLE2[triple]
    xt = normal_vector(n, 8)
    b = A @ xt
    xs = exact_solution(A, b)
    # a fixed number of refinement steps (target 0) so the iteration reaches its limiting accuracy
    p = Params(uf=uf, u=u, ur=ur, ua="u2", m=n, k=0, tau=1e-4 if u == "fp32" else 1e-8,
               imax=6, target=0.0, lu_mode="chop", max_its=n)
    x, info, _, _ = solve(A, b, p, xstar=xs)
    uu = UNIT_ROUNDOFF[u]
    assert normwise_berr(A, x, b) <= 10 * uu
    assert forward_err(x, xs) <= 10 * (uu + kinf * UNIT_ROUNDOFF[ur])


def test_tiny_fp64_equals_direct_solve():
    rng = np.random.default_rng(9)
    for n in (1, 2, 5, 8):
        A = rng.standard_normal((n, n)) + n * np.eye(n)
        b = rng.standard_normal(n)
        p = Params(uf="fp64", u="fp64", ur="dd", ua="u", m=n, k=min(2, n - 1), tau=1e-12,
                   imax=5, lu_mode="block", lu_w=4)
        x, info, _, _ = solve(A, b, p)
        xs = np.linalg.solve(A, b)
        assert np.abs(x - xs).max() <= 1e-14 * np.linalg.cond(A) * np.abs(xs).max()


def test_step_one_identical_with_and_without_recycling():
    A = randsvd(200, 1e4, seed=0)
    b = rhs_uniform(200, 0)
    base = dict(uf="fp16", u="fp32", ur="fp64", ua="u2", m=60, tau=1e-4, imax=1, target=0.0)
    x0, i0, _, _ = solve(A, b, Params(k=0, **base))
    x5, i5, _, _ = solve(A, b, Params(k=5, **base))
    assert i0.its[0] < 60                       # first cycle converged
    assert i0.its == i5.its and np.array_equal(x0, x5)


def test_recycling_helps_randsvd():
    """Sum of iterations over steps >= 2 is smaller with recycling (Tables 8-11 qualitatively)."""
    A = randsvd(200, 1e6, seed=0)
    b = rhs_uniform(200, 0)
    base = dict(uf="fp16", u="fp32", ur="fp64", ua="u2", m=60, tau=1e-4, imax=2, target=0.0, max_its=600)
    _, i0, _, _ = solve(A, b, Params(k=0, **base))
    _, i5, _, _ = solve(A, b, Params(k=10, **base))
    assert len(i0.its) == len(i5.its) == 2
    assert sum(i5.its[1:]) < sum(i0.its[1:])


def test_carry_modes_agree():
    A = prolate(100, 0.455)
    b = np.ones(100)
    base = dict(uf="fp32", u="fp64", ur="dd", ua="u", m=16, k=4, tau=1e-8, imax=4)
    x0, i0, _, _ = solve(A, b, Params(carry_mode=0, **base))
    x1, i1, _, _ = solve(A, b, Params(carry_mode=1, **base))
    assert i0.converged and i1.converged
    assert all(abs(a - c) <= 1 for a, c in zip(i0.its, i1.its))
    # both are backward stable; solutions agree to the conditioning (kappa_inf ~ 3e11 here)
    kinf = np.linalg.norm(A, np.inf) * np.linalg.norm(np.linalg.inv(A), np.inf)
    assert np.abs(x0 - x1).max() <= 10 * kinf * UNIT_ROUNDOFF["fp64"] * np.abs(x0).max()


def test_adjoint_gradients_match_finite_differences():
    n = 30
    A = convdiff(5, 50.0)[:25, :25] if False else randsvd(n, 1e3, seed=11)
    b = rhs_uniform(n, 4)
    xt = normal_vector(n, 5)
    p = Params(uf="bf16", u="fp64", ur="dd", ua="u", m=20, k=5, tau=1e-10, imax=10)

    def loss(Am, bm):
        x = solve(Am, bm, p)[0]
        return float(np.sum((x - xt) ** 2)), x

    L0, x = loss(A, b)
    g = 2 * (x - xt)
    db, dA, info = adjoint_gradients(A, b, x, g, p)
    assert info.converged
    # against the exact gradient of the FP64 solve
    lam = np.linalg.solve(A.T, g)
    assert np.abs(db - lam).max() <= 1e-8 * np.abs(lam).max()
    h = 1e-6
    for (i, j) in [(0, 0), (3, 7), (29, 1)]:
        Ap, Am = A.copy(), A.copy()
        Ap[i, j] += h
        Am[i, j] -= h
        fd = (loss(Ap, b)[0] - loss(Am, b)[0]) / (2 * h)
        assert abs(fd - dA[i, j]) <= 1e-5 * max(1.0, abs(fd))
    for i in (0, 17):
        bp, bm = b.copy(), b.copy()
        bp[i] += h
        bm[i] -= h
        fd = (loss(A, bp)[0] - loss(A, bm)[0]) / (2 * h)
        assert abs(fd - db[i]) <= 1e-5 * max(1.0, abs(fd))


def test_convdiff_structure():
    A = convdiff(10, 50.0)
    assert A.shape == (100, 100)
    # five-point stencil, upwind: row sums are h*(bx+by) in the interior
    h = 1 / 11
    r = 5 * 10 + 5
    assert np.count_nonzero(A[r]) == 5
    assert np.isclose(A[r].sum(), 0.0)
    assert np.isclose(A[r, r - 10], -1 - h * 50 / np.sqrt(2))


def test_status_paths():
    A = randsvd(40, 1e3, seed=1)
    p = Params(uf="bf16", u="fp64", m=10, k=3, imax=1, tau=1e-8)
    b = rhs_uniform(40, 1)
    x, info, _, _ = solve(A, b, p)
    assert not info.converged and info.status == "NOT_CONVERGED"
    bn = b.copy()
    bn[3] = np.nan
    x, info, _, _ = solve(A, bn, Params(uf="bf16", u="fp64", m=10, k=3, imax=3))
    assert info.status == "NONFINITE"
    As = A.copy()
    As[:, 5] = 0.0
    with pytest.raises(lum.SingularError):
        solve(As, b, p)


def test_batch_independent():
    As = [randsvd(n, 1e3, seed=n) for n in (20, 33)]
    bs = [rhs_uniform(A.shape[0], 1) for A in As]
    p = Params(uf="bf16", u="fp64", m=15, k=4, imax=10)
    res = batch_solve(As, bs, p)
    for (x, info), A, b in zip(res, As, bs):
        assert info.converged
        assert np.array_equal(x, solve(A, b, p)[0])


def test_componentwise_berr_oettli_prager():
    """The componentwise backward error (Table 2, middle column) is the smallest eps with
    (A + dA) x = b + db, |dA| <= eps |A|, |db| <= eps |b| (Oettli-Prager): the perturbation
    dA = D |A| diag(sign x), db = -D |b| with D = diag(r_i / (|A||x| + |b|)_i) attains it."""
    from oracle.ir import componentwise_berr
    rng = np.random.default_rng(21)
    n = 40
    A = rng.standard_normal((n, n))
    x = rng.standard_normal(n)
    b = A @ x + 1e-6 * rng.standard_normal(n)
    r = b - A @ x
    om = componentwise_berr(A, x, b, r)
    den = np.abs(A) @ np.abs(x) + np.abs(b)
    D = r / den
    dA = D[:, None] * np.abs(A) * np.sign(x)[None, :]
    db = -D * np.abs(b)
    assert np.abs((A + dA) @ x - (b + db)).max() <= 1e-13 * den.max()
    assert np.all(np.abs(dA) <= om * np.abs(A) * (1 + 1e-15))
    assert np.all(np.abs(db) <= om * np.abs(b) * (1 + 1e-15))
    # row i0 needs eps >= |r_i0| / den_i0 = om for any admissible perturbation
    assert om == pytest.approx(np.abs(D).max(), rel=1e-15)
    # normwise <= componentwise (|r_i| <= om (||A|| ||x|| + ||b||) for every row)
    assert normwise_berr(A, x, b, r) <= om
    # a diagonal system by hand: r = (0.5, 0, 0), |A||x| + |b| = (4.5, 6, 0), and 0/0 counts 0
    Ad = np.diag([2.0, -3.0, 0.0])
    xd = np.array([1.0, 1.0, 5.0])
    bd = np.array([2.5, -3.0, 0.0])
    assert componentwise_berr(Ad, xd, bd) == pytest.approx(0.5 / 4.5, rel=1e-15)
    assert componentwise_berr(np.zeros((1, 1)), np.ones(1), np.zeros(1)) == 0.0


def test_sir_error_recursion():
    """Algorithm 1 with an LU solve: x_{i+1} = x_i + M^-1 (b - A x_i), so the error obeys
    e_{i+1} = (I - M^-1 A) e_i up to rounding (M = the u_f factors, applied in FP64)."""
    n = 30
    A = randsvd(n, 1e2, seed=4)
    xs = normal_vector(n, 5)
    b = A @ xs
    p = Params(uf="bf16", u="fp64", ur="dd", ua="fp64", imax=1, target=0.0, solver="sir")
    F = lum.lu_block(A, "bf16", w=64)
    x0 = lum.apply_minv(F, b, "fp64")
    x1, info, _, _ = solve(A, b, p, F=F)
    Minv = np.column_stack([lum.apply_minv(F, e, "fp64") for e in np.eye(n)])
    G = np.eye(n) - Minv @ A
    e0, e1 = x0 - xs, x1 - xs
    assert np.linalg.norm(G @ e0 - e1) <= 1e-6 * np.linalg.norm(e0)
    assert np.linalg.norm(e1) < 0.5 * np.linalg.norm(e0)
    assert info.its == [0] and info.steps == 1


def test_sir_condition_limit():
    """SIR converges when kappa_inf(A) u_f < 1 and fails far above it, where GMRES-IR with
    the same factors still converges (the constraint the paper sets against GMRES-IR)."""
    n = 60
    b = rhs_uniform(n, 3)
    ok = randsvd(n, 10.0, seed=2)
    assert np.linalg.cond(ok, np.inf) * UNIT_ROUNDOFF["bf16"] < 1
    x, info, _, _ = solve(ok, b, Params(uf="bf16", u="fp64", ur="fp64", ua="fp64", imax=10, solver="sir"))
    assert info.converged and info.berr[-1] <= 2 * UNIT_ROUNDOFF["fp64"]
    hard = randsvd(n, 1e6, seed=2)
    x, info, _, _ = solve(hard, b, Params(uf="bf16", u="fp64", ur="fp64", ua="fp64", imax=10, solver="sir"))
    assert not info.converged and info.status in ("NOT_CONVERGED", "NONFINITE")
    x, info, _, _ = solve(hard, b, Params(uf="bf16", u="fp64", ur="fp64", ua="fp64", m=n, k=0, imax=10))
    assert info.converged


def test_stop_componentwise():
    """stop='cw' ends only when both the normwise and the componentwise backward errors meet
    the target; omega_i >= eta_i at every step."""
    A = randsvd(80, 1e4, seed=6)
    b = rhs_uniform(80, 6)
    p = Params(uf="bf16", u="fp64", ur="dd", ua="fp64", m=20, k=5, imax=10, stop="cw")
    x, info, _, _ = solve(A, b, p)
    assert info.converged
    assert info.cberr[-1] <= 2 * UNIT_ROUNDOFF["fp64"] and info.berr[-1] <= 2 * UNIT_ROUNDOFF["fp64"]
    assert all(c >= e for c, e in zip(info.cberr, info.berr))
    assert len(info.cberr) == len(info.berr) == info.steps + 1


def test_knee_k_gives_fewest_iterations():
    """Section 5 (Fig. 2): recycling the whole first-step subspace, k = its_1 - 1, gives the
    fewest total GMRES iterations. k_mode='knee' picks that k from the first step and then equals
    the fixed-k run with the same k."""
    A = randsvd(200, 1e4, seed=0)
    b = rhs_uniform(200, 0)
    base = dict(uf="bf16", u="fp64", ur="fp64", ua="u", m=100, tau=1e-8, imax=10, lu_w=32)
    xk, ik, _, _ = solve(A, b, Params(k=0, k_mode="knee", **base))
    assert ik.converged and len(ik.its) >= 2
    its1 = ik.its[0]
    assert ik.k_used == [its1 - 1] * len(ik.its)
    for k in (0, 5, 10, 20):
        _, i, _, _ = solve(A, b, Params(k=k, **base))
        assert i.its[0] == its1 and ik.total < i.total, (k, i.its, ik.its)
    xf, i_f, _, _ = solve(A, b, Params(k=its1 - 1, **base))
    assert i_f.its == ik.its and np.array_equal(xf, xk)
    # the cap: k never exceeds k_max
    _, ic, _, _ = solve(A, b, Params(k=0, k_mode="knee", k_max=7, **base))
    assert ic.k_used[0] == 7
