"""The batch as one persistent kernel launch (gir_batch_solve with engine="persistent"; left to
choose, the routing takes it for batches of many systems): every system of an uneven batch against
its own oracle solve, the same batch through the worker-stream engine, the other precision triples
and options the kernel implements, per-system failure statuses, and a batch shaped like the
512-system workload (n up to 4096) checked by properties that hold at any size.

Tolerances are those of the single-system parity tests: same convergence status, final normwise
backward error <= 4x the oracle's (floored at the unit roundoff of u), total GMRES iterations within
+-10% (+1), refinement steps within one, and Table 2's forward error for u = FP64."""
import numpy as np
import pytest
import torch

from oracle.ir import Params as OP, solve as osolve, normwise_berr, forward_err, exact_solution
from oracle.formats import UNIT_ROUNDOFF
from synth import randsvd, prolate, rhs_uniform, normal_vector

from test_gpu_solve import assert_parity, cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2201_09827_gb300 as p
    p.load()
    return p


def assert_parity_steps(A, b, x, info, xo, io, u="fp64", ur="fp64"):
    """assert_parity, except that the GPU may take one refinement step more than the oracle: at the
    2u target the last step can end on either side of it, and the GPU applies A~ in float-float
    (2^-46) where the oracle uses FP64. Then the iterations of the steps both took must agree."""
    if io.converged and info.status == 0 and info.ir_steps == io.steps + 1:
        common = sum(info.its[:io.steps])
        assert abs(common - io.total) <= 0.1 * io.total + 1, (info.its, io.its)
        assert normwise_berr(A, x, b) <= 4 * max(normwise_berr(A, xo, b), UNIT_ROUNDOFF[u])
        return
    assert_parity(A, b, x, info, xo, io, u, ur)


def _batch(count, lo, hi, klo, khi, seed, edge=()):
    rng = np.random.default_rng(seed)
    sizes = list(edge) + [int(v) for v in rng.integers(lo, hi, count - len(edge))]
    kappas = 10.0 ** rng.uniform(klo, khi, len(sizes))
    As = [randsvd(n, kp, seed=seed * 1000 + i) for i, (n, kp) in enumerate(zip(sizes, kappas))]
    bs = [A @ normal_vector(A.shape[0], seed * 1000 + 500 + i) for i, A in enumerate(As)]
    return sizes, kappas, As, bs


def _oracle(uf="bf16", u="fp64", ur="fp64", m=30, k=8, tau=1e-8, target=None, carry=1, k_mode="fixed",
            max_its=None, order="fma", basis=None):
    """The oracle's settings for the persistent kernel: 32-column panels and, by default, the
    'fma' summation order of the block LU, which is the order the kernel's FP32 updates use."""
    return OP(uf=uf, u=u, ur=ur, ua="u2" if u != "fp64" else "u", m=m, k=k, tau=tau, imax=10, target=target,
              lu_w=32, lu_order=order, max_its=max_its or 20 * m, carry_mode=carry, k_mode=k_mode, basis=basis)


def test_persistent_batch_parity_with_oracle(pkg):
    """40 systems, n from 1 to 1500 (the edge orders 1, 2, 31, 32, 33, 64, 65 and 97 around the
    32-row blocks and the 128-wide update tiles, then random), kappa_2 in [1e2, 10^3.7] (kappa u_f
    up to 20, where the iteration counts follow the rounding of the factors), BF16 LU,
    GCRO-DR(30, 8), target 2u, at most 300 Arnoldi steps per refinement step: one launch, each
    system matching its own oracle solve."""
    sizes, _, As, bs = _batch(40, 16, 1500, 2.0, 3.7, seed=7, edge=(1, 2, 31, 32, 33, 64, 65, 97))
    prm = pkg.Params(uf="bf16", u="fp64", ur="fp64", m=30, k=8, tau=1e-8, imax=10, target_berr=-1.0,
                     max_its=300)
    before = pkg.launch_count()
    xs, infos, st = pkg.batch_solve([cuda(A) for A in As], [cuda(b) for b in bs], prm, engine="persistent")
    assert pkg.launch_count() - before == 1, "the whole batch is one kernel launch"
    assert st in (0, 1)
    op = _oracle(max_its=300)
    for A, b, x, info in zip(As, bs, xs, infos):
        xo, io, _, _ = osolve(A, b, op)
        assert_parity_steps(A, b, x.cpu().numpy(), info, xo, io)
        assert info.ms_factor >= 0.0 and info.ms_solve >= 0.0


def test_persistent_batch_reference_order(pkg):
    """Well-conditioned systems (kappa_2 in [1e2, 1e3]) also match the oracle's reference 'dot'
    summation order of the LU: the order changes the iteration counts only where kappa u_f >> 1."""
    sizes, _, As, bs = _batch(12, 30, 1200, 2.0, 3.0, seed=9)
    prm = pkg.Params(uf="bf16", u="fp64", ur="fp64", m=30, k=8, tau=1e-8, imax=10, target_berr=-1.0)
    xs, infos, st = pkg.batch_solve([cuda(A) for A in As], [cuda(b) for b in bs], prm, engine="persistent")
    op = _oracle(order="dot")
    for A, b, x, info in zip(As, bs, xs, infos):
        xo, io, _, _ = osolve(A, b, op)
        assert_parity_steps(A, b, x.cpu().numpy(), info, xo, io)


def test_persistent_matches_stream_engine(pkg):
    """The same 24 systems through both engines: equal statuses, iteration counts within 10% and
    backward errors within 4x of each other."""
    sizes, _, As, bs = _batch(24, 40, 900, 2.0, 3.0, seed=11)
    prm = pkg.Params(uf="bf16", u="fp64", ur="fp64", m=30, k=8, tau=1e-8, imax=10, target_berr=1e-15)
    Ad, bd = [cuda(A) for A in As], [cuda(b) for b in bs]
    xp, ip, sp = pkg.batch_solve(Ad, bd, prm, engine="persistent")
    xq, iq, sq = pkg.batch_solve(Ad, bd, prm, engine="streams")
    assert sp == sq
    for A, b, x1, i1, x2, i2 in zip(As, bs, xp, ip, xq, iq):
        assert i1.status == i2.status
        assert abs(i1.total_its - i2.total_its) <= 0.1 * i2.total_its + 1
        b1, b2 = normwise_berr(A, x1.cpu().numpy(), b), normwise_berr(A, x2.cpu().numpy(), b)
        assert b1 <= 4 * max(b2, 2.0 ** -53) and b1 <= 1e-15


@pytest.mark.parametrize("uf,u,ur", [("fp16", "fp64", "fp64"), ("bf16", "fp64", "dd"), ("fp16", "fp32", "fp64")])
def test_persistent_precision_triples(pkg, uf, u, ur):
    """FP16 with its diagonal scaling, a double-double residual, and FP32 working precision
    (rounded x, r, d and basis vectors, tau = 1e-4): 12 systems each against the oracle."""
    tau = 1e-4 if u == "fp32" else 1e-8
    sizes, _, As, bs = _batch(12, 20, 700, 2.0, 3.0, seed=13)
    prm = pkg.Params(uf=uf, u=u, ur=ur, m=30, k=8, tau=tau, imax=10, target_berr=-1.0)
    xs, infos, st = pkg.batch_solve([cuda(A) for A in As], [cuda(b) for b in bs], prm, engine="persistent")
    op = _oracle(uf=uf, u=u, ur=ur, tau=tau)
    for A, b, x, info in zip(As, bs, xs, infos):
        xo, io, _, _ = osolve(A, b, op)
        assert_parity_steps(A, b, x.cpu().numpy(), info, xo, io, u, ur)


def test_persistent_prolate_recycling(pkg):
    """Prolate Toeplitz systems (u_r = dd, GCRO-DR(30, 10), target 2u), two of them where the
    recycled space cuts the second refinement step (the oracle gives 14 (11, 3) against 23 (11, 12)
    at n = 400, w = 0.49): GPU and oracle agree per system with k = 10 and k = 0 (status, backward
    error, iterations), and on the GPU too k = 10 needs fewer iterations on those two. These
    matrices have kappa_inf from 6e4 to 3e11: the backward-error stop ends the run while the forward
    error is about kappa_inf eta, and how far below that it lies depends on the accuracy of the last
    correction, which the float-float operator (2^-46) bounds; so the forward error is checked
    against kappa_inf eta, not against the oracle's FP64-operator value."""
    cases = [(400, 0.49), (600, 0.495), (300, 0.485), (800, 0.4975)]
    As = [prolate(n, w) for n, w in cases]
    bs = [rhs_uniform(n, 3 + i) for i, (n, _) in enumerate(cases)]
    total = {}
    for k in (10, 0):
        prm = pkg.Params(uf="bf16", u="fp64", ur="dd", m=30, k=k, tau=1e-8, imax=10, target_berr=-1.0)
        xs, infos, st = pkg.batch_solve([cuda(A) for A in As], [cuda(b) for b in bs], prm, engine="persistent")
        op = _oracle(ur="dd", k=k)
        for A, b, x, info in zip(As, bs, xs, infos):
            xo, io, _, _ = osolve(A, b, op)
            xh = x.cpu().numpy()
            assert (info.status == 0) == io.converged
            be = normwise_berr(A, xh, b)
            assert be <= 4 * max(normwise_berr(A, xo, b), 2.0 ** -53)
            assert abs(info.total_its - io.total) <= 0.1 * io.total + 1, (info.its, io.its)
            kinf = np.linalg.norm(A, np.inf) * np.linalg.norm(np.linalg.inv(A), np.inf)
            assert forward_err(xh, exact_solution(A, b)) <= 2 * kinf * be + 2.0 ** -50
        total[k] = [i.total_its for i in infos]
    assert total[10][0] < total[0][0] and total[10][2] < total[0][2]


def test_persistent_carry_literal_and_adaptive_k(pkg):
    """carry_mode 0 (QR of A~ Y~ recomputed at every refinement step) and k = its_1 - 1
    (GIR_FLAG_ADAPTIVE_K, the oracle's 'knee' mode) against the oracle."""
    sizes, _, As, bs = _batch(8, 100, 600, 2.5, 3.5, seed=17)
    cases = [(dict(carry_mode=0), dict(carry=0)),
             (dict(flags=pkg.GIR_FLAG_ADAPTIVE_K), dict(k_mode="knee"))]
    for gkw, okw in cases:
        prm = pkg.Params(uf="bf16", u="fp64", ur="fp64", m=30, k=8, tau=1e-8, imax=10, target_berr=-1.0, **gkw)
        xs, infos, st = pkg.batch_solve([cuda(A) for A in As], [cuda(b) for b in bs], prm, engine="persistent")
        op = _oracle(**okw)
        for A, b, x, info in zip(As, bs, xs, infos):
            xo, io, _, _ = osolve(A, b, op)
            assert_parity_steps(A, b, x.cpu().numpy(), info, xo, io)


def test_persistent_eig_fp64_and_fp32_basis(pkg):
    """The two GCRO-DR options the kernel runs through the same device functions as the single-system
    path: FP64 Hessenberg QR for the harmonic Ritz eigenvalues (GIR_FLAG_EIG_FP64) and FP32 storage
    of the Krylov and recycle vectors (GIR_FLAG_BASIS_FP32, the oracle's basis='fp32'), 8 systems
    each against the oracle, target 1e-15."""
    sizes, _, As, bs = _batch(8, 200, 900, 2.0, 3.0, seed=19)
    from paper_2201_09827_gb300 import gir
    for flag, basis in ((gir.GIR_FLAG_EIG_FP64, None), (gir.GIR_FLAG_BASIS_FP32, "fp32")):
        prm = pkg.Params(uf="bf16", u="fp64", ur="fp64", m=30, k=8, tau=1e-8, imax=10, target_berr=1e-15,
                         flags=flag)
        xs, infos, st = pkg.batch_solve([cuda(A) for A in As], [cuda(b) for b in bs], prm, engine="persistent")
        op = _oracle(target=1e-15, basis=basis)
        for A, b, x, info in zip(As, bs, xs, infos):
            xo, io, _, _ = osolve(A, b, op)
            assert_parity_steps(A, b, x.cpu().numpy(), info, xo, io)


def test_persistent_status_paths(pkg):
    """A zero column (GIR_SINGULAR), a NaN entry (GIR_NONFINITE) and one refinement step with
    target 0 (GIR_NOT_CONVERGED) in one batch; the healthy systems beside them still converge."""
    from paper_2201_09827_gb300 import gir
    n = 150
    A = randsvd(n, 1e3, seed=2)
    As_ = A.copy()
    As_[:, 7] = 0.0
    An = A.copy()
    An[3, 3] = np.nan
    good = [randsvd(m, 1e2, seed=40 + m) for m in (90, 200)]
    mats = [As_, good[0], An, good[1]]
    bs = [rhs_uniform(M.shape[0], i) for i, M in enumerate(mats)]
    prm = pkg.Params(uf="bf16", m=30, k=8, tau=1e-8, imax=10, target_berr=-1.0)
    xs, infos, st = pkg.batch_solve([cuda(M) for M in mats], [cuda(b) for b in bs], prm, engine="persistent")
    assert infos[0].status == gir.GIR_SINGULAR
    assert infos[2].status == gir.GIR_NONFINITE
    assert infos[1].status == gir.GIR_OK and infos[3].status == gir.GIR_OK
    assert st == max(gir.GIR_SINGULAR, gir.GIR_NONFINITE)
    prm1 = pkg.Params(uf="bf16", m=30, k=8, tau=1e-8, imax=1, target_berr=0.0)
    xs, infos, st = pkg.batch_solve([cuda(good[0])], [cuda(bs[1])], prm1, engine="persistent")
    assert st == gir.GIR_NOT_CONVERGED and infos[0].ir_steps == 1
    with pytest.raises(ValueError):
        pkg.batch_solve([cuda(good[0])], [cuda(bs[1])], prm1, engine="other")
    with pytest.raises(gir.GirError):   # the kernel forced on a format it does not implement
        pkg.batch_solve([cuda(good[0])], [cuda(bs[1])], pkg.Params(uf="e4m3"), engine="persistent")


def test_persistent_batch_large_orders(pkg):
    """Systems shaped like the 512-system workload (n up to 4096, kappa_2 = 1e2..1e3, b = A x*):
    each converged system meets the backward-error target and Table 2's forward error, measured on
    the host in FP64 against x*; the largest also against its oracle solve (n = 2048)."""
    sizes = [4096, 3000, 2048, 1100, 257]
    As, xstars, bs = [], [], []
    for i, n in enumerate(sizes):
        A = randsvd(n, 10.0 ** (2 + (i % 2)), seed=300 + i)
        xs_ = normal_vector(n, 400 + i)
        As.append(A)
        xstars.append(xs_)
        bs.append(A @ xs_)
    prm = pkg.Params(uf="bf16", u="fp64", ur="fp64", m=30, k=8, tau=1e-8, imax=10, target_berr=-1.0)
    xs, infos, st = pkg.batch_solve([cuda(A) for A in As], [cuda(b) for b in bs], prm, engine="persistent")
    assert st == 0
    for A, b, x, xst, info, i in zip(As, bs, xs, xstars, infos, range(len(sizes))):
        xh = x.cpu().numpy()
        assert normwise_berr(A, xh, b) <= 4 * 2.0 ** -52
        kinf = A.shape[0] * 10.0 ** (2 + (i % 2))     # kappa_inf <= n kappa_2
        assert np.abs(xh - xst).max() / np.abs(xst).max() <= 10 * (2.0 ** -53 + kinf * 2.0 ** -53)
    i = sizes.index(2048)
    xo, io, _, _ = osolve(As[i], bs[i], _oracle())
    assert_parity(As[i], bs[i], xs[i].cpu().numpy(), infos[i], xo, io, "fp64")


def test_persistent_batch_max_order(pkg):
    """The kernel's order limit: n = 8192 and a ragged 7777 (both padded row pitches, the panel in
    global memory, the float-float y and split v filling 128 KB of shared memory), kappa_2 = 1e2,
    b = A x*, in one launch: both converge to the backward-error target (double-double residual on
    the device) with Table 2's forward error against x*."""
    from synth import randsvd_torch
    sizes = [8192, 7777]
    As, xst, bs = [], [], []
    for i, n in enumerate(sizes):
        A = randsvd_torch(n, 1e2, seed=600 + i, device="cuda")
        g = torch.Generator(device="cuda")
        g.manual_seed(700 + i)
        x = torch.randn(n, dtype=torch.float64, device="cuda", generator=g)
        As.append(A)
        xst.append(x)
        bs.append(A @ x)
    prm = pkg.Params(uf="bf16", u="fp64", ur="fp64", m=30, k=8, tau=1e-8, imax=10, target_berr=-1.0)
    xs, infos, st = pkg.batch_solve(As, bs, prm, engine="persistent")
    assert st == 0
    for A, b, x, xs_, n in zip(As, bs, xs, xst, sizes):
        eta, _ = pkg.backward_errors(A, x, b, "dd")
        assert eta <= 4 * 2.0 ** -52
        ferr = ((x - xs_).abs().max() / xs_.abs().max()).item()
        assert ferr <= 10 * (2.0 ** -53 + n * 1e2 * 2.0 ** -53)
