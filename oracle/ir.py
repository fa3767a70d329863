"""GMRES-IR and RGMRES-IR (Algorithms 2 and 4), the adjoint solve and batches; the general
iterative refinement of Algorithm 1 (SIR, correction by LU substitution) as a comparator.

RGMRES-IR, Algorithm 4, in order:
  1. LU factorization in precision u_f (``oracle.lu``).
  2. x0 = M^-1 b by substitution, stored in u.
  3. For i = 0 .. i_max - 1:
     r_i = b - A x_i in precision u_r; eta_i = ||r_i||_inf / (||A||_inf ||x_i||_inf + ||b||_inf);
     stop when converged; s = ||r_i||_inf; r^ = fl_u(r_i / s);
     solve A~ d = M^-1 r^ by GCRO-DR(m, k) with tolerance tau, A~ = M^-1 A applied in u_a;
     x_{i+1} = fl_u(x_i + s d).
  GMRES-IR (Algorithm 2) is the same loop with k = 0 (GCRO-DR(m, 0) is restarted GMRES(m)).

Readings of the paper taken here:
* "converged": eta_i <= target (normwise relative backward error); with ``stop='cw'`` also
  omega_i <= target (componentwise backward error, the middle column of Table 2); or, with
  ``stop='all'`` and a known exact solution, max(normwise BE, componentwise BE,
  forward error) <= u; the test is made on x_i before the i-th solve, so the number of
  GCRO-DR calls is the number of refinement steps.
* u_a: 'u2' means double the working precision (FP64 for u = FP32, double-double for
  u = FP64, Algorithm 4); 'u' means uniform precision (Section 4.3.1).
* x0: in the paper's every-operation-rounded mode the substitution is in u_f; for the
  block-FMA factorization it is done in FP64 and rounded to u.
* ``k_mode='knee'``: Section 5 reports the fewest total iterations for k = its_1 - 1, with its_1
  the first step's count (the whole first-step subspace recycled). The first GCRO-DR call
  fixes k this way when its first cycle converges; otherwise k stays as given.
* Recycle carry between refinement steps: ``carry_mode=0`` recomputes QR(A~ Y~)
  literally; ``carry_mode=1`` reuses (U_k, C_k), valid because A~ U_k = C_k and A~ does
  not change between steps.
* The adjoint solve A^T lambda = g runs the same loop on A^T with preconditioner M^T
  (operator M^-T A^T); gradients of a loss of x = A^-1 b are db = lambda, dA = -lambda x^T.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from .formats import round_to, UNIT_ROUNDOFF
from . import dd as ddm
from . import lu as lum
from .gcrodr import gcrodr


@dataclass
class Params:
    uf: str = "bf16"
    u: str = "fp64"
    ur: str = "fp64"
    ua: str = "u"          # 'u', 'u2', or an explicit precision name
    m: int = 30
    k: int = 10
    tau: float = 1e-8
    imax: int = 10
    target: float | None = None   # normwise backward error target (default 2u)
    stop: str = "berr"            # 'berr', 'cw' (normwise and componentwise) or 'all'
    solver: str = "gcrodr"        # correction solver: 'gcrodr' (Algorithm 4) or 'sir' (Algorithm 1)
    k_mode: str = "fixed"         # 'fixed', or 'knee': k = its_1 - 1 (capped at k_max), Section 5
    k_max: int = 64
    carry_mode: int = 0
    lu_mode: str = "block"        # 'block' or 'chop'
    lu_w: int = 64
    lu_order: str = "dot"         # FP32 summation order of the block LU's U12 and trailing update
    max_its: int | None = None    # Arnoldi steps per GCRO-DR call
    basis: str | None = None      # storage format of the Krylov and recycle basis vectors (None: u)


@dataclass
class IrInfo:
    its: list = field(default_factory=list)        # Arnoldi steps per refinement step
    carry_applies: list = field(default_factory=list)
    berr: list = field(default_factory=list)       # eta_i of x_0, x_1, ...
    cberr: list = field(default_factory=list)      # componentwise omega_i of x_0, x_1, ...
    ferr: list = field(default_factory=list)
    converged: bool = False
    steps: int = 0
    k_eff: list = field(default_factory=list)
    k_used: list = field(default_factory=list)     # recycle dimension per refinement step
    resid: list = field(default_factory=list)
    status: str = "NOT_CONVERGED"

    @property
    def total(self):
        return int(sum(self.its))

    def paper_format(self):
        """'total (s1,s2,...)' as printed in Tables 5-11, or '-' when not converged."""
        if not self.converged:
            return "-"
        return f"{self.total} ({','.join(str(i) for i in self.its)})"


def ua_precision(p: Params) -> str:
    if p.ua == "u2":
        return "fp64" if p.u == "fp32" else "dd"
    if p.ua == "u":
        return p.u
    return p.ua


def residual(A, x, b, ur):
    """r = b - A x in precision u_r ('fp64', 'dd' or 'fp32'), returned in FP64."""
    if ur == "dd":
        h, l = ddm.dd_residual(A, x, b)
        return h + l
    if ur == "fp32":
        return (np.float32(1) * b.astype(np.float32) - A.astype(np.float32) @ x.astype(np.float32)).astype(np.float64)
    return b - A @ x


def normwise_berr(A, x, b, r=None, normA=None):
    """eta = ||b - A x||_inf / (||A||_inf ||x||_inf + ||b||_inf); r given or computed in dd."""
    if r is None:
        r = residual(A, x, b, "dd")
    if normA is None:
        normA = np.max(np.sum(np.abs(A), axis=1))
    return float(np.max(np.abs(r)) / (normA * np.max(np.abs(x)) + np.max(np.abs(b))))


def componentwise_berr(A, x, b, r=None):
    if r is None:
        r = residual(A, x, b, "dd")
    den = np.abs(A) @ np.abs(x) + np.abs(b)
    with np.errstate(divide="ignore", invalid="ignore"):
        q = np.where(den > 0, np.abs(r) / den, np.where(r == 0, 0.0, np.inf))
    return float(np.max(q))


def forward_err(x, xstar):
    return float(np.max(np.abs(x - xstar)) / np.max(np.abs(xstar)))


def factor(A, p: Params):
    if p.lu_mode == "chop":
        return lum.lu_chop(A, p.uf)
    return lum.lu_block(A, p.uf, w=p.lu_w, order=p.lu_order)


def solve(A, b, p: Params, F=None, xstar=None, transpose=False, Y0=None):
    """RGMRES-IR (GMRES-IR for k = 0). Returns x, info, F, recycle (U, C).

    transpose=True solves A^T x = b with the preconditioner M^T (adjoint solve).
    Y0 optionally seeds the recycle space of the first refinement step.
    """
    A = np.asarray(A, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    if F is None:
        F = factor(A, p)
    Aop = A.T.copy() if transpose else A
    ua = ua_precision(p)
    fu = (lambda z: round_to(z, p.u))
    target = p.target if p.target is not None else 2.0 * UNIT_ROUNDOFF[p.u]
    normA = np.max(np.sum(np.abs(Aop), axis=1))

    if transpose:
        minv = lambda v: lum.apply_minv_t(F, v, ua if ua != "fp32" else "fp64", p.u)
        op = lambda v: lum.apply_atilde_t(A, F, v, ua if ua != "fp32" else "fp64", p.u)
        x = fu(lum.apply_minv_t(F, b, "fp64"))
    else:
        minv = lambda v: lum.apply_minv(F, v, ua, p.u)
        op = lambda v: lum.apply_atilde(A, F, v, ua, p.u)
        if p.lu_mode == "chop":
            x = fu(lum.apply_minv(F, b, p.uf))
        else:
            x = fu(lum.apply_minv(F, b, "fp64"))

    info = IrInfo()
    Y = Y0
    carry = None
    kk = None          # the recycle dimension once k_mode='knee' has fixed it
    for i in range(p.imax + 1):
        r_ur = residual(Aop, x, b, p.ur)
        r = fu(r_ur)
        eta = float(np.max(np.abs(r)) / (normA * np.max(np.abs(x)) + np.max(np.abs(b))))
        info.berr.append(eta)
        omega = componentwise_berr(Aop, x, b, r_ur)
        info.cberr.append(omega)
        if xstar is not None:
            info.ferr.append(forward_err(x, xstar))
        if p.stop == "cw":
            done = eta <= target and omega <= target
        elif p.stop == "all" and xstar is not None:
            rr = residual(Aop, x, b, "dd")
            done = max(normwise_berr(Aop, x, b, rr, normA), componentwise_berr(Aop, x, b, rr),
                       forward_err(x, xstar)) <= UNIT_ROUNDOFF[p.u]
        else:
            done = eta <= target
        if not np.all(np.isfinite(x)) or not np.isfinite(eta):
            info.status = "NONFINITE"
            break
        if done:
            info.converged = True
            info.status = "OK"
            break
        if i == p.imax:
            break
        if p.solver == "sir":
            # Algorithm 1, correction and update: d = U^-1 L^-1 r by substitution (in u_a, stored in u), x = x + d
            x = fu(x + fu(minv(r)))
            info.its.append(0)
            info.carry_applies.append(0)
            info.steps += 1
            continue
        s = float(np.max(np.abs(r)))
        rhat = fu(r / s)
        c = minv(rhat)
        auto = p.k_max if (p.k_mode == "knee" and kk is None) else None
        d, U, C, gi = gcrodr(op, c, p.m, p.k if kk is None else kk, p.tau, Ytil=Y, u=p.u, max_its=p.max_its,
                             basis=p.basis,
                             carry=carry, k_auto=auto)
        if kk is None and p.k_mode == "knee":
            kk = gi.k_used
        info.k_used.append(gi.k_used)
        info.its.append(gi.its)
        info.carry_applies.append(gi.carry_applies)
        info.k_eff.append(gi.k_eff)
        info.resid.append(gi.resid)
        if (p.k if kk is None else kk) > 0 and U.shape[1] > 0:
            Y = U
            carry = (U, C) if p.carry_mode == 1 else None
        x = fu(x + s * d)
        info.steps += 1
    return x, info, F, (Y, carry)


def adjoint_gradients(A, b, x, g, p: Params, F=None):
    """Gradients of a scalar loss with dL/dx = g at x = A^-1 b: db = lambda, dA = -lambda x^T."""
    lam, info, F, _ = solve(A, g, p, F=F, transpose=True)
    return lam, -np.outer(lam, x), info


def batch_solve(As, bs, p: Params):
    """Independent RGMRES-IR solves of a list of systems (no data shared between them)."""
    return [solve(A, b, p)[:2] for A, b in zip(As, bs)]


def exact_solution(A, b, iters=6):
    """Reference solution of the stored FP64 system: FP64 LU + refinement with dd residuals.

    Plain LAPACK GEPP in FP64 and up to ``iters`` refinement steps with double-double
    residuals (classical mixed-precision IR, Algorithm 1 with u_f = u = FP64 and
    u_r = dd); converges to full FP64 accuracy for kappa_inf(A) well below 1e16.
    """
    import scipy.linalg as sla
    lu, piv = sla.lu_factor(A)
    x = sla.lu_solve((lu, piv), b)
    for _ in range(iters):
        h, l = ddm.dd_residual(A, x, b)
        dx = sla.lu_solve((lu, piv), h + l)
        x = x + dx
        if np.max(np.abs(dx)) <= 1e-17 * np.max(np.abs(x)):
            break
    return x
