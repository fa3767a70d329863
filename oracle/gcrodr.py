"""GCRO-DR(m, k) for A~ d = c with initial guess d0 = 0 (Algorithm 3), plain FP64 numpy.

The steps follow Algorithm 3 in its order:

* Recycle space known (from the previous system, Algorithm 3 end: Y~ := U_k):
  QR(A~ Y~) = QR, C = Q, U = Y~ R^-1, d1 = U C^T r0, r1 = r0 - C C^T r0.
* Otherwise one GMRES(m) cycle: v1 = r0/||r0||, Arnoldi, min ||c - H_m y||, d1 = V_m y,
  r1 = V_{m+1}(c - H_m y); then the harmonic Ritz vectors of
  H_m + h_{m+1,m}^2 H_m^-T e_m e_m^T with the k smallest |theta| give P_k;
  Y~ = V_m P_k, QR(H_m P_k) = QR, C = V_{m+1} Q, U = Y~ R^-1.
* While ||r|| > tau ||c||: m - k Arnoldi steps with (I - C C^T) A~ from v1 = r/||r|| giving
  V, H (Hessenberg) and B = C^T A~ V; U~ = U D with D = diag(1/||u_i||);
  V^ = [U~ V_{m-k}], W^ = [C V_{m-k+1}], G = [[D, B], [0, H]];
  y = argmin ||W^T r - G y||; d += V^ y; r -= W^ G y; harmonic Ritz vectors of the pencil
  G^T G z = theta G^T W^T V^ z with the k smallest |theta| give P_k;
  QR(G P_k) = QR, C = W^ Q, U = V^ P_k R^-1.

Readings where the paper is silent or garbled:
* "||r|| > tau": tau is relative to ||c|| (= ||r0||, d0 = 0), Section 4's "relative
  (preconditioned) residual norm drops below tau".
* Arnoldi stops early inside a cycle when the Givens residual estimate drops below the
  tolerance; the Hessenberg matrix of the j steps taken is then used. A first cycle that
  stops after j <= k steps forms no recycle space (there are not k harmonic Ritz vectors
  to take); the next system then starts with a GMRES cycle again. This reproduces the
  rows of Tables 5-6 where recycling leaves the counts unchanged.
* v1 = r/||r||_2 (the printed ||r||^2 is a typo); Y~ = V^ P_k and C = W^ Q (hats dropped in print).
* Orthogonalisation is block classical Gram-Schmidt over [C V_j], done twice (CGS2);
  the coefficients of both passes are summed into B and H.
* Real arithmetic: a complex conjugate pair of harmonic Ritz vectors contributes [Re z, Im z];
  when the k-th smallest |theta| would split a pair the pair is taken whole if k + 1 < m and
  k + 1 <= the subspace dimension, and dropped otherwise. Ties in |theta| are broken by the
  position in the eigen-solver's output (only conjugate pairs tie in practice).
  Parity of the selected vectors themselves is unpinned; only the subspace they span
  enters the method, and the tests compare that.
* QR factors are normalised to a non-negative diagonal of R; columns whose |R_ii| falls
  below 1e-12 max |R_jj| are dropped (the recycle dimension shrinks).
* Vectors are stored in precision u (rounded after each vector operation); inner products,
  norms and all small dense algebra (least squares, eigenproblems, QR) are FP64.

Low-precision basis storage (the mixed precision inside GCRO-DR that Section 5 names as future
work): with ``basis`` set to a format, every stored basis vector -- the Arnoldi vectors v_j and
the recycle vectors C_k and U_k -- is rounded to that format when it is formed, while the
working vectors (the vector being orthogonalised, d and r) stay in u. ``basis=None`` stores
them in u.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.linalg as sla

from .formats import round_to

RANK_DROP = 1e-12


@dataclass
class GcroInfo:
    its: int = 0              # Arnoldi steps (one A~ application each)
    carry_applies: int = 0    # A~ applications of the recycle-space carry (QR(A~ Y~))
    cycles: int = 0
    converged: bool = False
    k_eff: int = 0
    k_used: int = 0           # recycle dimension used (differs from the argument with k_auto)
    resid: list = field(default_factory=list)   # Givens residual estimate after each Arnoldi step


def _qr_pos(X):
    """Reduced Householder QR with a non-negative diagonal of R.

    Columns whose |R_ii| falls below RANK_DROP * max |R_jj| are dropped and the QR is
    recomputed; ``keep`` marks the columns of X that were kept.
    """
    idx = np.arange(X.shape[1])
    while True:
        Q, R = np.linalg.qr(X[:, idx])
        sgn = np.where(np.diag(R) < 0, -1.0, 1.0)
        Q = Q * sgn[None, :]
        R = R * sgn[:, None]
        dg = np.abs(np.diag(R))
        ok = dg > RANK_DROP * (dg.max() if dg.size else 0.0)
        if np.all(ok):
            keep = np.zeros(X.shape[1], dtype=bool)
            keep[idx] = True
            return Q, R, keep
        idx = idx[ok]


def select_harmonic(theta, Z, k, dim, m):
    """Real basis P (dim x k_eff) of the eigenvectors of the k smallest |theta|.

    Infinite or NaN theta sort last. See the module docstring for the pair rule.
    """
    theta = np.asarray(theta)
    mag = np.abs(theta)
    mag = np.where(np.isfinite(mag), mag, np.inf)
    order = np.argsort(mag, kind="stable")
    k = min(k, dim)
    chosen = list(order[:k])
    if k > 0:
        last = chosen[-1]
        if abs(theta[last].imag) > 0:
            conj = [i for i in range(len(theta)) if i != last and np.isclose(theta[i], np.conj(theta[last]), rtol=1e-12, atol=0)]
            if conj and conj[0] not in chosen:
                if k + 1 < m and k + 1 <= dim:
                    chosen.append(conj[0])
                else:
                    chosen = chosen[:-1]
    cols = []
    done = set()
    for i in chosen:
        if i in done:
            continue
        z = Z[:, i]
        if abs(theta[i].imag) > 0:
            partner = [p for p in chosen if p != i and p not in done and np.isclose(theta[p], np.conj(theta[i]), rtol=1e-12, atol=0)]
            cols.append(z.real)
            cols.append(z.imag)
            done.add(i)
            if partner:
                done.add(partner[0])
        else:
            cols.append(z.real)
            done.add(i)
    if not cols:
        return np.zeros((dim, 0))
    return np.stack(cols, axis=1).astype(np.float64)


def _givens_estimate(H, j, g, cs, sn):
    """Apply the previous rotations to column j of H, make rotation j, update g; return |g[j+1]|."""
    col = H[: j + 2, j].copy()
    for i in range(j):
        a, b = col[i], col[i + 1]
        col[i] = cs[i] * a + sn[i] * b
        col[i + 1] = -sn[i] * a + cs[i] * b
    a, b = col[j], col[j + 1]
    rho = np.hypot(a, b)
    if rho == 0.0:
        cs[j], sn[j] = 1.0, 0.0
    else:
        cs[j], sn[j] = a / rho, b / rho
    g[j + 1] = -sn[j] * g[j]
    g[j] = cs[j] * g[j]
    return abs(g[j + 1])


def arnoldi(op, r, C, steps, tol, u, store=None):
    """Up to ``steps`` Arnoldi steps of (I - C C^T) A~ from v1 = r/||r|| with CGS2.

    The basis vectors are stored in precision ``store`` (default: u). Returns V (n x (j+1)),
    H ((j+1) x j), B (kc x j), j, Givens estimates.
    """
    fu = (lambda z: round_to(z, u))
    fmt_v = store or u
    fb = (lambda z: round_to(z, fmt_v))
    n = r.shape[0]
    kc = C.shape[1]
    beta = np.linalg.norm(r)
    V = np.zeros((n, steps + 1))
    H = np.zeros((steps + 1, steps))
    B = np.zeros((kc, steps))
    V[:, 0] = fb(r / beta)
    g = np.zeros(steps + 1)
    g[0] = beta
    cs = np.zeros(steps)
    sn = np.zeros(steps)
    est = []
    j = 0
    while j < steps:
        w = op(V[:, j])
        for _ in range(2):
            basis = np.hstack([C, V[:, : j + 1]])
            s = basis.T @ w
            w = fu(w - basis @ s)
            B[:, j] += s[:kc]
            H[: j + 1, j] += s[kc:]
        h = np.linalg.norm(w)
        H[j + 1, j] = h
        if h > 0.0:
            V[:, j + 1] = fb(w / h)
        e = _givens_estimate(H, j, g, cs, sn)
        est.append(e)
        j += 1
        if e <= tol or h == 0.0:
            break
    return V[:, : j + 1], H[: j + 1, :j], B[:, :j], j, est


def _lstsq(G, rhs):
    """Householder least squares min ||rhs - G y|| (library QR as the step)."""
    Q, R = np.linalg.qr(G)
    return sla.solve_triangular(R, Q.T @ rhs, lower=False)


def gcrodr(op, c, m, k, tau, Ytil=None, u="fp64", max_its=None, carry=None, k_auto=None, basis=None):
    """Solve A~ d = c by GCRO-DR(m, k) from d0 = 0.

    op:     v -> A~ v (already rounded to u).
    Ytil:   recycle vectors from the previous system (n x k') or None.
    carry:  optional (U, C) pair with A~ U = C from the previous system; when given it is
            used instead of recomputing QR(A~ Y~) (same result in exact arithmetic,
            because A~ does not change between refinement steps).
    k_auto: None, or a cap k_max: when the first (GMRES) cycle converges after j steps, the
            recycle dimension becomes min(j - 1, k_max) -- Section 5's observation that recycling
            the whole first-step subspace, k = its_1 - 1, gives the fewest iterations.
    basis:  None (basis vectors stored in u) or the format in which the Arnoldi vectors and the
            recycle vectors C, U are stored (low-precision basis storage, Section 5).
    Returns d, U (the Y~ for the next system), C, info (info.k_used: the k that was used).
    """
    fu = (lambda z: round_to(z, u))
    fmt_b = basis or u
    fb = (lambda z: round_to(z, fmt_b))
    c = np.asarray(c, dtype=np.float64)
    n = c.shape[0]
    info = GcroInfo()
    d = np.zeros(n)
    r = c.copy()
    tol = tau * np.linalg.norm(c)
    if tol == 0.0:
        info.converged = True
        return d, np.zeros((n, 0)), np.zeros((n, 0)), info
    if max_its is None:
        max_its = 20 * m
    C = np.zeros((n, 0))
    U = np.zeros((n, 0))

    if carry is not None and carry[0].shape[1] > 0:
        U, C = carry
        U, C = U.copy(), C.copy()
        d = fu(d + U @ (C.T @ r))
        r = fu(r - C @ (C.T @ r))
    elif Ytil is not None and Ytil.shape[1] > 0:
        Z = np.stack([op(Ytil[:, i]) for i in range(Ytil.shape[1])], axis=1)
        info.carry_applies = Ytil.shape[1]
        Q, R, keep = _qr_pos(Z)
        C = fb(Q)
        U = fb(sla.solve_triangular(R, Ytil[:, keep].T, trans="T", lower=False).T)
        d = fu(d + U @ (C.T @ r))
        r = fu(r - C @ (C.T @ r))
    else:
        V, H, _, j, est = arnoldi(op, r, np.zeros((n, 0)), m, tol, u, basis)
        info.its += j
        info.cycles += 1
        info.resid += est
        if k_auto is not None and est and est[-1] <= tol:
            k = min(j - 1, k_auto)
        beta = np.linalg.norm(r)
        rhs = np.zeros(j + 1)
        rhs[0] = beta
        y = _lstsq(H, rhs)
        d = fu(d + V[:, :j] @ y)
        r = fu(V @ (rhs - H @ y))
        if k > 0 and j > k:
            Hj = H[:j, :j]
            h = H[j, j - 1]
            ej = np.zeros(j)
            ej[-1] = 1.0
            f = sla.solve(Hj.T, ej)
            M1 = Hj.copy()
            M1[:, -1] += h * h * f
            theta, Zv = np.linalg.eig(M1)
            P = select_harmonic(theta, Zv, k, j, m)
            if P.shape[1] > 0:
                Y = V[:, :j] @ P
                Q, R, keep = _qr_pos(H @ P)
                C = fb(V @ Q)
                U = fb(sla.solve_triangular(R, Y[:, keep].T, trans="T", lower=False).T)

    while np.linalg.norm(r) > tol and info.its < max_its:
        kc = C.shape[1]
        steps = max(1, min(m - kc, max_its - info.its))
        V, H, B, j, est = arnoldi(op, r, C, steps, tol, u, basis)
        info.its += j
        info.cycles += 1
        info.resid += est
        if kc > 0:
            dk = 1.0 / np.linalg.norm(U, axis=0)
            Ut = U * dk[None, :]
        else:
            dk = np.zeros(0)
            Ut = U
        Vhat = np.hstack([Ut, V[:, :j]])
        What = np.hstack([C, V])
        G = np.zeros((kc + j + 1, kc + j))
        G[:kc, :kc] = np.diag(dk)
        G[:kc, kc:] = B
        G[kc:, kc:] = H
        y = _lstsq(G, What.T @ r)
        d = fu(d + Vhat @ y)
        r = fu(r - What @ (G @ y))
        if k > 0:
            WtV = What.T @ Vhat
            theta, Zv = sla.eig(G.T @ G, G.T @ WtV)
            P = select_harmonic(theta, Zv, k, kc + j, m)
            if P.shape[1] > 0:
                Q, R, keep = _qr_pos(G @ P)
                C = fb(What @ Q)
                U = fb(sla.solve_triangular(R, (Vhat @ P)[:, keep].T, trans="T", lower=False).T)
    info.converged = bool(np.linalg.norm(r) <= tol)
    info.k_eff = U.shape[1]
    info.k_used = k
    return d, U, C, info
