"""Pins of oracle.dd against exact rational arithmetic."""
from fractions import Fraction

import numpy as np

from oracle import dd


def F(x):
    return Fraction(float(x))


def test_error_free_transforms():
    rng = np.random.default_rng(3)
    a = rng.standard_normal(2000) * np.exp(rng.uniform(-20, 20, 2000))
    b = rng.standard_normal(2000) * np.exp(rng.uniform(-20, 20, 2000))
    s, e = dd.two_sum(a, b)
    p, f = dd.two_prod(a, b)
    for i in range(2000):
        assert F(s[i]) + F(e[i]) == F(a[i]) + F(b[i])
        assert F(p[i]) + F(f[i]) == F(a[i]) * F(b[i])


def test_dd_residual_exact():
    rng = np.random.default_rng(4)
    for n in (1, 3, 8, 12):
        A = rng.standard_normal((n, n))
        x = rng.standard_normal(n)
        # b close to A x so the residual suffers heavy cancellation
        b = A @ x + 1e-14 * rng.standard_normal(n)
        h, l = dd.dd_residual(A, x, b)
        for i in range(n):
            exact = F(b[i]) - sum(F(A[i, j]) * F(x[j]) for j in range(n))
            scale = sum(abs(F(A[i, j]) * F(x[j])) for j in range(n)) + abs(F(b[i]))
            err = abs(F(h[i]) + F(l[i]) - exact)
            assert err <= 2 * n * Fraction(2) ** -106 * scale


def test_dd_triangular_solves():
    rng = np.random.default_rng(5)
    n = 10
    L = np.tril(rng.standard_normal((n, n)) * 0.3, -1) + np.eye(n)
    U = np.triu(rng.standard_normal((n, n))) + 3 * np.eye(n)
    z = rng.standard_normal(n)
    yh, yl = dd.dd_lower_solve(L, z, np.zeros(n), unit=True)
    # exact forward substitution in rationals
    y = []
    for i in range(n):
        y.append(F(z[i]) - sum(F(L[i, j]) * y[j] for j in range(i)))
    for i in range(n):
        assert abs(F(yh[i]) + F(yl[i]) - y[i]) <= Fraction(2) ** -95 * (1 + abs(y[i]))
    xh, xl = dd.dd_upper_solve(U, yh, yl)
    xs = [None] * n
    for i in range(n - 1, -1, -1):
        xs[i] = (F(yh[i]) + F(yl[i]) - sum(F(U[i, j]) * xs[j] for j in range(i + 1, n))) / F(U[i, i])
    for i in range(n):
        assert abs(F(xh[i]) + F(xl[i]) - xs[i]) <= Fraction(2) ** -95 * (1 + abs(xs[i]))


def test_dd_div():
    rng = np.random.default_rng(6)
    a = rng.standard_normal(100)
    b = rng.standard_normal(100)
    q, ql = dd.dd_div_d(a, np.zeros(100), b)
    for i in range(100):
        exact = F(a[i]) / F(b[i])
        assert abs(F(q[i]) + F(ql[i]) - exact) <= Fraction(2) ** -103 * abs(exact)
