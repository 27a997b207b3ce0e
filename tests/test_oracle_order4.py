"""Pins of the oracle's fourth-order Laplacian (Sec. 4.2: second- or fourth-order finite
differences) and of everything built on it: closed-form eigenvalues, the textbook
stencil rows, fourth-order accuracy on a smooth non-sine function, the three-colour
Gauss-Seidel against a brute-force sweep, multigrid against a dense solve, and the
PFASST limit with a fourth-order fine and a second-order coarse level."""
import itertools
import math

import numpy as np
import pytest

import oracle as O


def sine(dim, n, k):
    h = 1.0 / (n + 1)
    x = np.arange(1, n + 1) * h
    v = np.ones(1)
    for a in range(dim):  # axis 0 (x) varies fastest
        v = np.multiply.outer(np.sin(k[a] * np.pi * x), v)
    return v.reshape(-1)


def lam4(n, k):
    """Eigenvalue of the 4th-order stencil on a sine mode (with the odd reflection)."""
    h = 1.0 / (n + 1)
    return sum((-2 * math.cos(2 * kk * math.pi * h) + 32 * math.cos(kk * math.pi * h) - 30) / (12 * h * h)
               for kk in k)


def dense(dim, n, order, c=None, nu=1.0):
    N = n ** dim
    M = np.zeros((N, N))
    for q in range(N):
        e = np.zeros(N)
        e[q] = 1.0
        M[:, q] = O.apply_L(dim, n, c, e, order=order) if c is not None else O.apply_A(dim, n, nu, e, order=order)
    return M


@pytest.mark.parametrize("dim,n,k", [(1, 15, (1,)), (1, 15, (15,)), (2, 7, (2, 7)), (3, 7, (1, 4, 7)),
                                     (3, 15, (13, 2, 5))])
def test_sine_modes_are_eigenvectors_with_the_closed_form_eigenvalue(dim, n, k):
    v = sine(dim, n, k)
    np.testing.assert_allclose(O.apply_A(dim, n, 0.7, v, order=4), 0.7 * lam4(n, k) * v,
                               atol=1e-11 * abs(lam4(n, k)))


def test_one_dimensional_rows_are_the_textbook_stencil():
    n = 9
    h2 = (n + 1) ** 2
    A = dense(1, n, 4) / h2 * 12
    want = np.zeros((n, n))
    for i in range(n):
        for d, w in ((-2, -1), (-1, 16), (0, -30), (1, 16), (2, -1)):
            if 0 <= i + d < n:
                want[i, i + d] += w
    want[0, 0] += 1   # the point beyond the wall is -u at the first point
    want[-1, -1] += 1
    np.testing.assert_allclose(A, want, atol=1e-9)
    assert np.allclose(A, A.T) and np.all(np.linalg.eigvalsh(A) < 0)


def test_fourth_order_accuracy_on_a_smooth_odd_periodic_function():
    """u = sin(pi x) / (1.5 - cos(pi x)) is odd about both walls (so the reflection is
    consistent) and not a finite sine sum; the max error of the stencil falls 16x per
    halving of h (4x for the second-order stencil)."""
    sympy = pytest.importorskip("sympy")
    X = sympy.symbols("x")
    u = sympy.sin(sympy.pi * X) / (sympy.Rational(3, 2) - sympy.cos(sympy.pi * X))
    f, d2 = sympy.lambdify(X, u, "numpy"), sympy.lambdify(X, sympy.diff(u, X, 2), "numpy")
    errs = {2: [], 4: []}
    for n in (31, 63, 127):
        x = np.arange(1, n + 1) / (n + 1)
        for order in (2, 4):
            errs[order].append(np.abs(O.apply_A(1, n, 1.0, f(x), order=order) - d2(x)).max())
    r4 = [errs[4][i] / errs[4][i + 1] for i in range(2)]
    r2 = [errs[2][i] / errs[2][i + 1] for i in range(2)]
    assert all(13 < r < 19 for r in r4), r4
    assert all(3.5 < r < 4.5 for r in r2), r2


def test_same_colour_points_do_not_couple():
    dim, n = 2, 7
    A = dense(dim, n, 4)
    col = [(i + 1 + j + 1) % 3 for j, i in itertools.product(range(n), range(n))]
    for p in range(n * n):
        for q in range(n * n):
            if p != q and col[p] == col[q]:
                assert A[p, q] == 0.0


@pytest.mark.parametrize("dim", [1, 2, 3])
def test_three_colour_gauss_seidel_equals_a_brute_force_sweep(dim):
    n = 7
    c = 0.3 / (n + 1) ** 2
    rng = np.random.default_rng(dim)
    f, e0 = rng.standard_normal((2, n ** dim))
    omega = 0.9
    L = dense(dim, n, 4, c=c)
    e = e0.copy()
    idx = list(itertools.product(*([range(n)] * dim)))  # (slowest .. fastest axis)
    for colour in range(3):
        for t in idx:
            if (sum(t) + dim) % 3 != colour:
                continue
            p = 0
            for v in t:
                p = p * n + v
            e[p] += omega * (f[p] - L[p] @ e) / L[p, p]
    got = O.smooth(O.MGParams(smoother=1, omega=omega), dim, n, c, f, e0, order=4)
    np.testing.assert_allclose(got, e, atol=1e-12)


def test_jacobi_first_sweep_uses_the_exact_diagonal():
    dim, n, c, omega = 2, 7, 0.02, 2.0 / 3.0
    f = np.random.default_rng(5).standard_normal(n * n)
    L = dense(dim, n, 4, c=c)
    got = O.smooth(O.MGParams(smoother=0, omega=omega), dim, n, c, f, np.zeros(n * n), order=4)
    np.testing.assert_allclose(got, omega * f / np.diag(L), atol=1e-14)


@pytest.mark.parametrize("sm", [0, 1])
@pytest.mark.parametrize("dim,n", [(1, 63), (2, 31), (3, 15)])
def test_multigrid_with_a_fourth_order_finest_grid_solves_the_dense_system(sm, dim, n):
    c = 0.05
    rng = np.random.default_rng(dim * 10 + sm)
    b = rng.standard_normal(n ** dim)
    mg = O.MGParams(smoother=sm, omega=1.0 if sm else 0.6, vcycles=0, mg_tol=1e-13, mg_maxcycles=80, mg_stall=0.99)
    u, cyc = O.mg_solve(mg, dim, n, c, b, np.zeros_like(b), order=4)
    want = np.linalg.solve(dense(dim, n, 4, c=c), b) if n ** dim <= 4000 else None
    if want is not None:
        assert np.abs(u - want).max() <= 1e-11 * np.abs(want).max()
    r = b - O.apply_L(dim, n, c, u, order=4)
    assert np.abs(r).max() <= 1e-12 * max(1.0, np.abs(b).max())
    # and every V-cycle contracts (second-order coarse grids correct a fourth-order residual)
    mg1 = O.MGParams(smoother=sm, omega=1.0 if sm else 0.6, vcycles=1)
    e = np.zeros_like(b)
    rn = [np.abs(b).max()]
    for _ in range(4):
        e, _ = O.mg_solve(mg1, dim, n, c, b, e, order=4)
        rn.append(np.abs(b - O.apply_L(dim, n, c, e, order=4)).max())
    assert all(rn[i + 1] < 0.6 * rn[i] for i in range(4)), rn


def _pade(z, s):
    N = s - 1
    cf = [math.factorial(2 * N - j) * math.factorial(N) / (math.factorial(2 * N) * math.factorial(j)
                                                            * math.factorial(N - j)) for j in range(N + 1)]
    return sum(cf[j] * z ** j for j in range(N + 1)) / sum(cf[j] * (-z) ** j for j in range(N + 1))


@pytest.mark.parametrize("dim,n,nl", [(1, 31, 2), (2, 15, 2), (1, 31, 1), (2, 31, 3)])
def test_pfasst_limit_is_the_fourth_order_collocation_solution(dim, n, nl):
    """Fine level 4th order, coarser levels 2nd order: the converged end value of slice p
    is R(dt nu lambda_4)^(p+1) per sine mode (R the Pade stability function of the
    Gauss-Lobatto rule) -- the coarse operators enter only through FAS corrections."""
    P, nu, dt = 4, 0.5, 0.01
    ks = [(1,) * dim, tuple([3] + [2] * (dim - 1)), tuple([n - 2] * dim)]
    amps = [1.0, 0.5, 0.25]
    u0 = sum(a * sine(dim, n, k) for a, k in zip(amps, ks))
    mg = O.MGParams(smoother=1, omega=1.0, vcycles=3)
    if nl == 3:
        pf = O.MLPFASST(dim, n, (5, 3, 2), P, nu, dt, mg, order=4)
    else:
        pf = O.PFASST(dim, n, 5, 3, P, nu, dt, mg, nlevels=nl, order=4)
    pf.set_initial(u0)
    it, hist = pf.run(250, 1e-12)  # stiff high modes: Gauss-Lobatto damps them slowly
    end = pf.end_value()
    want = sum(a * _pade(dt * nu * lam4(n, k), 5) ** P * sine(dim, n, k) for a, k in zip(amps, ks))
    assert it < 250
    np.testing.assert_allclose(end, want, atol=1e-10 * np.abs(want).max())
