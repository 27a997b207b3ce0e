"""FP64 CPU oracle for SDC + multigrid + two-level PFASST.

TEST INFRASTRUCTURE ONLY.  The oracle is the slow, plain reference against which
the CUDA library is checked.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it; the
library in ``paper_1407_6486_gb300`` never does and shares no code with it.

The arithmetic lives in ``pfasst_oracle.c`` (plain loops, FP64, each function
citing the section or equation of the paper it follows).  This module compiles it
with gcc, binds it with ctypes and keeps the PFASST state in numpy arrays.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pfasst_oracle.c")
_LIB = os.path.join(_HERE, "_liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_liboracle.so`` (gcc, -O2, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _MG(ctypes.Structure):
    _fields_ = [("smoother", ctypes.c_int), ("omega", ctypes.c_double),
                ("nu1", ctypes.c_int), ("nu2", ctypes.c_int),
                ("vcycles", ctypes.c_int), ("mg_tol", ctypes.c_double),
                ("mg_stall", ctypes.c_double), ("mg_maxcycles", ctypes.c_int)]


class _Level(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("n", ctypes.c_int), ("s", ctypes.c_int),
                ("nu", ctypes.c_double), ("dt", ctypes.c_double), ("family", ctypes.c_int), ("order", ctypes.c_int)]


class _PFASST(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("n_f", ctypes.c_int), ("s_f", ctypes.c_int),
                ("s_c", ctypes.c_int), ("slices", ctypes.c_int), ("nlevels", ctypes.c_int),
                ("interp_order", ctypes.c_int), ("nu", ctypes.c_double),
                ("dt", ctypes.c_double), ("mg", _MG), ("fam_f", ctypes.c_int), ("fam_c", ctypes.c_int),
                ("order_f", ctypes.c_int), ("mg_c", _MG)]


_D = ctypes.POINTER(ctypes.c_double)


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        L = _lib
        L.orc_gauss_lobatto.argtypes = [ctypes.c_int, _D]
        L.orc_qmatrix.argtypes = [ctypes.c_int, _D, _D]
        L.orc_lagrange_weights.argtypes = [ctypes.c_int, _D, ctypes.c_double, _D]
        L.orc_apply_A.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, _D, _D]
        L.orc_apply_A_o.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double, _D, _D]
        L.orc_apply_L.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, _D, _D]
        L.orc_apply_L_o.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double, _D, _D]
        L.orc_smooth.argtypes = [ctypes.POINTER(_MG), ctypes.c_int, ctypes.c_int, ctypes.c_double, _D, _D]
        L.orc_smooth_o.argtypes = [ctypes.POINTER(_MG), ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                   _D, _D]
        L.orc_restrict_fw.argtypes = [ctypes.c_int, ctypes.c_int, _D, _D]
        L.orc_prolong_add.argtypes = [ctypes.c_int, ctypes.c_int, _D, _D]
        L.orc_mg_solve.argtypes = [ctypes.POINTER(_MG), ctypes.c_int, ctypes.c_int, ctypes.c_double, _D, _D]
        L.orc_mg_solve.restype = ctypes.c_int
        L.orc_mg_solve_o.argtypes = [ctypes.POINTER(_MG), ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                     _D, _D]
        L.orc_mg_solve_o.restype = ctypes.c_int
        L.orc_sweep.argtypes = [ctypes.POINTER(_Level), ctypes.POINTER(_MG), _D, _D, _D]
        L.orc_sweep.restype = ctypes.c_int
        L.orc_residual.argtypes = [ctypes.POINTER(_Level), _D, _D, _D]
        L.orc_residual.restype = ctypes.c_double
        L.orc_inject.argtypes = [ctypes.c_int, ctypes.c_int, _D, _D]
        L.orc_interp_add.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double, _D, _D]
        L.orc_pfasst_spread.argtypes = [ctypes.POINTER(_PFASST), _D, _D, _D]
        L.orc_pfasst_predict.argtypes = [ctypes.POINTER(_PFASST)] + [_D] * 6
        L.orc_pfasst_iteration.argtypes = [ctypes.POINTER(_PFASST)] + [_D] * 7
        L.orc_pfasst_interp_slice.argtypes = [ctypes.POINTER(_PFASST)] + [_D] * 4
        L.orc_set_threads.argtypes = [ctypes.c_int]
        L.orc_set_threads.restype = ctypes.c_int
    return _lib


def set_threads(n: int) -> int:
    """OpenMP threads of the oracle's grid loops (n <= 0: leave as is); returns the count."""
    return lib().orc_set_threads(n)


def _p(a: np.ndarray | None):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_D)


@dataclass
class MGParams:
    """Multigrid settings: smoother 0 = weighted Jacobi, 1 = red-black Gauss-Seidel."""
    smoother: int = 0
    omega: float = 2.0 / 3.0
    nu1: int = 2
    nu2: int = 1
    vcycles: int = 2            # 0 = full solve to mg_tol with the stall rule
    mg_tol: float = 1e-12
    mg_stall: float = 0.75
    mg_maxcycles: int = 50

    def c(self) -> _MG:
        return _MG(self.smoother, self.omega, self.nu1, self.nu2, self.vcycles,
                   self.mg_tol, self.mg_stall, self.mg_maxcycles)


def gauss_lobatto(s: int) -> np.ndarray:
    t = np.zeros(s)
    assert lib().orc_gauss_lobatto(s, _p(t)) == 0
    return t


def nodes(s: int, family: int = 0) -> np.ndarray:
    """family 0: Gauss-Lobatto; 1: uniform m/M, quadrature without the left endpoint."""
    t = np.zeros(s)
    assert lib().orc_nodes(s, family, _p(t)) == 0
    return t


def qmatrix(s: int, family: int = 0) -> np.ndarray:
    t = nodes(s, family)
    Q = np.zeros((s, s))
    assert lib().orc_qmatrix_family(s, family, _p(t), _p(Q)) == 0
    return Q


def lagrange_weights(tc: np.ndarray, t: float) -> np.ndarray:
    tc = np.ascontiguousarray(tc, dtype=np.float64)
    w = np.zeros(len(tc))
    lib().orc_lagrange_weights(len(tc), _p(tc), t, _p(w))
    return w


def _grid(u, dim, n):
    u = np.ascontiguousarray(u, dtype=np.float64)
    assert u.size == n ** dim
    return u


def apply_A(dim: int, n: int, nu: float, u: np.ndarray, order: int = 2) -> np.ndarray:
    """nu Lap_h u with the 2nd-order (Sec. 4.1) or 4th-order (Sec. 4.2) stencil."""
    u = _grid(u, dim, n)
    out = np.empty_like(u)
    if order == 2:
        lib().orc_apply_A(dim, n, nu, _p(u), _p(out))
    else:
        lib().orc_apply_A_o(dim, n, order, nu, _p(u), _p(out))
    return out


def apply_L(dim: int, n: int, c: float, e: np.ndarray, order: int = 2) -> np.ndarray:
    e = _grid(e, dim, n)
    out = np.empty_like(e)
    if order == 2:
        lib().orc_apply_L(dim, n, c, _p(e), _p(out))
    else:
        lib().orc_apply_L_o(dim, n, order, c, _p(e), _p(out))
    return out


def smooth(mg: MGParams, dim: int, n: int, c: float, f: np.ndarray, e: np.ndarray, order: int = 2) -> np.ndarray:
    """One sweep; with order 4 Gauss-Seidel runs in three colours (I+J+K) mod 3."""
    f = _grid(f, dim, n)
    e = _grid(e, dim, n).copy()
    m = mg.c()
    if order == 2:
        lib().orc_smooth(ctypes.byref(m), dim, n, c, _p(f), _p(e))
    else:
        lib().orc_smooth_o(ctypes.byref(m), dim, n, order, c, _p(f), _p(e))
    return e


def restrict_fw(dim: int, n: int, r: np.ndarray) -> np.ndarray:
    r = _grid(r, dim, n)
    out = np.zeros(((n - 1) // 2) ** dim)
    lib().orc_restrict_fw(dim, n, _p(r), _p(out))
    return out


def prolong_add(dim: int, n: int, ec: np.ndarray, e: np.ndarray) -> np.ndarray:
    ec = _grid(ec, dim, (n - 1) // 2)
    e = _grid(e, dim, n).copy()
    lib().orc_prolong_add(dim, n, _p(ec), _p(e))
    return e


def mg_solve(mg: MGParams, dim: int, n: int, c: float, b: np.ndarray, u: np.ndarray, order: int = 2):
    """Returns (u_new, V-cycles used); `order` is the finest grid's Laplacian order
    (coarser grids are 2nd order)."""
    b = _grid(b, dim, n)
    u = _grid(u, dim, n).copy()
    m = mg.c()
    if order == 2:
        cyc = lib().orc_mg_solve(ctypes.byref(m), dim, n, c, _p(b), _p(u))
    else:
        cyc = lib().orc_mg_solve_o(ctypes.byref(m), dim, n, order, c, _p(b), _p(u))
    return u, cyc


def sweep(dim, n, s, nu, dt, mg: MGParams, U, F, fas=None, family=0, order=2):
    """One SDC sweep on one slice, in place on copies; returns (U, F, V-cycles)."""
    U = np.ascontiguousarray(U, dtype=np.float64).copy()
    F = np.ascontiguousarray(F, dtype=np.float64).copy()
    L = _Level(dim, n, s, nu, dt, family, order)
    m = mg.c()
    cyc = lib().orc_sweep(ctypes.byref(L), ctypes.byref(m), _p(U), _p(F), _p(fas))
    return U, F, cyc


def residual(dim, n, s, nu, dt, U, F, fas=None, family=0) -> float:
    L = _Level(dim, n, s, nu, dt, family, 2)
    return lib().orc_residual(ctypes.byref(L), _p(np.ascontiguousarray(U)), _p(np.ascontiguousarray(F)), _p(fas))


def inject(dim: int, n: int, uf: np.ndarray) -> np.ndarray:
    uf = _grid(uf, dim, n)
    out = np.zeros(((n - 1) // 2) ** dim)
    lib().orc_inject(dim, n, _p(uf), _p(out))
    return out


def interp_add(dim: int, n: int, order: int, alpha: float, uc: np.ndarray, uf: np.ndarray) -> np.ndarray:
    uc = _grid(uc, dim, (n - 1) // 2)
    uf = _grid(uf, dim, n).copy()
    lib().orc_interp_add(dim, n, order, alpha, _p(uc), _p(uf))
    return uf


class PFASST:
    """Serial emulation of two-level PFASST over ``slices`` time slices.

    State: ``Uf, Ff`` of shape (slices, s_f, n^dim); ``Uc, Fc, fas, Uc0`` of shape
    (slices, s_c, n_c^dim).  ``nlevels == 1`` gives (parallel) single-level SDC.
    """

    def __init__(self, dim, n, s_f, s_c, slices, nu, dt, mg: MGParams, nlevels=2, interp_order=4, family=0,
                 coarse_family=None, order=2, mg_coarse: MGParams | None = None):
        """order: Laplacian order of the fine level (2 or 4); the coarse level is 2nd order.
        mg_coarse: multigrid settings of the coarse level's sub-step solves (default: mg)."""
        self.dim, self.n, self.s_f, self.s_c = dim, n, s_f, s_c
        self.slices, self.nu, self.dt, self.nlevels = slices, nu, dt, nlevels
        self.mg = mg
        fam_c = family if coarse_family is None else coarse_family
        self.family, self.coarse_family = family, fam_c
        if nlevels > 1:
            tf, tc = nodes(s_f, family), nodes(s_c, fam_c)
            if not all(np.min(np.abs(tf - t)) < 1e-14 for t in tc):
                raise ValueError("coarse nodes must be a subset of the fine nodes")
            if n < 7:
                raise ValueError("two levels need n >= 7")
        if order == 4 and n < 7:
            raise ValueError("the fourth-order stencil needs n >= 7")
        self._c = _PFASST(dim, n, s_f, s_c if nlevels > 1 else 2, slices, nlevels,
                          interp_order, nu, dt, mg.c(), family, fam_c, order, (mg_coarse or mg).c())
        Nf = n ** dim
        nc = (n - 1) // 2
        Nc = max(nc, 1) ** dim
        self.Uf = np.zeros((slices, s_f, Nf))
        self.Ff = np.zeros_like(self.Uf)
        sc = s_c if nlevels > 1 else 1
        self.Uc = np.zeros((slices, sc, Nc))
        self.Fc = np.zeros_like(self.Uc)
        self.fas = np.zeros_like(self.Uc)
        self.Uc0 = np.zeros_like(self.Uc)
        self.res = np.zeros(slices)

    def set_initial(self, u0: np.ndarray):
        u0 = np.ascontiguousarray(u0, dtype=np.float64).reshape(-1)
        lib().orc_pfasst_spread(ctypes.byref(self._c), _p(u0), _p(self.Uf), _p(self.Ff))

    def predict(self):
        lib().orc_pfasst_predict(ctypes.byref(self._c), _p(self.Uf), _p(self.Ff), _p(self.Uc),
                                 _p(self.Fc), _p(self.fas), _p(self.Uc0))

    def iteration(self) -> np.ndarray:
        lib().orc_pfasst_iteration(ctypes.byref(self._c), _p(self.Uf), _p(self.Ff), _p(self.Uc),
                                   _p(self.Fc), _p(self.fas), _p(self.Uc0), _p(self.res))
        return self.res.copy()

    def interp_slice(self, p: int):
        """Only the interpolation step of slice p: Uf[p] += I_t I_x (Uc[p] - Uc0[p]),
        then Ff[p] = A Uf[p]."""
        Uf, Ff = self.Uf[p], self.Ff[p]
        assert Uf.flags.c_contiguous and Ff.flags.c_contiguous
        lib().orc_pfasst_interp_slice(ctypes.byref(self._c), _p(Uf), _p(Ff),
                                      _p(np.ascontiguousarray(self.Uc[p])), _p(np.ascontiguousarray(self.Uc0[p])))

    def run(self, max_iter: int, tol: float):
        """Predictor, then iterations until max residual <= tol. Returns (iters, res history)."""
        self.predict()
        hist = []
        for k in range(max_iter):
            r = self.iteration()
            hist.append(r)
            if r.max() <= tol:
                return k + 1, hist
        return max_iter, hist

    def end_value(self) -> np.ndarray:
        return self.Uf[-1, -1].copy()


class _ML(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("n0", ctypes.c_int), ("slices", ctypes.c_int), ("nlevels", ctypes.c_int),
                ("interp_order", ctypes.c_int), ("s", ctypes.c_int * 3), ("fam", ctypes.c_int * 3),
                ("nu", ctypes.c_double), ("dt", ctypes.c_double), ("mg", _MG), ("order0", ctypes.c_int),
                ("mg_c", _MG)]


class _MLState(ctypes.Structure):
    _fields_ = [("U", _D * 3), ("F", _D * 3), ("tau", _D * 3), ("Ur", _D * 3)]


class MLPFASST:
    """Serial emulation of PFASST with up to three levels (level l grid: n_l = (n_{l-1}-1)/2).

    ``nodes``: node count per level, ``families``: node family per level (0 Gauss-Lobatto,
    1 uniform).  State ``U[l], F[l], tau[l], Ur[l]`` of shape (slices, s_l, n_l^dim).
    With two levels the schedule is the one of :class:`PFASST`.
    """

    def __init__(self, dim, n, nodes, slices, nu, dt, mg: MGParams, families=None, interp_order=4, order=2,
                 mg_coarse: MGParams | None = None):
        L = len(nodes)
        assert 1 <= L <= 3
        families = list(families) if families is not None else [0] * L
        self.dim, self.n, self.nodes, self.families = dim, n, list(nodes), families
        self.slices, self.nu, self.dt, self.L = slices, nu, dt, L
        grids = [n]
        for _ in range(1, L):
            grids.append((grids[-1] - 1) // 2)
        if min(grids) < 3:
            raise ValueError("every level needs at least 3 points per axis")
        for l in range(1, L):
            tf, tc = globals()["nodes"](nodes[l - 1], families[l - 1]), globals()["nodes"](nodes[l], families[l])
            if not all(np.min(np.abs(tf - t)) < 1e-14 for t in tc):
                raise ValueError("the nodes of every level must be a subset of the finer level's")
        self.grids = grids
        s = (ctypes.c_int * 3)(*(list(nodes) + [2] * (3 - L)))
        f = (ctypes.c_int * 3)(*(families + [0] * (3 - L)))
        self._c = _ML(dim, n, slices, L, interp_order, s, f, nu, dt, mg.c(), order, (mg_coarse or mg).c())
        self.U = [np.zeros((slices, nodes[l], grids[l] ** dim)) for l in range(L)]
        self.F = [np.zeros_like(u) for u in self.U]
        self.tau = [np.zeros_like(u) for u in self.U]
        self.Ur = [np.zeros_like(u) for u in self.U]
        self.res = np.zeros(slices)

    def _state(self):
        st = _MLState()
        for l in range(3):
            ll = min(l, self.L - 1)
            st.U[l] = _p(self.U[ll])
            st.F[l] = _p(self.F[ll])
            st.tau[l] = _p(self.tau[ll])
            st.Ur[l] = _p(self.Ur[ll])
        return st

    def set_initial(self, u0):
        u0 = np.ascontiguousarray(u0, dtype=np.float64).reshape(-1)
        st = self._state()
        lib().orc_ml_spread(ctypes.byref(self._c), _p(u0), ctypes.byref(st))

    def predict(self):
        st = self._state()
        lib().orc_ml_predict(ctypes.byref(self._c), ctypes.byref(st))

    def interp_slice(self, level, p):
        """Only the interpolation step level+1 -> level of slice p: U[level][p] +=
        I_t I_x (U[level+1][p] - Ur[level+1][p]), then F[level][p] = A U[level][p]."""
        st = self._state()
        lib().orc_ml_interp_slice(ctypes.byref(self._c), ctypes.byref(st), level, p)

    def sweep(self, level):
        """One sweep on ``level`` of every slice (the serial chain on the coarsest level)."""
        st = self._state()
        lib().orc_ml_sweep_level(ctypes.byref(self._c), ctypes.byref(st), level)

    def iteration(self) -> np.ndarray:
        st = self._state()
        lib().orc_ml_iteration(ctypes.byref(self._c), ctypes.byref(st), _p(self.res))
        return self.res.copy()

    def run(self, max_iter, tol):
        self.predict()
        hist = []
        for k in range(max_iter):
            r = self.iteration()
            hist.append(float(np.max(r)))
            if hist[-1] <= tol:
                return k + 1, hist
        return max_iter, hist

    def end_value(self):
        return self.U[0][-1, -1].copy()
