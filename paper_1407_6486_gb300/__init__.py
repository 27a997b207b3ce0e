"""Python binding of the pfasst_mg C ABI (``include/pfasst_mg.h``).

Batched SDC sweeps with geometric-multigrid sub-step solves and two-level PFASST
for the heat equation ("Interweaving PFASST and Parallel Multigrid", Sec. 2 - 4),
computed entirely by the CUDA kernels of ``libpfasst_mg.so`` (sm_103a).  This module
only marshals arguments: the functions carry the C names, PyTorch supplies device
memory (the solver workspace) and the CUDA stream.  There is no CPU fallback: if
the library has not been built, loading it raises.
"""
from __future__ import annotations

import ctypes
import os

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libpfasst_mg.so")

PMG_OK = 0
PMG_NOT_CONVERGED = 1
PMG_ERR_INVALID_ARG = -1
PMG_ERR_OOM = -2
PMG_ERR_CUDA = -3
PMG_ERR_DIVERGED = -4
PMG_ERR_TIMEOUT = -5
PMG_ERR_UNSUPPORTED = -6
PMG_SMOOTHER_JACOBI = 0
PMG_SMOOTHER_RBGS = 1
PMG_PREC_FP64 = 0
PMG_PREC_MIXED = 1

EXPORTS = [
    "pfasst_mg_default_options", "pfasst_mg_workspace_bytes", "pfasst_mg_create",
    "pfasst_mg_set_initial", "pfasst_mg_predict", "pfasst_mg_sweep", "pfasst_mg_iterate",
    "pfasst_mg_residual", "pfasst_mg_get_solution", "pfasst_mg_get_state", "pfasst_mg_advance",
    "pfasst_mg_launch_count", "pfasst_mg_destroy", "pfasst_mg_last_error",
    "pfasst_mg_helmholtz_solve", "pfasst_mg_profile", "pfasst_mg_profile_read", "pfasst_mg_kernel_name",
    "pfasst_mg_helmholtz_solve_noalloc", "pfasst_mg_batch_workspace_bytes", "pfasst_mg_create_batch",
    "pfasst_mg_batch_set_initial", "pfasst_mg_batch_run", "pfasst_mg_batch_get_solution", "pfasst_mg_tuning",
    "pfasst_mg_net_param_count", "pfasst_mg_net_init", "pfasst_mg_net_create", "pfasst_mg_net_set_params",
    "pfasst_mg_net_get_params", "pfasst_mg_net_forward", "pfasst_mg_net_gradients", "pfasst_mg_net_sample",
    "pfasst_mg_net_train", "pfasst_mg_net_launch_count", "pfasst_mg_net_destroy", "pfasst_mg_net_last_error",
    "pfasst_mg_set_smoother_net", "pfasst_mg_net_step", "pfasst_mg_net_profile", "pfasst_mg_net_profile_read",
    "pfasst_mg_check_narrowing", "pfasst_mg_fp64_peak", "pfasst_mg_check_widening", "pfasst_mg_net_substep_pairs",
]

NET_PARAMS = 7809  # W1[16][27], b1[16], W2[16][27][16], b2[16], W3[27][16], b3


class pmg_grid(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("n", ctypes.c_int), ("order", ctypes.c_int)]


class pmg_nodes_desc(ctypes.Structure):
    _fields_ = [("count", ctypes.c_int), ("family", ctypes.c_int)]


class pmg_levels(ctypes.Structure):
    _fields_ = [("nlevels", ctypes.c_int), ("coarse_nodes", pmg_nodes_desc), ("coarsest_nodes", pmg_nodes_desc)]


class pmg_options(ctypes.Structure):
    _fields_ = [("smoother", ctypes.c_int), ("omega", ctypes.c_double), ("nu1", ctypes.c_int),
                ("nu2", ctypes.c_int), ("vcycles", ctypes.c_int), ("mg_tol", ctypes.c_double),
                ("mg_stall", ctypes.c_double), ("mg_maxcycles", ctypes.c_int),
                ("precision", ctypes.c_int), ("interp_order", ctypes.c_int),
                ("use_graphs", ctypes.c_int), ("autotune", ctypes.c_int), ("slice_groups", ctypes.c_int),
                ("vcycle_tail", ctypes.c_int), ("coarse_vcycles", ctypes.c_int), ("single_grid_vcycle", ctypes.c_int)]


class pmg_problem_desc(ctypes.Structure):
    _fields_ = [("grid", pmg_grid), ("nodes", ctypes.c_int), ("nu", ctypes.c_double), ("dt", ctypes.c_double)]


class pmg_kernel_stat(ctypes.Structure):
    _fields_ = [("kernel", ctypes.c_int), ("n", ctypes.c_int), ("precision", ctypes.c_int),
                ("launches", ctypes.c_longlong), ("points", ctypes.c_longlong), ("ms", ctypes.c_double)]


class PMGError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"pfasst_mg error {code}: {msg}")
        self.code = code


_lib = None
_P = ctypes.c_void_p
_I = ctypes.c_int
_D = ctypes.c_double


def load() -> ctypes.CDLL:
    """Load ``libpfasst_mg.so`` (built by ``_build.build()``); raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} not built: run __graft_entry__.build() "
                          "(python -c 'import __graft_entry__ as g; g.build()')")
    L = ctypes.CDLL(LIB_PATH)
    L.pfasst_mg_default_options.argtypes = [ctypes.POINTER(pmg_options)]
    L.pfasst_mg_default_options.restype = None
    L.pfasst_mg_workspace_bytes.argtypes = [ctypes.POINTER(pmg_grid), ctypes.POINTER(pmg_nodes_desc),
                                            ctypes.POINTER(pmg_levels), _I, ctypes.POINTER(pmg_options),
                                            ctypes.POINTER(ctypes.c_size_t)]
    L.pfasst_mg_create.argtypes = [ctypes.POINTER(pmg_grid), ctypes.POINTER(pmg_nodes_desc),
                                   ctypes.POINTER(pmg_levels), _D, _D, _I, ctypes.POINTER(pmg_options),
                                   _P, _P, ctypes.c_size_t, ctypes.POINTER(_P)]
    L.pfasst_mg_set_initial.argtypes = [_P, _P, _I]
    L.pfasst_mg_predict.argtypes = [_P]
    L.pfasst_mg_sweep.argtypes = [_P, _I]
    L.pfasst_mg_iterate.argtypes = [_P, _I, _D, ctypes.POINTER(_I), ctypes.POINTER(_D)]
    L.pfasst_mg_residual.argtypes = [_P, _P]
    L.pfasst_mg_get_solution.argtypes = [_P, _I, _I, _P, _I]
    L.pfasst_mg_get_state.argtypes = [_P, _I, _P]
    L.pfasst_mg_advance.argtypes = [_P]
    L.pfasst_mg_launch_count.argtypes = [_P]
    L.pfasst_mg_launch_count.restype = ctypes.c_longlong
    L.pfasst_mg_destroy.argtypes = [_P]
    L.pfasst_mg_last_error.argtypes = [_P]
    L.pfasst_mg_last_error.restype = ctypes.c_char_p
    L.pfasst_mg_helmholtz_solve.argtypes = [ctypes.POINTER(pmg_grid), _D, _I, _P, _P,
                                            ctypes.POINTER(pmg_options), _P, ctypes.POINTER(_I)]
    L.pfasst_mg_helmholtz_solve_noalloc.argtypes = [ctypes.POINTER(pmg_grid), _D, _I, _P, _P,
                                                    ctypes.POINTER(pmg_options), _P, ctypes.POINTER(_I)]
    L.pfasst_mg_batch_workspace_bytes.argtypes = [_I, ctypes.POINTER(pmg_problem_desc), ctypes.POINTER(pmg_options),
                                                  ctypes.POINTER(ctypes.c_size_t)]
    L.pfasst_mg_create_batch.argtypes = [_I, ctypes.POINTER(pmg_problem_desc), ctypes.POINTER(pmg_options), _P, _P,
                                         ctypes.c_size_t, ctypes.POINTER(_P)]
    L.pfasst_mg_batch_set_initial.argtypes = [_P, _I, _P, _I]
    L.pfasst_mg_batch_run.argtypes = [_P, _I, _I, _P]
    L.pfasst_mg_batch_get_solution.argtypes = [_P, _I, _P, _I]
    L.pfasst_mg_tuning.argtypes = [_P, _I, _I, ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_I)]
    L.pfasst_mg_set_tuning.argtypes = [_P, _I, _I, _I, _I, _I]
    L.pfasst_mg_profile.argtypes = [_P, _I, ctypes.c_longlong]
    L.pfasst_mg_profile_read.argtypes = [_P, ctypes.POINTER(pmg_kernel_stat), _I, ctypes.POINTER(_I)]
    L.pfasst_mg_kernel_name.argtypes = [_I]
    L.pfasst_mg_kernel_name.restype = ctypes.c_char_p
    _U64 = ctypes.c_ulonglong
    L.pfasst_mg_net_param_count.argtypes = []
    L.pfasst_mg_net_init.argtypes = [_P, _U64]
    L.pfasst_mg_net_create.argtypes = [_I, _I, _P, ctypes.POINTER(_P)]
    L.pfasst_mg_net_set_params.argtypes = [_P, _P]
    L.pfasst_mg_net_get_params.argtypes = [_P, _P]
    L.pfasst_mg_net_forward.argtypes = [_P, _P, _P, _I]
    L.pfasst_mg_net_gradients.argtypes = [_P, _P, _P, _P, _I, _I, _P, ctypes.POINTER(_D)]
    L.pfasst_mg_net_sample.argtypes = [_P, _U64, _D, _D, _I, _P, _P, _P, _I]
    L.pfasst_mg_net_train.argtypes = [_P, _I, _D, _U64, _D, _D, _I, _I, _I, _P]
    L.pfasst_mg_net_step.argtypes = [_P, _P, _P, _P, _I, _D, _I, _I, ctypes.POINTER(_D)]
    L.pfasst_mg_net_profile.argtypes = [_P, _I, ctypes.c_longlong]
    L.pfasst_mg_net_profile_read.argtypes = [_P, ctypes.POINTER(pmg_kernel_stat), _I, ctypes.POINTER(_I)]
    L.pfasst_mg_net_launch_count.argtypes = [_P]
    L.pfasst_mg_net_launch_count.restype = ctypes.c_longlong
    L.pfasst_mg_net_destroy.argtypes = [_P]
    L.pfasst_mg_net_last_error.argtypes = [_P]
    L.pfasst_mg_net_last_error.restype = ctypes.c_char_p
    L.pfasst_mg_set_smoother_net.argtypes = [_P, _P, _I, _I, ctypes.POINTER(_D), ctypes.POINTER(_D),
                                             ctypes.POINTER(_I)]
    L.pfasst_mg_check_narrowing.argtypes = [ctypes.c_longlong, ctypes.c_ulonglong, ctypes.POINTER(ctypes.c_longlong)]
    for name in EXPORTS:
        if name not in ("pfasst_mg_default_options", "pfasst_mg_launch_count", "pfasst_mg_last_error",
                        "pfasst_mg_kernel_name", "pfasst_mg_net_launch_count", "pfasst_mg_net_last_error"):
            getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


def _check(rc, h=None, allow=(PMG_OK,)):
    if rc not in allow:
        msg = load().pfasst_mg_last_error(h)
        raise PMGError(rc, msg.decode() if msg else "")
    return rc


def _stream_ptr(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _dev_ptr(t):
    import torch
    assert t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()
    return ctypes.c_void_p(t.data_ptr())


# ---------------------------------------------------------------- same-name wrappers

def pfasst_mg_default_options(**overrides) -> pmg_options:
    o = pmg_options()
    load().pfasst_mg_default_options(ctypes.byref(o))
    for k, v in overrides.items():
        setattr(o, k, v)
    return o


def pfasst_mg_workspace_bytes(grid, fine_nodes, levels, slices, opt) -> int:
    nb = ctypes.c_size_t(0)
    _check(load().pfasst_mg_workspace_bytes(ctypes.byref(grid), ctypes.byref(fine_nodes), ctypes.byref(levels),
                                            slices, ctypes.byref(opt), ctypes.byref(nb)))
    return nb.value


def pfasst_mg_create(grid, fine_nodes, levels, nu, dt, slices, opt, stream=None, workspace=None):
    """Returns (handle, workspace tensor).  The workspace is a torch uint8 CUDA tensor
    that must stay alive as long as the handle (the caller keeps it)."""
    import torch
    nbytes = pfasst_mg_workspace_bytes(grid, fine_nodes, levels, slices, opt)
    if workspace is None:
        workspace = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    h = ctypes.c_void_p()
    _check(load().pfasst_mg_create(ctypes.byref(grid), ctypes.byref(fine_nodes), ctypes.byref(levels), nu, dt,
                                   slices, ctypes.byref(opt), _stream_ptr(stream), ctypes.c_void_p(workspace.data_ptr()),
                                   nbytes, ctypes.byref(h)))
    return h, workspace


def pfasst_mg_set_initial(h, u0):
    """u0: torch CUDA float64 tensor (n^d) or numpy float64 array (host)."""
    import numpy as np
    if hasattr(u0, "is_cuda"):
        _check(load().pfasst_mg_set_initial(h, _dev_ptr(u0), 1), h)
    else:
        a = np.ascontiguousarray(u0, dtype=np.float64)
        _check(load().pfasst_mg_set_initial(h, a.ctypes.data_as(ctypes.c_void_p), 0), h)


def pfasst_mg_predict(h):
    _check(load().pfasst_mg_predict(h), h)


def pfasst_mg_sweep(h, level):
    _check(load().pfasst_mg_sweep(h, level), h)


def pfasst_mg_iterate(h, max_iter, tol):
    """Returns (status, iterations done, final max residual)."""
    it = ctypes.c_int(0)
    res = ctypes.c_double(0.0)
    rc = _check(load().pfasst_mg_iterate(h, max_iter, tol, ctypes.byref(it), ctypes.byref(res)), h,
                allow=(PMG_OK, PMG_NOT_CONVERGED))
    return rc, it.value, res.value


def pfasst_mg_residual(h, slices):
    import numpy as np
    out = np.zeros(slices)
    _check(load().pfasst_mg_residual(h, out.ctypes.data_as(ctypes.c_void_p)), h)
    return out


def pfasst_mg_get_solution(h, slice_, node, out):
    """out: torch CUDA float64 tensor or numpy float64 array of n^d values."""
    if hasattr(out, "is_cuda"):
        _check(load().pfasst_mg_get_solution(h, slice_, node, _dev_ptr(out), 1), h)
    else:
        _check(load().pfasst_mg_get_solution(h, slice_, node, out.ctypes.data_as(ctypes.c_void_p), 0), h)
    return out


def pfasst_mg_get_state(h, level, out):
    _check(load().pfasst_mg_get_state(h, level, out.ctypes.data_as(ctypes.c_void_p)), h)
    return out


def pfasst_mg_advance(h):
    _check(load().pfasst_mg_advance(h), h)


def pfasst_mg_launch_count(h) -> int:
    return load().pfasst_mg_launch_count(h)


def pfasst_mg_destroy(h):
    _check(load().pfasst_mg_destroy(h))


def pfasst_mg_last_error(h=None) -> str:
    m = load().pfasst_mg_last_error(h)
    return m.decode() if m else ""


def pfasst_mg_helmholtz_solve(grid, c, batch, b, u, opt, stream=None) -> int:
    """Solve (I - c Lap_h) u = b in place on u (torch CUDA float64, [batch, n^d]).
    Returns the number of V-cycles done."""
    cyc = ctypes.c_int(0)
    _check(load().pfasst_mg_helmholtz_solve(ctypes.byref(grid), c, batch, _dev_ptr(b), _dev_ptr(u),
                                            ctypes.byref(opt), _stream_ptr(stream), ctypes.byref(cyc)))
    return cyc.value


def pfasst_mg_helmholtz_solve_noalloc(grid, c, batch, b, u, opt, stream=None) -> int:
    """Same as pfasst_mg_helmholtz_solve, but takes its scratch from a fixed 32 MiB
    device array inside the library instead of allocating, for callers that may not
    allocate (inside stream capture, under a framework-owned allocator).  Queued on
    the stream, not synchronised.  Returns the number of V-cycles."""
    cyc = ctypes.c_int(0)
    _check(load().pfasst_mg_helmholtz_solve_noalloc(ctypes.byref(grid), c, batch, _dev_ptr(b), _dev_ptr(u),
                                                    ctypes.byref(opt), _stream_ptr(stream), ctypes.byref(cyc)))
    return cyc.value


def pfasst_mg_tuning(h, level, narrow=0):
    """(fused, param, threads) chosen for a multigrid level."""
    a, b, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(load().pfasst_mg_tuning(h, level, narrow, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)), h)
    return a.value, b.value, c.value


def pfasst_mg_set_tuning(h, level, narrow, fused, param, threads=256):
    _check(load().pfasst_mg_set_tuning(h, level, narrow, fused, param, threads), h)


def pfasst_mg_profile(h, enable, min_points=0):
    _check(load().pfasst_mg_profile(h, 1 if enable else 0, min_points), h)


def pfasst_mg_profile_read(h):
    """Returns a list of dicts: kernel name, n, precision, launches, points, ms."""
    cap = 256
    arr = (pmg_kernel_stat * cap)()
    cnt = ctypes.c_int(0)
    _check(load().pfasst_mg_profile_read(h, arr, cap, ctypes.byref(cnt)), h)
    return [dict(kernel=pfasst_mg_kernel_name(a.kernel), n=a.n, precision=a.precision, launches=a.launches,
                 points=a.points, ms=a.ms) for a in arr[:min(cnt.value, cap)]]


def pfasst_mg_check_narrowing(samples, seed=1):
    """Mismatches of the library's FP64 -> FP32 integer rounding against the hardware
    conversion on `samples` generated inputs (0 expected)."""
    bad = ctypes.c_longlong(-1)
    _check(load().pfasst_mg_check_narrowing(samples, seed, ctypes.byref(bad)))
    return bad.value


def pfasst_mg_check_widening():
    """Mismatches of the library's FP32 -> FP64 integer widening against the hardware
    conversion over all 2^32 float bit patterns (0 expected)."""
    bad = ctypes.c_longlong(-1)
    _check(load().pfasst_mg_check_widening(ctypes.byref(bad)))
    return bad.value


def pfasst_mg_fp64_peak(launches=5, stream=None) -> float:
    """Measured FP64 FMA throughput of the current device in GFLOP/s (best of `launches`)."""
    g = ctypes.c_double(0.0)
    L = load()
    L.pfasst_mg_fp64_peak.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_double)]
    _check(L.pfasst_mg_fp64_peak(_stream_ptr(stream), launches, ctypes.byref(g)))
    return g.value


def pfasst_mg_kernel_name(k) -> str:
    return load().pfasst_mg_kernel_name(k).decode()


def pfasst_mg_batch_workspace_bytes(probs, opt) -> int:
    arr = (pmg_problem_desc * len(probs))(*probs)
    nb = ctypes.c_size_t(0)
    _check(load().pfasst_mg_batch_workspace_bytes(len(probs), arr, ctypes.byref(opt), ctypes.byref(nb)))
    return nb.value


def pfasst_mg_create_batch(probs, opt, stream=None, workspace=None):
    """Returns (handle, workspace tensor) for a list of pmg_problem_desc."""
    import torch
    arr = (pmg_problem_desc * len(probs))(*probs)
    nbytes = pfasst_mg_batch_workspace_bytes(probs, opt)
    if workspace is None:
        workspace = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    h = ctypes.c_void_p()
    _check(load().pfasst_mg_create_batch(len(probs), arr, ctypes.byref(opt), _stream_ptr(stream),
                                         ctypes.c_void_p(workspace.data_ptr()), nbytes, ctypes.byref(h)))
    return h, workspace


def pfasst_mg_batch_set_initial(h, prob, u0):
    import numpy as np
    if hasattr(u0, "is_cuda"):
        _check(load().pfasst_mg_batch_set_initial(h, prob, _dev_ptr(u0), 1), h)
    else:
        a = np.ascontiguousarray(u0, dtype=np.float64)
        _check(load().pfasst_mg_batch_set_initial(h, prob, a.ctypes.data_as(ctypes.c_void_p), 0), h)


def pfasst_mg_batch_run(h, steps, sweeps, nprob):
    import numpy as np
    res = np.zeros(nprob)
    _check(load().pfasst_mg_batch_run(h, steps, sweeps, res.ctypes.data_as(ctypes.c_void_p)), h)
    return res


def pfasst_mg_batch_get_solution(h, prob, out):
    if hasattr(out, "is_cuda"):
        _check(load().pfasst_mg_batch_get_solution(h, prob, _dev_ptr(out), 1), h)
    else:
        _check(load().pfasst_mg_batch_get_solution(h, prob, out.ctypes.data_as(ctypes.c_void_p), 0), h)
    return out


class BatchSolver:
    """Owns an uneven-batch handle (independent single-level SDC problems)."""

    def __init__(self, problems, stream=None, **opts):
        """problems: list of (dim, n, nodes, nu, dt)."""
        self.problems = list(problems)
        self.opt = pfasst_mg_default_options(**opts)
        descs = [pmg_problem_desc(pmg_grid(d, n), m, nu, dt) for (d, n, m, nu, dt) in self.problems]
        self.h, self.workspace = pfasst_mg_create_batch(descs, self.opt, stream)

    def set_initial(self, prob, u0):
        pfasst_mg_batch_set_initial(self.h, prob, u0)

    def run(self, steps, sweeps):
        return pfasst_mg_batch_run(self.h, steps, sweeps, len(self.problems))

    def solution(self, prob):
        import numpy as np
        d, n = self.problems[prob][0], self.problems[prob][1]
        return pfasst_mg_batch_get_solution(self.h, prob, np.zeros(n ** d))

    def launches(self):
        return pfasst_mg_launch_count(self.h)

    def close(self):
        if self.h:
            pfasst_mg_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------- convenience handle

# ---------------------------------------------------------------- learned correction network

def _ncheck(rc, h=None):
    if rc != PMG_OK:
        msg = load().pfasst_mg_net_last_error(h)
        raise PMGError(rc, msg.decode() if msg else "")
    return rc


def _f32(a, size):
    import numpy as np
    a = np.ascontiguousarray(a, dtype=np.float32)
    assert a.size == size, (a.size, size)
    return a


def pfasst_mg_net_param_count() -> int:
    return load().pfasst_mg_net_param_count()


def pfasst_mg_net_init(seed):
    import numpy as np
    p = np.zeros(NET_PARAMS, dtype=np.float32)
    _ncheck(load().pfasst_mg_net_init(p.ctypes.data_as(ctypes.c_void_p), seed))
    return p


def pfasst_mg_net_create(batch, n, stream=None):
    h = ctypes.c_void_p()
    _ncheck(load().pfasst_mg_net_create(batch, n, _stream_ptr(stream), ctypes.byref(h)))
    return h


def pfasst_mg_net_set_params(h, params):
    p = _f32(params, NET_PARAMS)
    _ncheck(load().pfasst_mg_net_set_params(h, p.ctypes.data_as(ctypes.c_void_p)), h)


def pfasst_mg_net_get_params(h):
    import numpy as np
    p = np.zeros(NET_PARAMS, dtype=np.float32)
    _ncheck(load().pfasst_mg_net_get_params(h, p.ctypes.data_as(ctypes.c_void_p)), h)
    return p


def pfasst_mg_net_forward(h, x, npts):
    """x: host float array of npts = batch * n^3 values; returns y (host)."""
    import numpy as np
    xa = _f32(x, npts)
    y = np.zeros(npts, dtype=np.float32)
    _ncheck(load().pfasst_mg_net_forward(h, xa.ctypes.data_as(ctypes.c_void_p), y.ctypes.data_as(ctypes.c_void_p),
                                         0), h)
    return y


def pfasst_mg_net_gradients(h, x, t, kappa, npts, power=1):
    """Host arrays; returns (loss, grad[7809])."""
    import numpy as np
    xa, ta = _f32(x, npts), _f32(t, npts)
    ka = np.ascontiguousarray(kappa, dtype=np.float32)
    g = np.zeros(NET_PARAMS, dtype=np.float32)
    loss = ctypes.c_double(0.0)
    _ncheck(load().pfasst_mg_net_gradients(h, xa.ctypes.data_as(ctypes.c_void_p), ta.ctypes.data_as(ctypes.c_void_p),
                                           ka.ctypes.data_as(ctypes.c_void_p), power, 0,
                                           g.ctypes.data_as(ctypes.c_void_p),
                                           ctypes.byref(loss)), h)
    return loss.value, g


def pfasst_mg_net_sample(h, seed, kappa_lo, kappa_hi, batch, npts, vcycles_max=0):
    """Returns host arrays (x, t, kappa)."""
    import numpy as np
    x = np.zeros(npts, dtype=np.float32)
    t = np.zeros(npts, dtype=np.float32)
    k = np.zeros(batch, dtype=np.float32)
    _ncheck(load().pfasst_mg_net_sample(h, seed, kappa_lo, kappa_hi, vcycles_max, x.ctypes.data_as(ctypes.c_void_p),
                                        t.ctypes.data_as(ctypes.c_void_p), k.ctypes.data_as(ctypes.c_void_p), 0), h)
    return x, t, k


def pfasst_mg_net_train(h, steps, lr, seed, kappa_lo, kappa_hi, vcycles_max=0, power=2, train_bias=0):
    """Returns the loss of every step (host)."""
    import numpy as np
    hist = np.zeros(steps)
    _ncheck(load().pfasst_mg_net_train(h, steps, lr, seed, kappa_lo, kappa_hi, vcycles_max, power, train_bias,
                                       hist.ctypes.data_as(ctypes.c_void_p)), h)
    return hist


def pfasst_mg_net_step(h, x, t, kappa, npts, power=1, lr=1e-3, train_bias=0):
    """One Adam step on host arrays x, t (npts floats) and kappa; returns the loss."""
    import numpy as np
    xa, ta = _f32(x, npts), _f32(t, npts)
    ka = np.ascontiguousarray(kappa, dtype=np.float32)
    loss = ctypes.c_double(0.0)
    _ncheck(load().pfasst_mg_net_step(h, xa.ctypes.data_as(ctypes.c_void_p), ta.ctypes.data_as(ctypes.c_void_p),
                                      ka.ctypes.data_as(ctypes.c_void_p), power, lr, train_bias, 0,
                                      ctypes.byref(loss)), h)
    return loss.value


def _is_dev(a):
    try:
        import torch
        return isinstance(a, torch.Tensor) and a.is_cuda
    except ImportError:
        return False


def pfasst_mg_net_step_dev(h, x, t, kappa, power=1, lr=1e-3, train_bias=0):
    """One Adam step on device tensors x, t (float32, contiguous, [batch][n^3]) and host
    kappa; returns the loss."""
    import numpy as np
    assert _is_dev(x) and _is_dev(t) and x.is_contiguous() and t.is_contiguous()
    ka = np.ascontiguousarray(kappa, dtype=np.float32)
    loss = ctypes.c_double(0.0)
    _ncheck(load().pfasst_mg_net_step(h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(t.data_ptr()),
                                      ka.ctypes.data_as(ctypes.c_void_p), power, lr, train_bias, 1,
                                      ctypes.byref(loss)), h)
    return loss.value


def pfasst_mg_net_substep_pairs(h, u0, kappa, x, t):
    """Sub-step training pairs (see include/pfasst_mg.h): u0 float64 [batch][n^3], x and t
    float32 outputs of the same shape -- all device tensors, or all host numpy arrays;
    kappa host floats, one per grid."""
    import numpy as np
    ka = np.ascontiguousarray(kappa, dtype=np.float32)
    dev = _is_dev(u0)
    if dev:
        assert _is_dev(x) and _is_dev(t) and u0.is_contiguous() and x.is_contiguous() and t.is_contiguous()
        ptr = lambda a: ctypes.c_void_p(a.data_ptr())  # noqa: E731
    else:
        assert u0.dtype == np.float64 and x.dtype == np.float32 and t.dtype == np.float32
        ptr = lambda a: a.ctypes.data_as(ctypes.c_void_p)  # noqa: E731
    _ncheck(load().pfasst_mg_net_substep_pairs(h, ptr(u0), ka.ctypes.data_as(ctypes.c_void_p), ptr(x), ptr(t),
                                               1 if dev else 0), h)


def pfasst_mg_net_profile(h, enable, min_points=0):
    _ncheck(load().pfasst_mg_net_profile(h, enable, min_points), h)


def pfasst_mg_net_profile_read(h):
    """Returns a list of dicts {kernel, n, precision, launches, points, ms}."""
    cap = 64
    arr = (pmg_kernel_stat * cap)()
    cnt = ctypes.c_int(0)
    _ncheck(load().pfasst_mg_net_profile_read(h, arr, cap, ctypes.byref(cnt)), h)
    return [dict(kernel=pfasst_mg_kernel_name(a.kernel), n=a.n, precision=a.precision, launches=a.launches,
                 points=a.points, ms=a.ms) for a in arr[:min(cnt.value, cap)]]


def pfasst_mg_net_launch_count(h) -> int:
    return load().pfasst_mg_net_launch_count(h)


def pfasst_mg_net_destroy(h):
    _ncheck(load().pfasst_mg_net_destroy(h))


def pfasst_mg_net_last_error(h=None) -> str:
    m = load().pfasst_mg_net_last_error(h)
    return m.decode() if m else ""


def pfasst_mg_set_smoother_net(h, params, min_n=15, calibrate=1):
    """Deploy params (or remove with None); returns (rho_plain, rho_net, level_mask)."""
    rp, rn, mask = ctypes.c_double(0.0), ctypes.c_double(0.0), ctypes.c_int(0)
    ptr = None
    if params is not None:
        p = _f32(params, NET_PARAMS)
        ptr = p.ctypes.data_as(ctypes.c_void_p)
    _check(load().pfasst_mg_set_smoother_net(h, ptr, min_n, calibrate, ctypes.byref(rp), ctypes.byref(rn),
                                             ctypes.byref(mask)), h)
    return rp.value, rn.value, mask.value


class NetTrainer:
    """Owns a pmg_net trainer handle (batch of n^3 grids); methods call the C ABI."""

    def __init__(self, batch, n, stream=None):
        self.batch, self.n = batch, n
        self.npts = batch * n ** 3
        self.h = pfasst_mg_net_create(batch, n, stream)

    def set_params(self, p):
        pfasst_mg_net_set_params(self.h, p)

    def params(self):
        return pfasst_mg_net_get_params(self.h)

    def forward(self, x):
        return pfasst_mg_net_forward(self.h, x, self.npts)

    def gradients(self, x, t, kappa, power=1):
        return pfasst_mg_net_gradients(self.h, x, t, kappa, self.npts, power)

    def sample(self, seed, kappa_lo, kappa_hi, vcycles_max=0):
        return pfasst_mg_net_sample(self.h, seed, kappa_lo, kappa_hi, self.batch, self.npts, vcycles_max)

    def train(self, steps, lr, seed, kappa_lo, kappa_hi, vcycles_max=0, power=2, train_bias=0):
        return pfasst_mg_net_train(self.h, steps, lr, seed, kappa_lo, kappa_hi, vcycles_max, power, train_bias)

    def profile(self, enable, min_points=0):
        pfasst_mg_net_profile(self.h, enable, min_points)

    def profile_read(self):
        return pfasst_mg_net_profile_read(self.h)

    def step(self, x, t, kappa, power=1, lr=1e-3, train_bias=0):
        if _is_dev(x):
            return pfasst_mg_net_step_dev(self.h, x, t, kappa, power, lr, train_bias)
        return pfasst_mg_net_step(self.h, x, t, kappa, self.npts, power, lr, train_bias)

    def substep_pairs(self, u0, kappa, x, t):
        pfasst_mg_net_substep_pairs(self.h, u0, kappa, x, t)

    def launches(self):
        return pfasst_mg_net_launch_count(self.h)

    def close(self):
        if self.h:
            pfasst_mg_net_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class PFASSTSolver:
    """Owns a pfasst_mg handle and its torch workspace; methods call the C ABI."""

    def __init__(self, dim, n, fine_nodes, coarse_nodes, slices, nu, dt, nlevels=2, stream=None, family=0,
                 coarsest_nodes=0, order=2, **opts):
        """family: 0 Gauss-Lobatto nodes, 1 the uniform family (every level);
        coarsest_nodes: node count of level 2 when nlevels == 3; order: Laplacian stencil
        of the fine level (2 or 4)."""
        self.dim, self.n, self.sf, self.sc, self.s2 = dim, n, fine_nodes, coarse_nodes, coarsest_nodes
        self.slices, self.nu, self.dt, self.nlevels = slices, nu, dt, nlevels
        self.opt = pfasst_mg_default_options(**opts)
        self.grid = pmg_grid(dim, n, order)
        self.fnodes = pmg_nodes_desc(fine_nodes, family)
        self.levels = pmg_levels(nlevels, pmg_nodes_desc(coarse_nodes if nlevels >= 2 else 0, family),
                                 pmg_nodes_desc(coarsest_nodes if nlevels == 3 else 0, family))
        self.h, self.workspace = pfasst_mg_create(self.grid, self.fnodes, self.levels, nu, dt, slices, self.opt, stream)

    @property
    def npts(self):
        return self.n ** self.dim

    def set_initial(self, u0):
        pfasst_mg_set_initial(self.h, u0)

    def predict(self):
        pfasst_mg_predict(self.h)

    def sweep(self, level=0):
        pfasst_mg_sweep(self.h, level)

    def iterate(self, max_iter, tol):
        return pfasst_mg_iterate(self.h, max_iter, tol)

    def residual(self):
        return pfasst_mg_residual(self.h, self.slices)

    def solution(self, slice_, node):
        import numpy as np
        return pfasst_mg_get_solution(self.h, slice_, node, np.zeros(self.npts))

    def state(self, level=0):
        import numpy as np
        s = (self.sf, self.sc, self.s2)[level]
        n = self.n
        for _ in range(level):
            n = (n - 1) // 2
        return pfasst_mg_get_state(self.h, level, np.zeros((self.slices, s, n ** self.dim)))

    def advance(self):
        pfasst_mg_advance(self.h)

    def set_smoother_net(self, params, min_n=15, calibrate=1):
        return pfasst_mg_set_smoother_net(self.h, params, min_n, calibrate)

    def launches(self):
        return pfasst_mg_launch_count(self.h)

    def close(self):
        if self.h:
            pfasst_mg_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
