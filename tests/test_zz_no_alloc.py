"""The allocation-free multigrid solve against the allocating one.

pfasst_mg_helmholtz_solve_noalloc exists for callers that cannot allocate device
memory (applications whose own pool allocator holds all GPU memory, real-time loops in
which an allocation would synchronise the device); it must give the same results as
pfasst_mg_helmholtz_solve, call after call,
although every call reuses the same fixed scratch array.  This file is collected
last so that a failure here comes after every other test has run.
"""
import ctypes

import numpy as np
import pytest

import paper_1407_6486_gb300 as pmg

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

FP64_TOL = 1e-12


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1407_6486_gb300 import _build
    _build.build()
    return pmg.load()


def _solve(lib, fn, dim, n, c, b, u, opt):
    """Call one of the two C entry points directly; returns (rc, cycles)."""
    cyc = ctypes.c_int(0)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = getattr(lib, fn)(ctypes.byref(pmg.pmg_grid(dim, n)), c, b.shape[0], ctypes.c_void_p(b.data_ptr()),
                          ctypes.c_void_p(u.data_ptr()), ctypes.byref(opt), stream, ctypes.byref(cyc))
    torch.cuda.synchronize()
    return rc, cyc.value


@pytest.mark.parametrize("dim,n,batch,smoother,precision", [
    (3, 31, 4, 1, 0), (2, 127, 3, 0, 0), (1, 1023, 2, 1, 0), (3, 15, 6, 0, 1),
])
def test_noalloc_matches_allocating_solve_on_two_calls_in_a_row(lib, dim, n, batch, smoother, precision):
    opt = pmg.pfasst_mg_default_options(smoother=smoother, omega=1.0 if smoother else 2.0 / 3.0, vcycles=2,
                                        precision=precision)
    c = 0.5 / (n + 1) ** 2
    rng = np.random.default_rng(100 * dim + n)
    for call in range(2):
        b = torch.tensor(rng.standard_normal((batch, n ** dim)), device="cuda")
        u0 = torch.tensor(rng.standard_normal((batch, n ** dim)), device="cuda")
        u_ref, u_new = u0.clone(), u0.clone()
        rc_ref, cyc_ref = _solve(lib, "pfasst_mg_helmholtz_solve", dim, n, c, b, u_ref, opt)
        rc_new, cyc_new = _solve(lib, "pfasst_mg_helmholtz_solve_noalloc", dim, n, c, b, u_new, opt)
        assert rc_ref == pmg.PMG_OK and rc_new == pmg.PMG_OK, pmg.pfasst_mg_last_error()
        assert cyc_new == cyc_ref == 2
        err = (torch.linalg.norm(u_new - u_ref) / torch.linalg.norm(u_ref)).item()
        assert err <= FP64_TOL, f"call {call}: rel l2 {err:.3e}"
        assert (u_new - u0).abs().max().item() > 0.0


def test_noalloc_rejects_problems_beyond_its_scratch(lib):
    opt = pmg.pfasst_mg_default_options(vcycles=1)
    b = torch.zeros((1, 255 ** 3), dtype=torch.float64, device="cuda")
    u = torch.zeros_like(b)
    rc, _ = _solve(lib, "pfasst_mg_helmholtz_solve_noalloc", 3, 255, 1e-4, b, u, opt)
    assert rc == pmg.PMG_ERR_INVALID_ARG
    assert "32 MiB" in pmg.pfasst_mg_last_error()


def test_noalloc_rejects_tolerance_mode(lib):
    opt = pmg.pfasst_mg_default_options(vcycles=0)
    b = torch.zeros((1, 15 ** 2), dtype=torch.float64, device="cuda")
    u = torch.zeros_like(b)
    rc, _ = _solve(lib, "pfasst_mg_helmholtz_solve_noalloc", 2, 15, 1e-3, b, u, opt)
    assert rc == pmg.PMG_ERR_UNSUPPORTED
