"""GPU parity of the fourth-order Laplacian (Sec. 4.2): V-cycles whose finest grid
carries the 5-point-per-axis stencil (three-colour Gauss-Seidel or weighted Jacobi,
second-order coarse grids), and PFASST / SDC with a fourth-order fine level, against
the FP64 oracle through the C ABI.  Tolerances as in test_gpu_parity: FP64 paths agree
to rounding order (relative l2 <= 1e-12), FP32 V-cycles to FP32 accuracy."""
import math

import numpy as np
import pytest

import oracle as O
from parity import worst_rel
import paper_1407_6486_gb300 as pmg
from paper_1407_6486_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

FP64_TOL = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1407_6486_gb300 import _build
    _build.build()
    pmg.load()


def rel(a, b):
    """Worst relative l2 error over the grid functions (slices, nodes, grids) of a."""
    return worst_rel(a, b)


def omega(sm):
    return 1.0 if sm == 1 else 2.0 / 3.0


@pytest.mark.parametrize("dim,n,sm,vc,batch", [
    (1, 7, 1, 1, 3), (1, 63, 0, 2, 3), (1, 255, 1, 2, 2), (2, 31, 1, 1, 3), (2, 63, 0, 2, 2), (3, 15, 1, 2, 3),
    (3, 31, 0, 1, 2), (3, 63, 1, 2, 4), (3, 127, 1, 1, 2),
])
def test_vcycles_fp64_match_oracle(dim, n, sm, vc, batch):
    c = 0.37 / (n + 1) ** 2 * 4
    rng = np.random.default_rng(dim * 1000 + n + 4)
    b = rng.standard_normal((batch, n ** dim))
    u = rng.standard_normal((batch, n ** dim))
    opt = pmg.pfasst_mg_default_options(smoother=sm, omega=omega(sm), vcycles=vc)
    ut = torch.tensor(u, device="cuda")
    assert pmg.pfasst_mg_helmholtz_solve(pmg.pmg_grid(dim, n, 4), c, batch, torch.tensor(b, device="cuda"), ut,
                                         opt) == vc
    mg = O.MGParams(smoother=sm, omega=omega(sm), vcycles=vc)
    want = np.stack([O.mg_solve(mg, dim, n, c, b[q], u[q], order=4)[0] for q in range(batch)])
    assert rel(ut.cpu().numpy(), want) < FP64_TOL


@pytest.mark.parametrize("dim,n,sm", [(1, 127, 0), (2, 63, 1), (3, 31, 1)])
def test_full_solve_matches_oracle(dim, n, sm):
    batch, c = 2, 0.01
    b = np.random.default_rng(8).standard_normal((batch, n ** dim))
    opt = pmg.pfasst_mg_default_options(smoother=sm, omega=omega(sm), vcycles=0, mg_tol=1e-12)
    ut = torch.zeros((batch, n ** dim), dtype=torch.float64, device="cuda")
    cyc = pmg.pfasst_mg_helmholtz_solve(pmg.pmg_grid(dim, n, 4), c, batch, torch.tensor(b, device="cuda"), ut, opt)
    mg = O.MGParams(smoother=sm, omega=omega(sm), vcycles=0, mg_tol=1e-12)
    outs = [O.mg_solve(mg, dim, n, c, b[q], np.zeros(n ** dim), order=4) for q in range(batch)]
    assert cyc == max(o[1] for o in outs)
    assert rel(ut.cpu().numpy(), np.stack([o[0] for o in outs])) < 1e-11


@pytest.mark.parametrize("dim,n,sm,batch", [(2, 127, 0, 2), (3, 63, 1, 3)])
def test_mixed_vcycle_and_refinement(dim, n, sm, batch):
    c = 0.02
    b = np.random.default_rng(12).standard_normal((batch, n ** dim))
    g = pmg.pmg_grid(dim, n, 4)
    ut = torch.zeros((batch, n ** dim), dtype=torch.float64, device="cuda")
    pmg.pfasst_mg_helmholtz_solve(g, c, batch, torch.tensor(b, device="cuda"), ut,
                                  pmg.pfasst_mg_default_options(smoother=sm, omega=omega(sm), vcycles=1, precision=1))
    mg1 = O.MGParams(smoother=sm, omega=omega(sm), vcycles=1)
    want1 = np.stack([O.mg_solve(mg1, dim, n, c, b[q], np.zeros(n ** dim), order=4)[0] for q in range(batch)])
    assert rel(ut.cpu().numpy(), want1) < 2e-6
    ut.zero_()
    pmg.pfasst_mg_helmholtz_solve(g, c, batch, torch.tensor(b, device="cuda"), ut,
                                  pmg.pfasst_mg_default_options(smoother=sm, omega=omega(sm), vcycles=0, precision=1,
                                                                mg_tol=1e-12))
    mgf = O.MGParams(smoother=sm, omega=omega(sm), vcycles=0, mg_tol=1e-14, mg_maxcycles=80)
    wantf = np.stack([O.mg_solve(mgf, dim, n, c, b[q], np.zeros(n ** dim), order=4)[0] for q in range(batch)])
    assert rel(ut.cpu().numpy(), wantf) < 1e-11


def _u0(dim, n):
    modes, amps = inputs.random_modes(dim, 4, 4, 99)
    return inputs.sine_sum(dim, n, modes, amps)


CASES = [
    # dim, n, sf, sc, P, nlevels, smoother, vcycles, interp
    (1, 63, 5, 3, 3, 2, 0, 2, 4),
    (2, 31, 5, 3, 4, 2, 1, 2, 4),
    (3, 15, 5, 3, 2, 2, 1, 2, 4),
    (3, 31, 3, 2, 3, 2, 1, 1, 2),
    (2, 31, 3, 0, 3, 1, 0, 2, 4),
    (2, 31, 5, 3, 3, 2, 1, 0, 4),     # sub-steps solved to 1e-12: F stored, colloc residual from F
]


@pytest.mark.parametrize("case", CASES, ids=[f"d{c[0]}n{c[1]}s{c[2]}x{c[3]}L{c[5]}sm{c[6]}v{c[7]}" for c in CASES])
def test_pfasst_with_a_fourth_order_fine_level_matches_oracle(case):
    dim, n, sf, sc, P, nl, sm, vc, interp = case
    kw = dict(smoother=sm, omega=omega(sm), vcycles=vc, interp_order=interp)
    if vc == 0:
        kw["mg_tol"] = 1e-12
    s = pmg.PFASSTSolver(dim, n, sf, sc if nl == 2 else 0, P, 1.0, 0.01, nlevels=nl, order=4, **kw)
    mg = O.MGParams(smoother=sm, omega=omega(sm), vcycles=vc, mg_tol=1e-12)
    o = O.PFASST(dim, n, sf, sc if nl == 2 else 2, P, 1.0, 0.01, mg, nlevels=nl, interp_order=interp, order=4)
    u0 = _u0(dim, n)
    s.set_initial(u0)
    o.set_initial(u0)
    s.predict()
    o.predict()
    assert rel(s.state(0), o.Uf) < FP64_TOL
    tol = FP64_TOL if vc > 0 else 1e-10  # full solves: the stopping test may differ by a cycle at the margin
    for k in range(3):
        s.iterate(1, 0.0)
        ores = o.iteration()
        assert rel(s.state(0), o.Uf) < tol, f"iteration {k}"
        if nl == 2:
            assert rel(s.state(1), o.Uc) < tol
        np.testing.assert_allclose(s.residual(), ores, rtol=1e-7, atol=1e-13)
    s.close()


def test_three_levels_with_a_fourth_order_fine_level_match_oracle():
    dim, n, P, nodes = 2, 31, 3, (5, 3, 2)
    s = pmg.PFASSTSolver(dim, n, nodes[0], nodes[1], P, 1.0, 0.01, nlevels=3, coarsest_nodes=nodes[2], order=4,
                         smoother=1, omega=1.0, vcycles=2)
    o = O.MLPFASST(dim, n, list(nodes), P, 1.0, 0.01, O.MGParams(smoother=1, omega=1.0, vcycles=2), order=4)
    u0 = _u0(dim, n)
    s.set_initial(u0)
    o.set_initial(u0)
    s.predict()
    o.predict()
    for k in range(3):
        s.iterate(1, 0.0)
        o.iteration()
        for l in range(3):
            assert rel(s.state(l), o.U[l]) < FP64_TOL, (k, l)
    s.close()


def test_3d_fixed_point_is_the_fourth_order_collocation_solution_mixed():
    """3D heat, mixed precision, fourth-order fine level, second-order coarse level:
    PFASST converges on every sine mode to Pade(z4)^P with z4 = dt nu lambda_4(k)."""
    wl = inputs.heat3d_c3(n=63, slices=4)
    s = pmg.PFASSTSolver(3, wl.n, 5, 3, wl.slices, wl.nu, wl.dt, order=4, smoother=1, omega=1.0, vcycles=2,
                         precision=1)
    s.set_initial(wl.u0())
    rc, it, res = s.iterate(200, 1e-10)
    assert rc == pmg.PMG_OK, (it, res)
    n, h = wl.n, 1.0 / (wl.n + 1)
    x = np.arange(1, n + 1) * h

    def pade44(z):
        return (1 + z / 2 + 3 * z * z / 28 + z ** 3 / 84 + z ** 4 / 1680) / (
            1 - z / 2 + 3 * z * z / 28 - z ** 3 / 84 + z ** 4 / 1680)

    want = np.zeros((n, n, n))
    for k, a in zip(wl.modes, wl.amps):
        lam = sum((-2 * math.cos(2 * kk * math.pi * h) + 32 * math.cos(kk * math.pi * h) - 30) / (12 * h * h)
                  for kk in k)
        want += a * pade44(wl.dt * wl.nu * lam) ** wl.slices * np.einsum(
            "k,j,i->kji", np.sin(k[2] * np.pi * x), np.sin(k[1] * np.pi * x), np.sin(k[0] * np.pi * x))
    end = s.solution(wl.slices - 1, 4).reshape(n, n, n)
    assert np.abs(end - want).max() <= 1e-8 * np.abs(want).max()
    s.close()


def test_fourth_order_level_keeps_the_per_point_smoothers():
    s = pmg.PFASSTSolver(3, 127, 5, 3, 4, 0.5, 0.002, order=4, smoother=1, omega=1.0, vcycles=2, precision=1)
    fused, _, _ = pmg.pfasst_mg_tuning(s.h, 0)
    assert fused == 0
    with pytest.raises(pmg.PMGError):
        pmg.pfasst_mg_set_tuning(s.h, 0, 0, 1, 16, 256)
    s.close()
