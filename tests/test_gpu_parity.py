"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Tolerances: the FP64 path follows the oracle's algorithm step for step with fixed
V-cycle counts, so the two differ only by rounding order: relative l2 <= 1e-12 on
every compared state.  The mixed path (FP32 V-cycles, FP64 residuals, iterative
refinement) converges to the same fixed point: <= 1e-9 relative l2 once both are
converged to a collocation residual of 1e-12.
"""
import math

import numpy as np
import pytest

import oracle as O
from parity import ulp_perturbed, worst_rel, worst_rel_floor
import paper_1407_6486_gb300 as pmg
from paper_1407_6486_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

FP64_TOL = 1e-12
MIXED_TOL = 1e-9


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


# ---------------------------------------------------------------- multigrid alone

@pytest.mark.parametrize("dim,n,sm,vc,batch", [
    (1, 3, 0, 1, 3), (1, 63, 0, 2, 3), (1, 1023, 1, 2, 3), (2, 31, 0, 1, 3), (2, 255, 1, 2, 3), (2, 127, 0, 3, 3),
    (3, 7, 1, 1, 3), (3, 15, 0, 2, 3), (3, 31, 1, 2, 3), (3, 63, 0, 1, 3), (3, 63, 1, 2, 3), (3, 127, 1, 1, 3),
    # large enough batches for the tiled z-marching kernels (partial tiles in y and z)
    (3, 127, 1, 2, 9), (3, 63, 1, 2, 70),
])
def test_vcycles_fp64_match_oracle(dim, n, sm, vc, batch):
    c = 0.37 / (n + 1) ** 2 * 4
    rng = np.random.default_rng(dim * 1000 + n)
    b = rng.standard_normal((batch, n ** dim))
    u = rng.standard_normal((batch, n ** dim))
    opt = pmg.pfasst_mg_default_options(smoother=sm, omega=omega(sm), vcycles=vc)
    bt = torch.tensor(b, device="cuda")
    ut = torch.tensor(u, device="cuda")
    cyc = pmg.pfasst_mg_helmholtz_solve(pmg.pmg_grid(dim, n), c, batch, bt, ut, opt)
    assert cyc == vc
    mg = O.MGParams(smoother=sm, omega=omega(sm), vcycles=vc)
    want = np.stack([O.mg_solve(mg, dim, n, c, b[q], u[q])[0] for q in range(batch)])
    assert rel(ut.cpu().numpy(), want) < FP64_TOL


@pytest.mark.parametrize("dim,n,sm", [(1, 127, 0), (2, 63, 1), (3, 15, 0)])
def test_full_solve_matches_oracle(dim, n, sm):
    batch, c = 2, 0.01
    rng = np.random.default_rng(7)
    b = rng.standard_normal((batch, n ** dim))
    opt = pmg.pfasst_mg_default_options(smoother=sm, omega=omega(sm), vcycles=0, mg_tol=1e-12)
    ut = torch.zeros((batch, n ** dim), dtype=torch.float64, device="cuda")
    cyc = pmg.pfasst_mg_helmholtz_solve(pmg.pmg_grid(dim, n), c, batch, torch.tensor(b, device="cuda"), ut, opt)
    mg = O.MGParams(smoother=sm, omega=omega(sm), vcycles=0, mg_tol=1e-12)
    outs = [O.mg_solve(mg, dim, n, c, b[q], np.zeros(n ** dim)) for q in range(batch)]
    assert cyc == max(o[1] for o in outs)
    assert rel(ut.cpu().numpy(), np.stack([o[0] for o in outs])) < 1e-11


@pytest.mark.parametrize("dim,n,sm,batch", [(2, 127, 0, 2), (3, 31, 1, 2), (3, 127, 1, 9)])
def test_mixed_vcycle_and_refinement(dim, n, sm, batch):
    """FP32 V-cycles: one cycle matches the FP64 oracle to FP32 accuracy; the full solve
    (FP64 residual, FP32 correction) refines to the FP64 solution."""
    c = 0.02
    rng = np.random.default_rng(11)
    b = rng.standard_normal((batch, n ** dim))
    g = pmg.pmg_grid(dim, n)
    ut = torch.zeros((batch, n ** dim), dtype=torch.float64, device="cuda")
    opt1 = pmg.pfasst_mg_default_options(smoother=sm, omega=omega(sm), vcycles=1, precision=1)
    pmg.pfasst_mg_helmholtz_solve(g, c, batch, torch.tensor(b, device="cuda"), ut, opt1)
    mg1 = O.MGParams(smoother=sm, omega=omega(sm), vcycles=1)
    want1 = np.stack([O.mg_solve(mg1, dim, n, c, b[q], np.zeros(n ** dim))[0] for q in range(batch)])
    assert rel(ut.cpu().numpy(), want1) < 2e-6
    ut.zero_()
    optf = pmg.pfasst_mg_default_options(smoother=sm, omega=omega(sm), vcycles=0, precision=1, mg_tol=1e-12)
    pmg.pfasst_mg_helmholtz_solve(g, c, batch, torch.tensor(b, device="cuda"), ut, optf)
    mgf = O.MGParams(smoother=sm, omega=omega(sm), vcycles=0, mg_tol=1e-14, mg_maxcycles=60)
    wantf = np.stack([O.mg_solve(mgf, dim, n, c, b[q], np.zeros(n ** dim))[0] for q in range(batch)])
    assert rel(ut.cpu().numpy(), wantf) < 1e-11


# ---------------------------------------------------------------- SDC / PFASST

CASES = [
    # dim, n, sf, sc, P, nlevels, smoother, vcycles, interp
    (1, 63, 5, 3, 3, 2, 0, 2, 4),
    (2, 31, 5, 3, 4, 2, 0, 1, 4),
    (2, 63, 3, 2, 2, 2, 1, 2, 2),
    (3, 15, 5, 3, 4, 2, 1, 2, 4),
    (3, 7, 3, 2, 2, 2, 0, 1, 4),
    (2, 31, 3, 0, 3, 1, 0, 2, 4),
    (1, 127, 9, 3, 2, 2, 1, 1, 4),
    # one slice, two levels: MLSDC (Sec. 2.3), the predictor is one coarse sweep
    (2, 31, 5, 3, 1, 2, 1, 2, 4),
    (3, 15, 5, 3, 1, 2, 0, 1, 4),
]


def _u0(dim, n):
    modes, amps = inputs.random_modes(dim, 4, 4, 99)
    return inputs.sine_sum(dim, n, modes, amps)


def _pair(dim, n, sf, sc, P, nl, sm, vc, interp, precision=0, dt=0.01, nu=1.0, with_pert=False):
    """GPU solver and oracle on the same u0; with_pert: also an oracle started from u0
    moved by one ulp (the conditioning floor of the comparison)."""
    s = pmg.PFASSTSolver(dim, n, sf, sc if nl == 2 else 0, P, nu, dt, nlevels=nl, smoother=sm, omega=omega(sm),
                         vcycles=vc, precision=precision, interp_order=interp)

    def orc(u):
        o = O.PFASST(dim, n, sf, sc if nl == 2 else 2, P, nu, dt,
                     O.MGParams(smoother=sm, omega=omega(sm), vcycles=vc), nlevels=nl, interp_order=interp)
        o.set_initial(u)
        return o

    u0 = _u0(dim, n)
    s.set_initial(u0)
    if with_pert:
        return s, orc(u0), orc(ulp_perturbed(u0))
    return s, orc(u0)


@pytest.mark.parametrize("case", CASES, ids=[f"d{c[0]}n{c[1]}s{c[2]}x{c[3]}P{c[4]}L{c[5]}sm{c[6]}v{c[7]}" for c in CASES])
def test_pfasst_state_matches_oracle_every_iteration(case):
    dim, n, sf, sc, P, nl, sm, vc, interp = case
    s, o, op = _pair(*case, with_pert=True)
    s.predict()
    o.predict()
    op.predict()
    assert worst_rel_floor(s.state(0), o.Uf, op.Uf, FP64_TOL, "predictor fine") < 1
    if nl == 2:
        assert worst_rel_floor(s.state(1), o.Uc, op.Uc, FP64_TOL, "predictor coarse") < 1
    for k in range(3):
        rc, it, res = s.iterate(1, 0.0)
        ores = o.iteration()
        op.iteration()
        assert worst_rel_floor(s.state(0), o.Uf, op.Uf, FP64_TOL, f"iteration {k} fine") < 1
        if nl == 2:
            assert worst_rel_floor(s.state(1), o.Uc, op.Uc, FP64_TOL, f"iteration {k} coarse") < 1
        gres = s.residual()
        np.testing.assert_allclose(gres, ores, rtol=1e-7, atol=1e-13)
    s.close()


@pytest.mark.parametrize("nl", [2, 3])
def test_predictor_on_a_non_spread_state_matches_oracle(nl):
    """pfasst_mg_predict called after iterations (slices no longer hold one spread value):
    the library runs the full staged predictor there, not the serial chain it uses right
    after a spread; both levels against the oracle's stage loop."""
    dim, n, P = 2, 31, 4
    if nl == 2:
        s, o = _pair(dim, n, 5, 3, P, 2, 1, 2, 4)
        o.predict()
        o.iteration()
        o.iteration()
        s.iterate(2, 0.0)
        s.predict()
        o.predict()
        assert rel(s.state(0), o.Uf) < FP64_TOL
        assert rel(s.state(1), o.Uc) < FP64_TOL
    else:
        s = pmg.PFASSTSolver(dim, n, 5, 3, P, 1.0, 0.01, nlevels=3, coarsest_nodes=2, smoother=1, omega=1.0,
                             vcycles=2)
        o = O.MLPFASST(dim, n, [5, 3, 2], P, 1.0, 0.01, O.MGParams(smoother=1, omega=1.0, vcycles=2))
        u0 = _u0(dim, n)
        s.set_initial(u0)
        o.set_initial(u0)
        o.predict()
        o.iteration()
        s.iterate(1, 0.0)
        s.predict()
        o.predict()
        for lv in range(3):
            assert rel(s.state(lv), o.U[lv]) < FP64_TOL, lv
    s.close()


def test_sweep_entry_points_match_oracle():
    dim, n, sf, sc, P = 2, 31, 5, 3, 3
    s, o = _pair(dim, n, sf, sc, P, 2, 0, 2, 4)
    s.sweep(0)
    mg = O.MGParams(vcycles=2)
    for p in range(P):
        o.Uf[p], o.Ff[p], _ = O.sweep(dim, n, sf, 1.0, 0.01, mg, o.Uf[p], o.Ff[p])
    assert rel(s.state(0), o.Uf) < FP64_TOL
    s.close()


def test_isdc_heat1d_workload_full_size():
    """1D heat, 127 points, 3 nodes, single-level SDC, dt = 0.01 to T = 0.1, V(2,1)
    Jacobi: sweep each step to residual 1e-9; same iteration counts and end values."""
    wl = inputs.heat1d_c1()
    s = pmg.PFASSTSolver(wl.dim, wl.n, wl.fine_nodes, 0, 1, wl.nu, wl.dt, nlevels=1, smoother=wl.smoother,
                         omega=wl.omega, vcycles=wl.vcycles)
    o = O.PFASST(wl.dim, wl.n, wl.fine_nodes, 2, 1, wl.nu, wl.dt,
                 O.MGParams(smoother=wl.smoother, omega=wl.omega, vcycles=wl.vcycles), nlevels=1)
    u = wl.u0()
    s.set_initial(u)
    for step in range(wl.steps):
        o.set_initial(u)
        it_o, _ = o.run(wl.iterations, 1e-9)
        rc, it_g, res = s.iterate(wl.iterations, 1e-9)
        assert it_g == it_o and rc == pmg.PMG_OK
        u = o.end_value()
        assert rel(s.solution(0, wl.fine_nodes - 1), u) < FP64_TOL
        s.advance()
    s.close()


def test_heat2d_workload_full_size_fp64():
    """2D heat 255^2 / 127^2, 16 slices, 5/3 nodes, 2 V-cycles: 3 PFASST iterations."""
    wl = inputs.heat2d_c2(vcycles=2, precision=0)
    s = pmg.PFASSTSolver(wl.dim, wl.n, wl.fine_nodes, wl.coarse_nodes, wl.slices, wl.nu, wl.dt,
                         smoother=wl.smoother, omega=wl.omega, vcycles=wl.vcycles)
    u0 = wl.u0()
    s.set_initial(u0)
    orcs = []
    for u in (u0, ulp_perturbed(u0)):
        o = O.PFASST(wl.dim, wl.n, wl.fine_nodes, wl.coarse_nodes, wl.slices, wl.nu, wl.dt,
                     O.MGParams(smoother=wl.smoother, omega=wl.omega, vcycles=wl.vcycles))
        o.set_initial(u)
        o.predict()
        orcs.append(o)
    for k in range(3):
        ores = orcs[0].iteration()
        orcs[1].iteration()
        rc, it, res = s.iterate(1, 0.0)
        assert abs(res - ores.max()) <= 1e-7 * ores.max()
    # the last slices' solution has decayed to ~1e-6 of the first's: the floor matters there
    assert worst_rel_floor(s.state(0), orcs[0].Uf, orcs[1].Uf, FP64_TOL) < 1
    s.close()


@pytest.mark.parametrize("dim,n,P,sm", [(2, 31, 2, 0), (3, 15, 4, 1)])
def test_mixed_precision_reaches_fp64_fixed_point(dim, n, P, sm):
    s, _ = _pair(dim, n, 5, 3, P, 2, sm, 2, 4, precision=1)
    rc, it, res = s.iterate(200, 1e-12)
    assert rc == pmg.PMG_OK and res <= 1e-12
    o = O.PFASST(dim, n, 5, 3, P, 1.0, 0.01, O.MGParams(smoother=sm, omega=omega(sm), vcycles=0, mg_tol=1e-14))
    o.set_initial(_u0(dim, n))
    o.run(200, 1e-13)
    assert rel(s.state(0), o.Uf) < MIXED_TOL
    s.close()


def test_full_solve_pfasst_matches_oracle():
    dim, n, P = 2, 31, 2
    s = pmg.PFASSTSolver(dim, n, 5, 3, P, 1.0, 0.01, vcycles=0, mg_tol=1e-12)
    o = O.PFASST(dim, n, 5, 3, P, 1.0, 0.01, O.MGParams(vcycles=0, mg_tol=1e-12))
    u0 = _u0(dim, n)
    s.set_initial(u0)
    o.set_initial(u0)
    o.predict()
    for _ in range(2):
        o.iteration()
    s.iterate(2, 0.0)
    assert rel(s.state(0), o.Uf) < 1e-11
    s.close()


def _pade(z, s):
    N = s - 1
    c = [math.factorial(2 * N - j) * math.factorial(N) / (math.factorial(2 * N) * math.factorial(j)
                                                           * math.factorial(N - j)) for j in range(N + 1)]
    return sum(c[j] * z ** j for j in range(N + 1)) / sum(c[j] * (-z) ** j for j in range(N + 1))


def test_heat3d_fixed_point_with_32_slices():
    """3D heat (nu = 0.5, dt = 0.002, 16 sine modes |k| <= 8), 32 slices, 5/3 nodes, mixed
    precision, red-black Gauss-Seidel, on a 63^3 / 31^3 grid where the iteration reaches
    1e-10: on every sine mode the end of the block must be the serial collocation value
    R(lambda dt)^32 (R = Pade (4,4), Gauss-Lobatto 5 nodes); the residual the GPU reports
    must match a host recomputation on the last slice."""
    wl = inputs.heat3d_c3(n=63, slices=32)
    s = pmg.PFASSTSolver(wl.dim, wl.n, wl.fine_nodes, wl.coarse_nodes, wl.slices, wl.nu, wl.dt,
                         smoother=wl.smoother, omega=wl.omega, vcycles=wl.vcycles, precision=wl.precision)
    s.set_initial(wl.u0())
    rc, it, res = s.iterate(150, 1e-10)
    assert rc == pmg.PMG_OK, (it, res)
    n, h = wl.n, 1.0 / (wl.n + 1)
    end = s.solution(wl.slices - 1, wl.fine_nodes - 1).reshape(n, n, n)
    want = np.zeros_like(end)
    x = np.arange(1, n + 1) * h
    for k, a in zip(wl.modes, wl.amps):
        lam = wl.nu * sum((2 * math.cos(kk * math.pi * h) - 2) / h ** 2 for kk in k)
        amp = a * _pade(lam * wl.dt, wl.fine_nodes) ** wl.slices
        want += amp * np.einsum("k,j,i->kji", np.sin(k[2] * np.pi * x), np.sin(k[1] * np.pi * x),
                                np.sin(k[0] * np.pi * x))
    assert np.abs(end - want).max() <= 1e-8 * np.abs(want).max()
    U = np.stack([s.solution(wl.slices - 1, m).reshape(n, n, n) for m in range(wl.fine_nodes)])

    def lap(u):
        p = np.pad(u, 1)
        return (p[2:, 1:-1, 1:-1] + p[:-2, 1:-1, 1:-1] + p[1:-1, 2:, 1:-1] + p[1:-1, :-2, 1:-1]
                + p[1:-1, 1:-1, 2:] + p[1:-1, 1:-1, :-2] - 6 * u) / h ** 2

    F = np.stack([wl.nu * lap(u) for u in U])
    Q = O.qmatrix(wl.fine_nodes)
    r = max(np.abs(U[0] + wl.dt * np.tensordot(Q[m], F, axes=1) - U[m]).max() for m in range(wl.fine_nodes))
    gres = s.residual()[-1]
    assert abs(r - gres) <= 1e-3 * gres + 1e-14
    s.close()


@pytest.mark.parametrize("precision,tol", [(0, FP64_TOL), (1, 1e-6)])
def test_heat3d_workload_full_size_first_slices_match_oracle(precision, tol):
    """The full 3D workload (255^3 / 127^3, 32 slices, as timed by bench.py): slice p
    depends only on slices 0..p, so the oracle run on the first two slices reproduces
    them.  Compared after the predictor and one PFASST iteration, all fine nodes.
    FP64 path: rounding only (1e-12).  Mixed path: the FP32 V-cycle corrections carry
    ~1e-7 relative rounding, bounded here by 1e-6 relative l2 on the unconverged state."""
    wl = inputs.heat3d_c3(precision=precision)
    s = pmg.PFASSTSolver(wl.dim, wl.n, wl.fine_nodes, wl.coarse_nodes, wl.slices, wl.nu, wl.dt,
                         smoother=wl.smoother, omega=wl.omega, vcycles=wl.vcycles, precision=precision)
    u0 = wl.u0()
    s.set_initial(u0)
    s.iterate(1, 0.0)
    gpu = np.stack([[s.solution(p, m) for m in range(wl.fine_nodes)] for p in range(2)])
    s.close()
    torch.cuda.empty_cache()
    o = O.PFASST(wl.dim, wl.n, wl.fine_nodes, wl.coarse_nodes, 2, wl.nu, wl.dt,
                 O.MGParams(smoother=wl.smoother, omega=wl.omega, vcycles=wl.vcycles))
    o.set_initial(u0)
    o.predict()
    o.iteration()
    assert rel(gpu, o.Uf) < tol


@pytest.mark.parametrize("precision,graphs,groups,autotune,n", [
    (1, 1, 2, 1, 63), (0, 1, 2, 1, 63), (1, 0, 2, 1, 63), (1, 1, 4, 0, 31), (0, 0, 4, 0, 31)])
def test_slice_group_pipeline_gives_identical_iterates(precision, graphs, groups, autotune, n):
    """The pipelined iteration (coarse chain of group g overlapping the fine sweeps of
    later groups on other streams) runs the same operations on the same data as the
    serial schedule: every iterate is bit-identical."""
    wl = inputs.heat3d_c3(n=n, slices=8)
    states = []
    for G in (1, groups):
        s = pmg.PFASSTSolver(wl.dim, wl.n, wl.fine_nodes, wl.coarse_nodes, wl.slices, wl.nu, wl.dt,
                             smoother=wl.smoother, omega=wl.omega, vcycles=wl.vcycles, precision=precision,
                             use_graphs=graphs, autotune=autotune, slice_groups=G)
        s.set_initial(wl.u0())
        rc, it, res = s.iterate(3, 0.0)
        states.append((s.state(0), s.state(1), s.residual()))
        s.close()
    assert np.array_equal(states[0][0], states[1][0])
    assert np.array_equal(states[0][1], states[1][1])
    assert np.array_equal(states[0][2], states[1][2])


@pytest.mark.parametrize("dim,n,precision", [(3, 31, 0), (3, 63, 1), (2, 63, 0), (1, 127, 0)])
def test_vcycle_tail_matches_per_level_kernels(dim, n, precision):
    """The one-launch V-cycle bottom runs the same operations as the per-level kernels:
    PFASST iterates agree to rounding (FP64: 1e-12 relative)."""
    nu, dt = (0.5, 0.002) if dim == 3 else (1.0, 0.005)
    smoother = 1 if dim == 3 else 0
    omega = 1.0 if smoother == 1 else 2.0 / 3.0
    rng = np.random.default_rng(dim * 100 + n)
    u0 = rng.standard_normal(n ** dim)
    out = []
    for tail in (0, 1):
        s = pmg.PFASSTSolver(dim, n, 5, 3, 4, nu, dt, smoother=smoother, omega=omega, vcycles=2,
                             precision=precision, vcycle_tail=tail, slice_groups=1)
        s.set_initial(u0)
        s.iterate(3, 0.0)
        out.append(s.state(0))
        s.close()
    err = worst_rel(out[1], out[0], "tail vs per-level")
    assert err <= (1e-12 if precision == 0 else 1e-5), err


@pytest.mark.parametrize("n,level,zchunk", [(127, 0, 32), (255, 1, 16), (127, 0, 7)])
def test_tma_staged_sweep_matches_the_fused_sweep(n, level, zchunk):
    """The TMA-staged sweep (planes streamed by cp.async.bulk.tensor into a shared-memory
    ring) computes the same red-black sweep as the register-prefetch fused kernel: PFASST
    iterates agree to FP32 rounding."""
    wl = inputs.heat3d_c3(n=n, slices=2)
    out = []
    for fused, param, threads in ((1, zchunk, 256), (2, zchunk, 512)):
        s = pmg.PFASSTSolver(wl.dim, wl.n, wl.fine_nodes, wl.coarse_nodes, wl.slices, wl.nu, wl.dt,
                             smoother=wl.smoother, omega=wl.omega, vcycles=wl.vcycles, precision=1, autotune=0)
        for narrow in (0, 1):
            pmg.pfasst_mg_set_tuning(s.h, level, narrow, fused, param, threads)
        assert pmg.pfasst_mg_tuning(s.h, level, 0)[:2] == (fused, param)
        s.set_initial(wl.u0())
        s.iterate(2, 0.0)
        out.append(s.state(0))
        s.close()
    err = worst_rel(out[1], out[0], "TMA vs fused")
    assert err <= 1e-6, err


@pytest.mark.parametrize("n,slices,level,zchunk,vcycles", [(127, 2, 0, 32, 2), (255, 2, 1, 16, 2), (127, 3, 0, 7, 1),
                                                           (255, 1, 0, 64, 1)])
def test_tma_quad_sweep_is_bitwise_the_pair_sweep(n, slices, level, zchunk, vcycles):
    """Four x points per thread (128-bit shared loads, one shuffle per half-sweep) against
    two per thread: the same points, arithmetic and summation order, so the PFASST
    iterates (the sweep from zero, the plain sweep and the sweep fused with u += e all
    run) must be identical bit for bit."""
    wl = inputs.heat3d_c3(n=n, slices=slices)
    out = []
    for fused in (2, 3):
        s = pmg.PFASSTSolver(wl.dim, wl.n, wl.fine_nodes, wl.coarse_nodes, wl.slices, wl.nu, wl.dt,
                             smoother=wl.smoother, omega=wl.omega, vcycles=vcycles, precision=1, autotune=0)
        for narrow in (0, 1):
            pmg.pfasst_mg_set_tuning(s.h, level, narrow, fused, zchunk, 0)
        t = pmg.pfasst_mg_tuning(s.h, level, 0)
        assert t[:2] == (fused, zchunk) and t[2] == (512 if fused == 2 else 2 * ((n + 1) >> level)), t
        s.set_initial(wl.u0())
        s.iterate(2, 0.0)
        out.append(s.state(0))
        s.close()
    assert np.array_equal(out[0], out[1]), worst_rel(out[1], out[0], "quad vs pair")


UNIFORM_CASES = [
    # dim, n, sf, sc, P, nlevels, smoother, vcycles, interp  (uniform nodes, Sec. 3)
    (1, 63, 5, 3, 3, 2, 0, 2, 4),
    (2, 31, 3, 2, 4, 2, 0, 1, 4),    # {0, 1/2, 1} over {0, 1}: backward Euler on the coarse level
    (3, 15, 5, 3, 2, 2, 1, 2, 4),
    (2, 31, 5, 0, 3, 1, 0, 2, 4),
]


@pytest.mark.parametrize("case", UNIFORM_CASES, ids=[f"d{c[0]}n{c[1]}s{c[2]}x{c[3]}P{c[4]}" for c in UNIFORM_CASES])
def test_uniform_nodes_match_oracle_every_iteration(case):
    dim, n, sf, sc, P, nl, sm, vc, interp = case
    s = pmg.PFASSTSolver(dim, n, sf, sc if nl == 2 else 0, P, 1.0, 0.01, nlevels=nl, smoother=sm, omega=omega(sm),
                         vcycles=vc, interp_order=interp, family=1)
    u0 = _u0(dim, n)
    s.set_initial(u0)
    o, op = (O.PFASST(dim, n, sf, sc if nl == 2 else 2, P, 1.0, 0.01, O.MGParams(smoother=sm, omega=omega(sm),
                                                                                 vcycles=vc),
                      nlevels=nl, interp_order=interp, family=1) for _ in range(2))
    o.set_initial(u0)
    op.set_initial(ulp_perturbed(u0))
    s.predict()
    o.predict()
    op.predict()
    assert worst_rel_floor(s.state(0), o.Uf, op.Uf, FP64_TOL, "predictor") < 1
    for k in range(3):
        s.iterate(1, 0.0)
        ores = o.iteration()
        op.iteration()
        assert worst_rel_floor(s.state(0), o.Uf, op.Uf, FP64_TOL, f"iteration {k} fine") < 1
        if nl == 2:
            assert worst_rel_floor(s.state(1), o.Uc, op.Uc, FP64_TOL, f"iteration {k} coarse") < 1
        np.testing.assert_allclose(s.residual(), ores, rtol=1e-7, atol=1e-13)
    s.close()


def test_uniform_nodes_3d_fixed_point_is_the_midpoint_right_rule():
    """3D heat with the paper's second-order rule (3 uniform nodes, coarse backward Euler),
    mixed precision: PFASST converges on every sine mode to R(lambda dt)^P with
    R(z) = (1 + z/4) / (1 - 3z/4 + z^2/4), the rule's stability function."""
    wl = inputs.heat3d_c3(n=63, slices=4)
    s = pmg.PFASSTSolver(3, wl.n, 3, 2, wl.slices, wl.nu, wl.dt, smoother=1, omega=1.0, vcycles=2, precision=1,
                         family=1)
    s.set_initial(wl.u0())
    rc, it, res = s.iterate(200, 1e-10)
    assert rc == pmg.PMG_OK, (it, res)
    n, h = wl.n, 1.0 / (wl.n + 1)
    x = np.arange(1, n + 1) * h
    want = np.zeros((n, n, n))
    for k, a in zip(wl.modes, wl.amps):
        z = wl.dt * wl.nu * sum((2 * math.cos(kk * math.pi * h) - 2) / h ** 2 for kk in k)
        want += a * ((1 + z / 4) / (1 - 3 * z / 4 + z * z / 4)) ** wl.slices * np.einsum(
            "k,j,i->kji", np.sin(k[2] * np.pi * x), np.sin(k[1] * np.pi * x), np.sin(k[0] * np.pi * x))
    end = s.solution(wl.slices - 1, 2).reshape(n, n, n)
    assert np.abs(end - want).max() <= 1e-8 * np.abs(want).max()
    s.close()


# ---------------------------------------------------------------- three levels

THREE_CASES = [
    # dim, n, (s0, s1, s2), family, P, smoother, vcycles, interp
    (1, 63, (5, 3, 2), 0, 4, 0, 2, 4),
    (2, 31, (5, 3, 2), 1, 3, 1, 1, 4),     # uniform nodes: level 2 is backward Euler
    (3, 15, (5, 3, 2), 0, 3, 1, 2, 4),     # level 2 on the 3^3 grid: exact sub-step solves
    (3, 31, (9, 5, 3), 1, 2, 1, 2, 2),     # uniform M = 8, 4, 2
    (2, 63, (7, 4, 2), 1, 5, 0, 1, 4),     # uniform M = 6, 3, 1
    (2, 31, (7, 3, 2), 0, 4, 1, 2, 4),     # Gauss-Lobatto: 3 nodes nest in any odd count
]


@pytest.mark.parametrize("case", THREE_CASES,
                         ids=[f"d{c[0]}n{c[1]}s{'-'.join(map(str, c[2]))}f{c[3]}P{c[4]}" for c in THREE_CASES])
def test_three_levels_match_oracle_every_iteration(case):
    """Multi-level PFASST (Sec. 2.4; a level-1 sweep on every slice between the two
    restrictions, the serial chain on level 2): predictor and each iteration against
    the oracle's three-level schedule, on all three levels."""
    dim, n, nodes, fam, P, sm, vc, interp = case
    s = pmg.PFASSTSolver(dim, n, nodes[0], nodes[1], P, 1.0, 0.01, nlevels=3, coarsest_nodes=nodes[2], family=fam,
                         smoother=sm, omega=omega(sm), vcycles=vc, interp_order=interp)
    o, op = (O.MLPFASST(dim, n, list(nodes), P, 1.0, 0.01, O.MGParams(smoother=sm, omega=omega(sm), vcycles=vc),
                        families=[fam] * 3, interp_order=interp) for _ in range(2))
    u0 = _u0(dim, n)
    s.set_initial(u0)
    o.set_initial(u0)
    op.set_initial(ulp_perturbed(u0))
    s.predict()
    o.predict()
    op.predict()
    for l in range(3):
        assert worst_rel_floor(s.state(l), o.U[l], op.U[l], FP64_TOL, f"predictor level {l}") < 1
    for k in range(3):
        s.iterate(1, 0.0)
        ores = o.iteration()
        op.iteration()
        for l in range(3):
            assert worst_rel_floor(s.state(l), o.U[l], op.U[l], FP64_TOL, f"iteration {k} level {l}") < 1
        np.testing.assert_allclose(s.residual(), ores, rtol=1e-7, atol=1e-13)
    s.close()


def test_three_levels_converge_to_the_two_level_fixed_point_mixed():
    """3D heat, mixed precision: both hierarchies converge to the fine collocation
    solution (the fixed point does not depend on the coarse levels)."""
    wl = inputs.heat3d_c3(n=63, slices=4)
    out = []
    for nl in (2, 3):
        s = pmg.PFASSTSolver(3, wl.n, 5, 3, wl.slices, wl.nu, wl.dt, nlevels=nl, coarsest_nodes=2 if nl == 3 else 0,
                             smoother=1, omega=1.0, vcycles=2, precision=1)
        s.set_initial(wl.u0())
        rc, it, res = s.iterate(60, 1e-12)
        assert rc == pmg.PMG_OK, (nl, it, res)
        out.append(s.state(0))
        s.close()
    assert rel(out[1], out[0]) < MIXED_TOL


def test_three_level_standalone_sweeps_match_oracle():
    """pfasst_mg_sweep on each level of three after two iterations: level 1 (every
    slice; F_1 = A U_1 refreshed first, as the oracle keeps it), level 2 (the serial
    chain), level 0."""
    dim, n, P, nodes = 2, 31, 3, (5, 3, 2)
    s = pmg.PFASSTSolver(dim, n, nodes[0], nodes[1], P, 1.0, 0.01, nlevels=3, coarsest_nodes=nodes[2], smoother=1,
                         omega=1.0, vcycles=2)
    o = O.MLPFASST(dim, n, list(nodes), P, 1.0, 0.01, O.MGParams(smoother=1, omega=1.0, vcycles=2))
    u0 = _u0(dim, n)
    s.set_initial(u0)
    o.set_initial(u0)
    s.iterate(2, 0.0)
    o.predict()
    o.iteration()
    o.iteration()
    for level in (1, 2, 0):
        s.sweep(level)
        o.sweep(level)
        for l in range(3):
            assert rel(s.state(l), o.U[l]) < FP64_TOL, (level, l)
    s.close()


def test_three_level_weak_scaling_shape_of_the_paper():
    """Sec. 4.2.2 through the C ABI: 1D, k = nu = L = T = 1, N_x = N_t = N parallel steps,
    three levels (3 uniform nodes on levels 0 and 1, backward Euler on level 2), two
    V(2,2) Gauss-Seidel cycles per solve.  The PDE error of the last step reaches its
    floor at an iteration that stays <= 6 and does not grow with N (the paper: 5, 3, 3),
    and every iteration's error equals the oracle's."""
    reach = []
    for N in (32, 64, 128):
        n, P, dt = N - 1, N, 1.0 / N
        x = np.arange(1, n + 1) / (n + 1)
        pde = math.exp(-math.pi ** 2) * np.sin(np.pi * x)
        s = pmg.PFASSTSolver(1, n, 3, 3, P, 1.0, dt, nlevels=3, coarsest_nodes=2, family=1, smoother=1, omega=1.0,
                             nu1=2, nu2=2, vcycles=2)
        o = O.MLPFASST(1, n, (3, 3, 2), P, 1.0, dt, O.MGParams(smoother=1, omega=1.0, nu1=2, nu2=2, vcycles=2),
                       families=(1, 1, 1))
        s.set_initial(np.sin(np.pi * x))
        o.set_initial(np.sin(np.pi * x))
        o.predict()
        errs = []
        for _ in range(10):
            s.iterate(1, 0.0)
            o.iteration()
            end = s.solution(P - 1, 2)
            assert np.abs(end - o.end_value()).max() <= 1e-12
            errs.append(np.abs(end - pde).max())
        s.close()
        reach.append(next(k + 1 for k, e in enumerate(errs) if e <= 1.6 * errs[-1]))
    assert max(reach) <= 6 and reach[2] <= reach[0], reach


def test_integer_narrowing_matches_the_hardware_conversion():
    """The FP64 -> FP32 rounding done with integer operations (mixed-precision residuals,
    time interpolation) equals the hardware round-to-nearest-even conversion bit for bit
    on 2^28 inputs: uniform bit patterns, the float range down to subnormals and up to
    overflow, exact ties."""
    assert pmg.pfasst_mg_check_narrowing(1 << 28, seed=12345) == 0


# ---------------------------------------------------------------- the TMA kernels on the workload grids

def _colloc_state(wl, n, nodes, slices):
    """The collocation solution of every node of every slice (Eq. collocationM), per sine
    mode: Y = (I - z Q)^-1 1 y0 with z = dt nu lambda(k) and Q the oracle's integration
    matrix; slice p starts from the last node of slice p-1.  Shape (slices, nodes, n^3)."""
    h = 1.0 / (n + 1)
    x = np.arange(1, n + 1) * h
    Q = O.qmatrix(nodes)
    out = np.zeros((slices, nodes, n ** 3))
    for k, a in zip(wl.modes, wl.amps):
        z = wl.dt * wl.nu * sum((2 * math.cos(kk * math.pi * h) - 2) / h ** 2 for kk in k)
        phi = np.einsum("k,j,i->kji", np.sin(k[2] * np.pi * x), np.sin(k[1] * np.pi * x),
                        np.sin(k[0] * np.pi * x)).reshape(-1)
        y0 = a
        for p in range(slices):
            Y = np.linalg.solve(np.eye(nodes) - z * Q, np.full(nodes, y0))
            out[p] += Y[:, None] * phi[None, :]
            y0 = Y[-1]
    return out


@pytest.mark.parametrize("kind", [2, 3])
def test_mixed_fixed_point_127_with_tma_kernels_pinned(kind):
    """Mixed precision on the 3D workload's coarse-grid size 127^3 (9 slices, so that the
    batched fine level takes the z-marching kernels), with the TMA-staged sweep pinned on
    the finest multigrid level: the pre-smoothing sweep from zero, the plain sweep, the
    post-smoothing sweep fused with u += e, and the TMA-staged residual + restriction.
    Converged to a collocation residual of 1e-11, every (slice, node) grid function must
    match the collocation solution computed per sine mode from the oracle's Q to 1e-9."""
    wl = inputs.heat3d_c3(n=127, slices=9)
    s = pmg.PFASSTSolver(3, wl.n, 5, 3, wl.slices, wl.nu, wl.dt, smoother=1, omega=1.0, vcycles=2, precision=1,
                         autotune=0)
    for narrow in (0, 1):
        pmg.pfasst_mg_set_tuning(s.h, 0, narrow, kind, 32, 512)
    assert pmg.pfasst_mg_tuning(s.h, 0, 0)[:2] == (kind, 32)
    s.set_initial(wl.u0())
    rc, it, res = s.iterate(400, 1e-11)
    assert rc == pmg.PMG_OK, (it, res)
    gpu = s.state(0)
    s.close()
    assert rel(gpu, _colloc_state(wl, wl.n, 5, wl.slices)) < MIXED_TOL


@pytest.mark.parametrize("kind", [2, 3])
def test_fp32_sweep_255_with_tma_kernels_matches_oracle(kind):
    """One SDC sweep (4 sub-steps, one FP32 V(2,1) red-black cycle each) on two slices of
    the 255^3 grid of the 3D workload with the TMA-staged sweep pinned on the finest
    level (the batch of two takes the TMA-staged residual + restriction too), against
    the oracle's FP64 sweep: FP32 rounding of the corrections only, <= 2e-6 per node."""
    wl = inputs.heat3d_c3(n=255, slices=2)
    s = pmg.PFASSTSolver(3, wl.n, 5, 0, 2, wl.nu, wl.dt, nlevels=1, smoother=1, omega=1.0, vcycles=1, precision=1,
                         autotune=0)
    for narrow in (0, 1):
        pmg.pfasst_mg_set_tuning(s.h, 0, narrow, kind, 32, 512)
    u0 = wl.u0()
    s.set_initial(u0)
    s.sweep(0)
    gpu = s.state(0)
    s.close()
    torch.cuda.empty_cache()
    # single level, no send-forward: both slices start from the spread u0 and sweep alike
    U = np.repeat(u0[None, :], 5, axis=0)
    F = np.stack([O.apply_A(3, wl.n, wl.nu, u) for u in U])
    want, _, _ = O.sweep(3, wl.n, 5, wl.nu, wl.dt, O.MGParams(smoother=1, omega=1.0, vcycles=1), U, F)
    assert rel(gpu, np.stack([want, want])) < 2e-6


def test_integer_widening_matches_the_hardware_conversion_on_every_float():
    """The FP32 -> FP64 widening done with integer operations (FP32 corrections added to
    FP64 iterates: interpolation, update sweeps) equals the hardware conversion bit for
    bit on all 2^32 float bit patterns (normal, subnormal, zero, Inf; NaN stays NaN)."""
    assert pmg.pfasst_mg_check_widening() == 0


def test_fp64_probe_reports_a_plausible_rate():
    """The FP64 FMA probe (the roofline denominator of the FP64-bound kernels) measures a
    positive rate no higher than the unit-count bound 152 SMs x 2 FMA/clk x 2 flops at
    the maximum SM clock (with 5 % slack for the clock reading), and not far below it."""
    gflops = pmg.pfasst_mg_fp64_peak(3)
    nominal = 152 * 2 * 2 * 2.07
    assert 0.3 * nominal < gflops < 1.05 * nominal, gflops


@pytest.mark.parametrize("nl,cvc,sm,fam", [(2, 0, 1, 0), (2, 4, 0, 1), (3, 3, 1, 1), (3, 0, 0, 0)])
def test_coarse_level_vcycle_count_matches_oracle(nl, cvc, sm, fam):
    """coarse_vcycles (reading g16 made an option): the coarse PFASST levels solve their
    sub-steps with their own V-cycle count (cvc > 0) or to the tolerance (cvc = 0) while
    the fine level keeps 2 V-cycles; predictor and three iterations against the oracle
    with the same per-level multigrid settings, on every level."""
    dim, n, P = 2, 31, 3
    nodes = [5, 3, 2][:nl]
    mg = O.MGParams(smoother=sm, omega=omega(sm), vcycles=2)
    mgc = O.MGParams(smoother=sm, omega=omega(sm), vcycles=cvc, mg_tol=1e-12)
    s = pmg.PFASSTSolver(dim, n, nodes[0], nodes[1], P, 1.0, 0.01, nlevels=nl, coarsest_nodes=nodes[2] if nl == 3 else 0,
                         family=fam, smoother=sm, omega=omega(sm), vcycles=2, coarse_vcycles=cvc, mg_tol=1e-12)
    u0 = _u0(dim, n)
    s.set_initial(u0)
    o, op = (O.MLPFASST(dim, n, nodes, P, 1.0, 0.01, mg, families=[fam] * nl, mg_coarse=mgc) for _ in range(2))
    o.set_initial(u0)
    op.set_initial(ulp_perturbed(u0))
    o.predict()
    op.predict()
    s.predict()
    for l in range(nl):
        assert worst_rel_floor(s.state(l), o.U[l], op.U[l], FP64_TOL, f"predictor level {l}") < 1
    for k in range(3):
        s.iterate(1, 0.0)
        ores = o.iteration()
        op.iteration()
        for l in range(nl):
            assert worst_rel_floor(s.state(l), o.U[l], op.U[l], FP64_TOL, f"iteration {k} level {l}") < 1
        np.testing.assert_allclose(s.residual(), ores, rtol=1e-7, atol=1e-13)
    s.close()


@pytest.mark.parametrize("dim,n,P,nl,precision", [(2, 31, 4, 2, 0), (3, 15, 3, 3, 1), (1, 127, 1, 1, 0)])
def test_device_side_iteration_loop_matches_host_loop(dim, n, P, nl, precision):
    """With graphs on, pfasst_mg_iterate runs the whole loop as one graph launch (a
    conditional while-node; the check of residual and iteration count is a kernel).
    Against the host-driven loop (graphs off): the same iteration count, residual and
    bitwise state, when stopping on the tolerance and when the iteration cap is reached."""
    u0 = _u0(dim, n)
    out = []
    for graphs in (1, 0):
        s = pmg.PFASSTSolver(dim, n, 5, 3 if nl >= 2 else 0, P, 1.0, 0.01, nlevels=nl,
                             coarsest_nodes=2 if nl == 3 else 0, smoother=1, omega=1.0, vcycles=2,
                             precision=precision, use_graphs=graphs)
        s.set_initial(u0)
        rc1, it1, res1 = s.iterate(200, 1e-8)
        st1 = s.state(0)
        s.set_initial(u0)
        rc2, it2, res2 = s.iterate(3, 0.0)
        out.append((rc1, it1, res1, st1, rc2, it2, res2, s.state(0)))
        s.close()
    g, h = out
    assert g[0] == h[0] == pmg.PMG_OK and g[1] == h[1] and g[2] == h[2] and g[2] <= 1e-8
    assert np.array_equal(g[3], h[3])
    assert g[4] == h[4] == pmg.PMG_NOT_CONVERGED and g[5] == h[5] == 3 and g[6] == h[6]
    assert np.array_equal(g[7], h[7])


@pytest.mark.parametrize("dim,n,P,precision,nl", [(3, 63, 4, 1, 2), (3, 31, 3, 0, 2), (2, 127, 4, 0, 2),
                                                  (3, 31, 2, 1, 3), (3, 63, 1, 0, 1)])
def test_persistent_single_grid_vcycles_match_per_level_launches(dim, n, P, precision, nl):
    """The V-cycles of single-grid sub-step solves (the serial coarse chain; every solve of
    a one-slice handle) as one persistent cooperative launch with grid-wide barriers give
    the same iterates, bit for bit, as one launch per sweep, restriction and prolongation
    (point smoothers: autotuning off), FP64 and mixed, two and three levels."""
    rng = np.random.default_rng(dim * 10 + n)
    u0 = rng.standard_normal(n ** dim)
    out = []
    for coop in (1, 0):
        s = pmg.PFASSTSolver(dim, n, 5, 3 if nl >= 2 else 0, P, 0.5, 0.002, nlevels=nl,
                             coarsest_nodes=2 if nl == 3 else 0, smoother=1, omega=1.0, vcycles=2,
                             precision=precision, autotune=0, single_grid_vcycle=coop)
        s.set_initial(u0)
        s.iterate(3, 0.0)
        out.append([s.state(l) for l in range(nl)] + [s.residual()])
        s.close()
    for a, b in zip(out[0], out[1]):
        assert np.array_equal(a, b)


def test_persistent_single_grid_vcycles_in_the_standalone_solve():
    """pfasst_mg_helmholtz_solve on one grid (batch 1) with single_grid_vcycle = 1 takes the
    persistent V-cycles: against the oracle's V-cycles to 1e-12."""
    dim, n, vc = 3, 31, 2
    c = 0.37 / (n + 1) ** 2 * 4
    rng = np.random.default_rng(5)
    b = rng.standard_normal((1, n ** dim))
    u = rng.standard_normal((1, n ** dim))
    opt = pmg.pfasst_mg_default_options(smoother=1, omega=1.0, vcycles=vc)
    assert opt.single_grid_vcycle == 0
    opt.single_grid_vcycle = 1
    ut = torch.tensor(u, device="cuda")
    pmg.pfasst_mg_helmholtz_solve(pmg.pmg_grid(dim, n), c, 1, torch.tensor(b, device="cuda"), ut, opt)
    want = O.mg_solve(O.MGParams(smoother=1, omega=1.0, vcycles=vc), dim, n, c, b[0], u[0])[0]
    assert rel(ut.cpu().numpy(), want[None]) < FP64_TOL
