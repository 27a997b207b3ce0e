"""GPU parity of the uneven batch (independent single-level SDC problems of different
sizes, run as branches of one CUDA graph per time step) against the FP64 oracle run
problem by problem, and equivalence of graph and eager execution and of the
autotuned and default smoother choices."""
import numpy as np
import pytest

import oracle as O
from parity import worst_rel
import paper_1407_6486_gb300 as pmg
from paper_1407_6486_gb300 import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


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


def small_batch():
    # the generator of the uneven workload at small sizes (1D added by hand)
    probs = inputs.heat_uneven_c4(seed=64, n2d=(15, 31, 63), n3d=(7, 15, 31), count2d=4, count3d=4)
    probs.append(inputs.Problem(1, 127, 5, 0.7, 0.004, [(1, 1, 1), (5, 1, 1)], [1.0, -0.3]))
    return probs


def oracle_run(p, steps, sweeps, smoother):
    mg = O.MGParams(smoother=smoother, omega=1.0 if smoother else 2.0 / 3.0, vcycles=2)
    o = O.PFASST(p.dim, p.n, p.nodes, 2, 1, p.nu, p.dt, mg, nlevels=1)
    u = p.u0()
    res = None
    for _ in range(steps):
        o.set_initial(u)
        o.predict()
        for _ in range(sweeps):
            res = o.iteration()
        u = o.end_value()
    return u, res[0]


@pytest.mark.parametrize("smoother,autotune,graphs", [(1, 1, 1), (1, 0, 1), (0, 1, 1), (1, 1, 0)])
def test_batch_matches_oracle_per_problem(smoother, autotune, graphs):
    probs = small_batch()
    steps, sweeps = 2, 3
    b = pmg.BatchSolver([(p.dim, p.n, p.nodes, p.nu, p.dt) for p in probs], smoother=smoother,
                        omega=1.0 if smoother else 2.0 / 3.0, vcycles=2, precision=0, autotune=autotune,
                        use_graphs=graphs)
    for i, p in enumerate(probs):
        b.set_initial(i, p.u0())
    res = b.run(steps, sweeps)
    for i, p in enumerate(probs):
        want, wres = oracle_run(p, steps, sweeps, smoother)
        assert rel(b.solution(i), want) < 1e-12, (i, p.dim, p.n)
        assert abs(res[i] - wres) <= 1e-7 * wres + 1e-14
    assert b.launches() > 0
    b.close()


def test_batch_mixed_precision_and_repeated_runs():
    probs = small_batch()
    b = pmg.BatchSolver([(p.dim, p.n, p.nodes, p.nu, p.dt) for p in probs], smoother=1, omega=1.0, vcycles=2,
                        precision=1)
    for i, p in enumerate(probs):
        b.set_initial(i, p.u0())
    b.run(1, 3)
    b.run(1, 3)  # the captured graph is replayed; state carries over
    for i, p in enumerate(probs):
        want, _ = oracle_run(p, 2, 3, 1)
        assert rel(b.solution(i), want) < 1e-6, (i, p.dim, p.n)
    b.close()


@pytest.mark.parametrize("precision,tol", [(0, 1e-12), (1, 1e-6)])
def test_batch_with_the_workload_extremes_matches_oracle(precision, tol):
    """An uneven batch holding the largest members the uneven workload draws -- a 511^2
    and a 127^3 grid -- next to small ones, autotuned (the 127^3 member may take the
    fused or TMA-staged z-marching sweep), red-black V(2,1), FP64 or mixed: every member
    against the oracle run on its own, one time step of two sweeps."""
    probs = [inputs.Problem(2, 511, 5, 0.8, 0.004, [(1, 2, 1), (7, 3, 1)], [1.0, 0.4]),
             inputs.Problem(3, 127, 3, 1.3, 0.006, [(1, 1, 1), (2, 5, 3)], [0.9, -0.5]),
             inputs.Problem(2, 63, 3, 0.3, 0.002, [(2, 2, 1)], [1.1]),
             inputs.Problem(3, 31, 5, 1.9, 0.009, [(1, 2, 2), (3, 1, 1)], [0.7, 0.2])]
    b = pmg.BatchSolver([(p.dim, p.n, p.nodes, p.nu, p.dt) for p in probs], smoother=1, omega=1.0, vcycles=2,
                        precision=precision, autotune=1)
    for i, p in enumerate(probs):
        b.set_initial(i, p.u0())
    res = b.run(1, 2)
    for i, p in enumerate(probs):
        want, wres = oracle_run(p, 1, 2, 1)
        assert rel(b.solution(i), want) < tol, (i, p.dim, p.n)
        if precision == 0:
            assert abs(res[i] - wres) <= 1e-7 * wres + 1e-14
    b.close()
