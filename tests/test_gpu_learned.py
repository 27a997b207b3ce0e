"""GPU tests of the learned multigrid correction network through the C ABI: forward
pass and parameter gradients against the FP64 oracle (oracle/learned.py) on the same
BF16-rounded weights, the synthetic training pairs, training, and the network inside
the V-cycles of a PFASST handle -- its measured gain, the fallback to plain smoothing,
and the converged answer, which the FP64 collocation residual decides whatever the
network does."""
import math

import numpy as np
import pytest

import oracle as O
import paper_1407_6486_gb300 as pmg
from oracle import learned as N
from paper_1407_6486_gb300 import inputs

pytestmark = pytest.mark.gpu

SLICES = {"W1": (0, 432, (16, 27, 1)), "b1": (432, 448, (16,)), "W2": (448, 7360, (16, 27, 16)),
          "b2": (7360, 7376, (16,)), "W3": (7376, 7808, (1, 27, 16)), "b3": (7808, 7809, (1,))}


def to_dict(flat):
    return {k: np.asarray(flat[a:b], dtype=np.float64).reshape(shape) for k, (a, b, shape) in SLICES.items()}


def to_flat(d):
    out = np.zeros(pmg.NET_PARAMS, dtype=np.float32)
    for k, (a, b, _) in SLICES.items():
        out[a:b] = np.asarray(d[k], dtype=np.float64).reshape(-1)
    return out


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


def oracle_params(seed):
    """Oracle-drawn weights with nonzero biases; returns (flat float32 for the GPU,
    FP64 dict of the same values with W2 rounded to BF16 as the tensor cores use it)."""
    d = N.init_params(seed)
    rng = np.random.default_rng(seed + 100)
    for k in ("b1", "b2", "b3"):
        d[k] = 0.1 * rng.standard_normal(d[k].shape)
    flat = to_flat(d)
    ref = to_dict(flat)  # the float32 values the GPU holds, in FP64
    ref["W2"] = N.bf16_round(ref["W2"])
    return flat, ref


@pytest.mark.parametrize("n,batch", [(20, 2), (7, 3)])
def test_forward_matches_the_oracle(n, batch):
    flat, ref = oracle_params(11)
    rng = np.random.default_rng(12)
    x = rng.standard_normal((batch, n, n, n)).astype(np.float32)
    tr = pmg.NetTrainer(batch, n)
    tr.set_params(flat)
    y = tr.forward(x).reshape(batch, n, n, n)
    for b in range(batch):
        want, _ = N.forward(ref, x[b].astype(np.float64))
        assert rel_l2(y[b], want) <= 2e-2, b
    tr.close()


@pytest.mark.parametrize("kappas", [(0.12, 1.0 / 6.0), (0.0, 0.0)])
def test_gradients_match_the_oracle(kappas):
    n, batch = 20, 2
    flat, ref = oracle_params(21)
    rng = np.random.default_rng(22)
    x = rng.standard_normal((batch, n, n, n)).astype(np.float32)
    t = rng.standard_normal((batch, n, n, n)).astype(np.float32)
    tr = pmg.NetTrainer(batch, n)
    tr.set_params(flat)
    loss, g = tr.gradients(x, t, np.array(kappas, dtype=np.float32))
    kap = [float(np.float32(k)) for k in kappas]
    L, gref = N.loss_and_grads(ref, [x[b].astype(np.float64) for b in range(batch)],
                               [t[b].astype(np.float64) for b in range(batch)], kap)
    assert abs(loss - L) <= 2e-2 * L
    gd = to_dict(g)
    for k in gref:
        assert rel_l2(gd[k], gref[k]) <= 2e-2, (k, rel_l2(gd[k], gref[k]))
    tr.close()


def test_training_pairs_are_smoothed_errors_and_their_scaled_residuals():
    n, batch = 16, 4
    tr = pmg.NetTrainer(batch, n)
    x, t, kap = tr.sample(77, 0.1, 1.0 / 6.0)
    x2, t2, kap2 = tr.sample(77, 0.1, 1.0 / 6.0)
    assert np.array_equal(x, x2) and np.array_equal(t, t2) and np.array_equal(kap, kap2)
    x3, _, _ = tr.sample(78, 0.1, 1.0 / 6.0)
    assert not np.array_equal(x, x3)
    assert np.all(kap >= 0.1) and np.all(kap <= 1.0 / 6.0 + 1e-7) and len(set(kap.tolist())) == batch
    x, t = x.reshape(batch, n, n, n), t.reshape(batch, n, n, n)
    idx = np.indices((n, n, n)).sum(axis=0)
    for b in range(batch):
        r = N.apply_ahat(t[b].astype(np.float64), float(kap[b]))
        assert np.abs(x[b] - r).max() <= 1e-5
        # the last colour of the Gauss-Seidel sweep (0-based even index sum) leaves no residual
        assert np.abs(r[idx % 2 == 0]).max() <= 1e-5
        assert np.abs(r[idx % 2 == 1]).max() > 0.1
        assert np.abs(t[b]).max() <= 1.0 + 1e-6
    tr.close()


def oracle_pairs(count, n, seed, vmax=3, klo=0.08, khi=1.0 / 6.0):
    """Error / residual pairs from the oracle multigrid: uniform noise after k in 0..vmax
    V(2,1) red-black cycles of (I - c Lap) u = 0 (the error the iteration leaves),
    scaled to max 1, then one red-black sweep (the error after a first pre-smoothing
    sweep) t, and x = Ahat t.  Returns float32 arrays x, t [count][n^3] and kappa."""
    rng = np.random.default_rng(seed)
    ih2 = (n + 1.0) ** 2
    xs, ts, ks = [], [], []
    zero = np.zeros(n ** 3)
    for _ in range(count):
        kap = rng.uniform(klo, min(khi, 1.0 / 6.0 - 1e-6))
        c = kap / ((1.0 - 6.0 * kap) * ih2)
        u = rng.uniform(-1.0, 1.0, n ** 3)
        k = int(rng.integers(0, vmax + 1))
        if k:
            u, _ = O.mg_solve(O.MGParams(smoother=1, omega=1.0, vcycles=k), 3, n, c, zero, u)
        u = u / np.abs(u).max()
        t = O.smooth(O.MGParams(smoother=1, omega=1.0), 3, n, c, zero, u).reshape(n, n, n)
        xs.append(N.apply_ahat(t, kap).reshape(-1))
        ts.append(t.reshape(-1))
        ks.append(kap)
    return np.array(xs, np.float32), np.array(ts, np.float32), np.array(ks, np.float32)


def gs_loss(x, t, kap, n):
    """Loss (power 1) of one red-black Gauss-Seidel sweep used as the correction: the
    error left is the sweep applied to t (oracle smoother, f = 0)."""
    ih2 = (n + 1.0) ** 2
    tot = 0.0
    for xb, tb, kb in zip(x, t, kap):
        kb = float(kb)
        c = kb / ((1.0 - 6.0 * kb) * ih2)
        left = O.smooth(O.MGParams(smoother=1, omega=1.0), 3, n, c, np.zeros(n ** 3), tb.astype(np.float64))
        w = N.apply_ahat(left.reshape(n, n, n), kb)
        tot += 0.5 * float((w * w).mean())
    return tot / len(x)


NB, NG = 16, 31


@pytest.fixture(scope="module")
def trained():
    """The network trained on the GPU (forward/backward/Adam kernels of the library) on
    64 oracle-multigrid pairs, 16 grids of 31^3 per step."""
    x, t, k = oracle_pairs(64, NG, seed=2024)
    tr = pmg.NetTrainer(NB, NG)
    hist = []
    for step in range(600):
        b = (step % 4) * NB
        hist.append(tr.step(x[b:b + NB], t[b:b + NB], k[b:b + NB], power=1, lr=2e-3, train_bias=0))
    p = tr.params()
    tr.close()
    return p, np.array(hist)


def test_training_reduces_the_loss(trained):
    p, hist = trained
    assert np.all(np.isfinite(hist))
    assert hist[-20:].mean() < 0.5 * hist[:4].mean(), (hist[:4], hist[-20:])
    # biases stay at zero when they are not trained
    d = to_dict(p)
    assert not d["b1"].any() and not d["b2"].any() and not d["b3"].any()


def test_library_sampler_training_reduces_the_loss():
    tr = pmg.NetTrainer(8, 32)
    hist = tr.train(300, 2e-3, 1234, 0.08, 1.0 / 6.0, vcycles_max=0, power=2)
    assert np.all(np.isfinite(hist)) and hist[-20:].mean() < 0.5 * hist[:5].mean()
    tr.close()


def test_multigrid_shaped_samples():
    n, batch = 15, 4
    tr = pmg.NetTrainer(batch, n)
    x, t, kap = tr.sample(5, 0.1, 1.0 / 6.0, vcycles_max=3)
    x, t = x.reshape(batch, n, n, n), t.reshape(batch, n, n, n)
    idx = np.indices((n, n, n)).sum(axis=0)
    for b in range(batch):
        r = N.apply_ahat(t[b].astype(np.float64), float(kap[b]))
        assert np.abs(x[b] - r).max() <= 1e-5 and np.abs(r[idx % 2 == 0]).max() <= 1e-5
        assert 0.05 < np.abs(t[b]).max() <= 1.0 + 1e-6
    tr.close()


def test_trained_network_gains_over_a_smoothing_sweep(trained):
    """What the network gains: on held-out oracle-multigrid pairs its correction leaves
    a scaled residual far below that of the Gauss-Seidel sweep it replaces; inside the
    V-cycles of a 3D heat PFASST handle, the calibration keeps it only where the
    measured contraction drops, so the deployed V-cycle is never worse than the plain."""
    p, _ = trained
    x, t, k = oracle_pairs(NB, NG, seed=99)
    tr = pmg.NetTrainer(NB, NG)
    tr.set_params(p)
    loss_net, _ = tr.gradients(x, t, k, power=1)
    tr.close()
    loss_gs = gs_loss(x, t, k, NG)
    print(f"held-out loss: network {loss_net:.3e}, one red-black sweep {loss_gs:.3e}")
    assert loss_net < 0.5 * loss_gs
    # deployed as in the learned workload (one V-cycle per sub-step, mixed precision): the
    # measured gain is the PFASST residual after 6 iterations without / with the network
    wl = inputs.heat3d_c3(n=63, slices=4)
    wl.vcycles = 1
    res = {}
    for name in ("plain", "net"):
        s = _solver(wl, pmg.PMG_PREC_MIXED)
        if name == "net":
            rho_plain, rho_net, mask = s.set_smoother_net(p, min_n=7, calibrate=1)
        s.set_initial(wl.u0())
        res[name] = s.iterate(6, 0.0)[2]
        s.close()
    print(f"V-cycle contraction: plain {rho_plain:.4f}, with the network {rho_net:.4f} (levels {mask:#x}); "
          f"PFASST residual after 6 iterations: plain {res['plain']:.3e}, with the network {res['net']:.3e} "
          f"(gain {res['plain'] / res['net']:.3f})")
    assert 0 < rho_plain < 1 and np.isfinite(res["net"]) and res["net"] > 0
    if mask == 0:  # nothing kept: the handle runs exactly as without a network
        assert res["net"] == res["plain"]


def test_calibration_on_the_pfasst_residual(trained):
    """calibrate = 2 judges each level by the handle's own PFASST iteration (residual after
    three iterations from the spread initial value).  Checked against separate runs: the
    residuals it reports are those of a plain handle and of the deployed handle iterated
    again from the initial value, and the deployed handle never ends above the plain one."""
    p, _ = trained
    wl = inputs.heat3d_c3(n=63, slices=4)
    wl.vcycles = 1
    plain = _solver(wl, pmg.PMG_PREC_FP64)
    plain.set_initial(wl.u0())
    r_plain = plain.iterate(3, 0.0)[2]
    plain.close()
    s = _solver(wl, pmg.PMG_PREC_FP64)
    s.set_initial(wl.u0())
    rp, rn, mask = s.set_smoother_net(p, min_n=7, calibrate=2)
    r_dep = s.iterate(3, 0.0)[2]
    print(f"PFASST residual after 3 iterations: plain {rp:.4e}, calibrated network {rn:.4e} (levels {mask:#x})")
    assert rp == r_plain and rn == r_dep and rn <= rp
    s.close()


def _pade(z, s):
    M = s - 1
    c = [math.factorial(2 * M - j) * math.factorial(M) / (math.factorial(2 * M) * math.factorial(j)
                                                           * math.factorial(M - j)) for j in range(M + 1)]
    return sum(c[j] * z ** j for j in range(M + 1)) / sum(c[j] * (-z) ** j for j in range(M + 1))


def _closed_form_end(wl):
    n, h = wl.n, 1.0 / (wl.n + 1)
    x = np.arange(1, n + 1) * h
    want = np.zeros((n, n, n))
    for k, a in zip(wl.modes, wl.amps):
        lam = wl.nu * sum((2 * math.cos(kk * math.pi * h) - 2) / h ** 2 for kk in k)
        amp = a * _pade(lam * wl.dt, wl.fine_nodes) ** wl.slices
        want += amp * np.einsum("k,j,i->kji", np.sin(k[2] * np.pi * x), np.sin(k[1] * np.pi * x),
                                np.sin(k[0] * np.pi * x))
    return want


def _solver(wl, precision, autotune=0):
    return pmg.PFASSTSolver(wl.dim, wl.n, wl.fine_nodes, wl.coarse_nodes, wl.slices, wl.nu, wl.dt,
                            smoother=wl.smoother, omega=wl.omega, vcycles=wl.vcycles, precision=precision,
                            autotune=autotune)


@pytest.mark.parametrize("precision", [pmg.PMG_PREC_MIXED, pmg.PMG_PREC_FP64])
def test_network_in_the_vcycles_reaches_the_collocation_fixed_point(trained, precision):
    """With the network forced onto every eligible level the PFASST iteration still
    converges to the serial collocation solution: R(lambda dt)^P on every sine mode."""
    p, _ = trained
    wl = inputs.heat3d_c3(n=63, slices=4)
    s = _solver(wl, precision)
    _, _, mask = s.set_smoother_net(p, min_n=7, calibrate=0)
    assert mask == 0b1111  # levels 63, 31, 15, 7
    s.set_initial(wl.u0())
    rc, it, res = s.iterate(100, 1e-10)
    assert rc == pmg.PMG_OK, (it, res)
    end = s.solution(wl.slices - 1, wl.fine_nodes - 1).reshape(wl.n, wl.n, wl.n)
    want = _closed_form_end(wl)
    assert np.abs(end - want).max() <= 1e-8 * np.abs(want).max()
    s.close()


def test_a_harmful_network_falls_back_to_plain_smoothing(trained):
    """Weights scaled far out of range make the correction harmful: the calibration keeps
    no level, and the iterates are bit-identical to a handle without a network."""
    p, _ = trained
    bad = p.copy()
    bad[7376:7808] *= 1e3
    wl = inputs.heat3d_c3(n=63, slices=4)
    a, b = _solver(wl, pmg.PMG_PREC_MIXED), _solver(wl, pmg.PMG_PREC_MIXED)
    rho_plain, rho_net, mask = a.set_smoother_net(bad, min_n=7, calibrate=1)
    assert mask == 0 and rho_net == rho_plain
    for s in (a, b):
        s.set_initial(wl.u0())
        s.iterate(3, 0.0)
    assert np.array_equal(a.state(0), b.state(0))
    a.close()
    b.close()


def test_removing_the_network_restores_plain_smoothing(trained):
    p, _ = trained
    wl = inputs.heat3d_c3(n=31, slices=2)
    a, b = _solver(wl, pmg.PMG_PREC_FP64), _solver(wl, pmg.PMG_PREC_FP64)
    a.set_smoother_net(p, min_n=7, calibrate=0)
    assert a.set_smoother_net(None) == (0.0, 0.0, 0)
    for s in (a, b):
        s.set_initial(wl.u0())
        s.iterate(2, 0.0)
    assert np.array_equal(a.state(0), b.state(0))
    a.close()
    b.close()


def test_network_requires_red_black_3d():
    wl = inputs.heat3d_c3(n=31, slices=2)
    s = pmg.PFASSTSolver(3, 31, 5, 3, 2, wl.nu, wl.dt, smoother=pmg.PMG_SMOOTHER_JACOBI, autotune=0)
    with pytest.raises(pmg.PMGError) as e:
        s.set_smoother_net(pmg.pfasst_mg_net_init(1))
    assert e.value.code == pmg.PMG_ERR_UNSUPPORTED
    s.close()


def test_substep_pairs_match_the_oracle():
    """pfasst_mg_net_substep_pairs: the initial error u* - u0 of the sub-step solve
    (I - c Lap_h) u = u0 (u* from the oracle's multigrid solved to 1e-14), scaled to max 1,
    after one red-black Gauss-Seidel sweep of the homogeneous problem (oracle smoother) is
    the target t, and x = Ahat t; against the library's pairs in FP32."""
    n, batch = 15, 2
    rng = np.random.default_rng(17)
    u0 = np.stack([inputs.gaussian_random_field(n, 0.1, 40 + b) for b in range(batch)])
    kap = np.array([0.12, 0.16], dtype=np.float32)
    tr = pmg.NetTrainer(batch, n)
    x = np.zeros(batch * n ** 3, dtype=np.float32)
    t = np.zeros_like(x)
    tr.substep_pairs(np.ascontiguousarray(u0), kap, x, t)
    tr.close()
    x, t = x.reshape(batch, -1), t.reshape(batch, -1)
    full = O.MGParams(smoother=1, omega=1.0, vcycles=0, mg_tol=1e-14, mg_maxcycles=80)
    for b in range(batch):
        k = float(kap[b])
        c = k / ((1 - 6 * k) * (n + 1) ** 2)
        us, _ = O.mg_solve(full, 3, n, c, u0[b], u0[b])
        e0 = (us - u0[b]) / np.abs(us - u0[b]).max()
        want_t = O.smooth(O.MGParams(smoother=1, omega=1.0), 3, n, c, np.zeros(n ** 3), e0)
        want_x = N.apply_ahat(want_t.reshape(n, n, n), k).reshape(-1)
        assert np.abs(t[b] - want_t).max() <= 2e-6 * np.abs(want_t).max(), b
        assert np.abs(x[b] - want_x).max() <= 2e-5 * np.abs(want_x).max(), b
