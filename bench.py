#!/usr/bin/env python
"""Benchmark: DOF-sweeps/s of batched SDC + multigrid (two-level PFASST) at a fixed
collocation residual, with the HBM-roofline fraction of the dominant kernel.

Workload (default): 3D heat nu = 0.5 on [0,1]^3, 255^3 fine / 127^3 coarse grid, two-level
PFASST with 5/3 Gauss-Lobatto nodes, 32 time slices batched on one GPU, dt = 0.002,
u0 = 16 seeded sine modes with |k| <= 8, V(2,1) red-black Gauss-Seidel, 2 V-cycles per
sub-step, FP32 V-cycles with FP64 SDC/FAS/residuals, 10 PFASST iterations.

One step = one PFASST block solve through the C ABI: spread u0, predictor, iterations
until the residual target.  The residual target and K_ref (the fine sweeps it takes)
come from the plain FP64 GPU path run for the workload's 10 iterations (untimed).
value = n^3 * M_fine * slices * K_ref / (time per step).

--impl reference times the FP64 CPU oracle on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

# algorithmic bytes per grid point of one launch, by kernel and data precision
# (the reads and writes a kernel cannot avoid)
def algo_bytes_per_point(kernel: str, tsize: int, sf: int = 5, sc: int = 3) -> float:
    t = tsize
    return {
        "residual0": 8 + 8 + 8 + t,            # read u_m, q_m, u_{m+1} (FP64), write f
        "smooth_jacobi": 3 * t,                # read e, f, write e'
        "smooth_rbgs": t + t / 2 + t / 2,      # read all e, f of one colour, write one colour
        "residual_restrict": 2 * t + t / 8,    # read e, f, write coarse f (3D)
        "prolong_add": 2 * t + t / 8,          # read/write e, read coarse e
        "update_u": 8 + 8 + t,                 # read/write u (FP64), read e
        "apply_A": 16.0,                       # read u, write F
        "sf_rhs": 8 * sf + 8 * (sf - 1),       # read F at all nodes, write q per sub-step
        "interp_correction": 16 * sf + 2 * 8 * sc / 8.0,
        "colloc_residual": 16 * sf,
        "copy": 16.0, "pack": 16.0, "unpack": 16.0, "zero": t,
        "rbgs_sweep3d": 3 * t,                 # read e_in, f, write e_out (one fused red+black sweep)
        "rbgs_sweep3d_zero": 2 * t,            # from e = 0: read f, write e
        "rbgs_sweep3d_upd": 2 * t + 16,        # read e_in, f, read/write u (FP64): u += e
        "resrestrict3d": 2 * t + t / 8,
        "prolong3d": 2 * t + t / 8,
        "resid_pt": 16 + t,                    # read u_m, q_m (FP64), write f
        "fine_rhs_residual": 8 * sf + 8 * (sf - 1),  # read U at all nodes, write q per sub-step
        "interp_space": 16 + t / 8.0,          # per fine node-point: read/write U, read the coarse correction
    }.get(kernel, 0.0)


# FP64-pipe-bound kernels: algorithmic FP64 flops per grid point (FMA = 2), 3D
def algo_fp64_flops_per_point(kernel: str, sf: int = 5, sc: int = 3) -> float:
    stencil = 7  # 6 neighbour/centre terms: 5 adds + 1 FMA
    return {
        # G_j = Lap U_j at nodes 1..M (node 0's is the previous slice's node M after the
        # send-forward), P_m = sum_j w_mj G_j, residual and next rhs per sub-step
        "fine_rhs_residual": stencil * (sf - 1) + 2 * sf * (sf - 1) + 4 * (sf - 1),
        # at each coarse point (1/8 of the fine points): fine G at every fine node, coarse F, tau
        "fas_restrict": (stencil * sf + 8 * sc + 2 * sc * sf + 2 * sc * sc + sc) / 8.0,
        "apply_A": 8.0,
    }.get(kernel, 0.0)


# nominal FP64 peak from unit counts and clock: 152 SMs x 2.07 GHz x 2 DFMA/clk x 2 flops
# (context only: the roofline uses the library's measured FP64 FMA probe)
FP64_NOMINAL_GFLOPS = 152 * 2.07 * 2 * 2


def dist_env():
    return int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")), int(os.environ.get("LOCAL_RANK", "0"))


def job_time_and_value(ms_local, units_per_rank, world, device="cuda"):
    """Replicas (one independent problem per GPU): the job's step time is the slowest
    rank's (MAX over ranks), and the whole-job throughput counts every rank's units.
    Returns (ms, units per second)."""
    import torch
    t = torch.tensor([float(ms_local)], dtype=torch.float64, device=device)
    if world > 1:
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    ms = float(t.item())
    return ms, world * units_per_rank / (ms / 1000.0)


def sample_clocks_start():
    try:
        p = subprocess.Popen(["nvidia-smi", "--query-gpu=index,clocks.sm,clocks.max.sm,power.draw,"
                              "clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
                              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
                              "clocks_event_reasons.sw_power_cap", "--format=csv,noheader,nounits", "-lms", "200"],
                             stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        return p, None
    except Exception:
        return None, None


def sample_clocks_stop(p, f, gpu_index):
    if p is None:
        return None
    p.terminate()
    try:
        out, _ = p.communicate(timeout=5)
    except Exception:
        p.kill()
        out = ""
    rows = []
    for line in out.splitlines():
        parts = [x.strip() for x in line.split(",")]
        if len(parts) < 9:
            continue
        try:
            if int(parts[0]) != gpu_index:
                continue
            rows.append(parts)
        except ValueError:
            continue
    if not rows:
        return None
    sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
    mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    reasons = sorted({names[i] for r in rows for i in range(4) if "Active" in r[5 + i] and "Not" not in r[5 + i]})
    return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
            "reasons": reasons, "samples": len(rows)}


def measured_peak_gbs():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def kernel_src_hash(files=None):
    """sha256 prefix of the given files of paper_1407_6486_gb300/csrc (all of them by default)."""
    csrc = os.path.join(ROOT, "paper_1407_6486_gb300", "csrc")
    h = hashlib.sha256()
    for f in sorted(files if files else os.listdir(csrc)):
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def traffic_for(kernel: str, n: int):
    """DRAM bytes per grid point from a committed ncu summary, if taken on the current
    sources of that kernel (the entry lists the source files its hash covers)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
    except Exception:
        return None
    e = d.get(f"{kernel}@{n}")
    if not e or e.get("src_hash") != kernel_src_hash(e.get("src_files")):
        return None
    return float(e["bytes_per_point"])


def make_workload(name):
    from paper_1407_6486_gb300 import inputs
    if name == "heat3d":
        return inputs.heat3d_c3()
    if name == "heat3d-small":
        return inputs.heat3d_c3(n=63, slices=8)
    if name == "heat3d-mid":  # small enough for ncu replays, large enough for the tiled kernels
        return inputs.heat3d_c3(n=127, slices=12)
    if name == "heat3d-255x4":  # the fine grid of the 3D workload on 4 slices: ncu case of the 256-wide rows
        return inputs.heat3d_c3(n=255, slices=4)
    if name == "heat2d":
        return inputs.heat2d_c2(vcycles=2, precision=1)
    raise SystemExit(f"unknown workload {name}")


def cpu_model():
    """Host CPU model name (lscpu, else /proc/cpuinfo, else the machine type)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        with open("/proc/cpuinfo") as fh:
            for line in fh:
                if line.startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform
    return platform.machine()


class OracleSample:
    """The FP64 oracle on `slices` of the workload's slices: predictor once, then each
    sample() times one PFASST iteration (fine sweeps, FAS restriction, coarse chain,
    interpolation, residual) and returns (DOF-sweeps/s, seconds, cores)."""

    def __init__(self, wl, slices: int):
        import oracle as O
        self.wl, self.slices = wl, slices
        self.o = O.PFASST(wl.dim, wl.n, wl.fine_nodes, wl.coarse_nodes, slices, wl.nu, wl.dt,
                          O.MGParams(smoother=wl.smoother, omega=wl.omega, vcycles=wl.vcycles), nlevels=wl.nlevels)
        self.o.set_initial(wl.u0())
        self.o.predict()

    def sample(self, threads: int = 0):
        """threads > 0: run the oracle's loops on that many threads; 0: all host cores."""
        import oracle as O
        cores = O.set_threads(threads if threads > 0 else (os.cpu_count() or 1))
        t0 = time.perf_counter()
        self.o.iteration()
        t = time.perf_counter() - t0
        dofs = self.wl.dofs * (self.wl.fine_nodes - 1) * self.slices
        return dofs / t, t, cores


def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return
    wl = make_workload(args.workload)
    sl = args.ref_slices
    orc = OracleSample(wl, sl)
    for _ in range(args.warmup):
        orc.sample()
    vals, secs = [], []
    for _ in range(args.steps):
        v, t, cores = orc.sample(args.ref_threads)
        vals.append(v)
        secs.append(t)
    value = len(vals) / sum(1.0 / v for v in vals)
    sample = (f"one PFASST iteration (fine sweeps, FAS restriction, coarse chain, interpolation, residual) "
              f"on {sl} of the {wl.slices} slices of {wl.name}, FP64 oracle")
    line = {"impl": "reference", "metric": "DOF-sweeps/s", "value": value, "unit": "DOF-sweeps/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * sum(secs) / len(secs),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": wl.name},
            "cpu_baseline": {"value": value, "unit": "DOF-sweeps/s", "cores": cores, "kind": "oracle", "sample": sample,
                             "nproc": os.cpu_count(), "cpu_model": cpu_model()},
            "e2e": {"value": value, "unit": "DOF-sweeps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_uneven(args):
    """64 independent problems of uneven sizes (2D 63^2..511^2, 3D 31^3..127^3) advanced
    together: 10 time steps of a fixed number of SDC sweeps each, every time step one
    replay of a CUDA graph with one branch per problem.  One bench step = the whole job."""
    import torch
    import paper_1407_6486_gb300 as pmg
    from paper_1407_6486_gb300 import _build, inputs

    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    _build.build()
    pmg.load()
    probs = inputs.heat_uneven_c4()
    steps, sweeps = 10, args.iters if args.iters > 0 else 8
    desc = [(p.dim, p.n, p.nodes, p.nu, p.dt) for p in probs]
    u0s = [torch.tensor(p.u0(), device="cuda") for p in probs]
    opts = dict(smoother=1, omega=1.0, vcycles=2, precision=1)
    if args.vcycle_tail >= 0:
        opts["vcycle_tail"] = args.vcycle_tail

    def job(b):
        for i, u in enumerate(u0s):
            pmg.pfasst_mg_batch_set_initial(b.h, i, u)
        return b.run(steps, sweeps)

    b = pmg.BatchSolver(desc, **opts)
    for _ in range(args.warmup):
        job(b)
    torch.cuda.synchronize()
    l0 = b.launches()
    cp, cf = sample_clocks_start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    for _ in range(args.steps):
        res = job(b)
    ev1.record()
    torch.cuda.synchronize()
    clocks = sample_clocks_stop(cp, cf, local)
    ms = ev0.elapsed_time(ev1) / args.steps
    launches = b.launches() - l0
    dof_sweeps = sum(p.dofs * (p.nodes - 1) for p in probs) * sweeps * steps
    # same job issued eagerly, problem after problem (no graph branches)
    e = pmg.BatchSolver(desc, use_graphs=0, **opts)
    job(e)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    job(e)
    torch.cuda.synchronize()
    eager_ms = 1000 * (time.perf_counter() - t1)
    e.close()
    # end to end: host initial values in, host end values out
    hosts = [p.u0() for p in probs]
    outs = [np.zeros(p.dofs) for p in probs]
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    for _ in range(args.steps):
        for i, u in enumerate(hosts):
            pmg.pfasst_mg_batch_set_initial(b.h, i, u)
        b.run(steps, sweeps)
        for i in range(len(probs)):
            pmg.pfasst_mg_batch_get_solution(b.h, i, outs[i])
    e2e_ms = 1000 * (time.perf_counter() - t2) / args.steps
    nbytes = sum(p.dofs * 8 for p in probs)
    b.close()
    line = {"metric": "DOF-sweeps/s", "value": dof_sweeps / (ms / 1000.0), "unit": "DOF-sweeps/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": "heat_uneven_batch64", "problems": len(probs),
                       "grids": "2D {63,127,255,511}^2, 3D {31,63,127}^3 (seed 64)", "time_steps": steps,
                       "sweeps_per_step": sweeps, "smoother": "V(2,1) red-black Gauss-Seidel", "vcycles": 2,
                       "precision": "FP32 V-cycles, FP64 SDC", "max_residual": float(np.max(res)),
                       "eager_ms_per_step": eager_ms, "graph_speedup_vs_eager": eager_ms / ms,
                       "l2": "problems are small; the graph is replayed on warm caches (no flush)"},
            "e2e": {"value": dof_sweeps / (e2e_ms / 1000.0), "unit": "DOF-sweeps/s", "h2d_bytes_per_step": nbytes,
                    "d2h_bytes_per_step": nbytes, "ms_per_step": e2e_ms},
            "gpu_launches": launches, "clocks": clocks}
    if rank == 0:
        print(json.dumps(line), flush=True)


NET_LAYER2_FLOPS = 2 * 27 * 16 * 16  # one point of the 16 -> 16 layer (tensor cores)
NET_FLOPS_FWD = 2 * 27 * (1 * 16 + 16 * 16 + 16 * 1)  # one point, three layers


def run_learned(args):
    """Training of the learned multigrid correction network: one step = one Adam step on
    a fresh batch of 16 grids of 63^3 points drawn by the library's sampler (noise after
    one red-black sweep, loss power 2): sampling, forward, loss, backward, weight
    gradients, Adam -- all library kernels.  value = grid points through forward and
    backward per second.  Roofline: the 16 -> 16 tensor-core layer (forward)."""
    import torch
    import paper_1407_6486_gb300 as pmg
    from paper_1407_6486_gb300 import _build

    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    _build.build()
    pmg.load()
    B, n = 16, 63
    pts = B * n ** 3
    tr = pmg.NetTrainer(B, n)
    tr.train(max(args.warmup, 3), 2e-3, 7, 0.08, 1.0 / 6.0, 0, 2)
    torch.cuda.synchronize()
    tr.profile(1, 0)
    l0 = tr.launches()
    clk_p, clk_f = sample_clocks_start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    hist = tr.train(args.steps, 2e-3, 1000, 0.08, 1.0 / 6.0, 0, 2)
    ev1.record()
    torch.cuda.synchronize()
    clocks = sample_clocks_stop(clk_p, clk_f, local)
    ms = ev0.elapsed_time(ev1) / args.steps
    launches = tr.launches() - l0
    stats = tr.profile_read()
    tr.profile(0, 0)
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            peak, peak_src = float(json.load(fh)["bf16_tflops"]), "measured bf16_tflops (burst)"
    except Exception:
        peak, peak_src = 1900.0, "fallback"
    by = {st["kernel"]: st for st in stats}
    l2 = by.get("net_layer2_mma")
    roof = None
    if l2 and l2["launches"]:
        avg_ms = l2["ms"] / l2["launches"]
        ach = NET_LAYER2_FLOPS * (l2["points"] / l2["launches"]) / (avg_ms / 1000.0) / 1e12
        roof = {"bound": "tensor", "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
                "traffic": None, "kernel": "net_layer2_mma", "launches": l2["launches"], "avg_launch_ms": avg_ms,
                "algo_flops_per_point": NET_LAYER2_FLOPS, "peak_source": peak_src}
    kernels = sorted(({"kernel": st["kernel"], "ms_per_step": st["ms"] / args.steps,
                       "launches_per_step": st["launches"] / args.steps} for st in stats),
                     key=lambda d: -d["ms_per_step"])
    # end to end through the public API: host batch in (x, t, kappa), loss out
    x, t, k = tr.sample(4242, 0.08, 1.0 / 6.0)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        tr.step(x, t, k, power=2, lr=2e-3)
    e2e_ms = 1000 * (time.perf_counter() - t0) / args.steps
    tr.close()
    line = {"metric": "network training points/s", "value": pts / (ms / 1000.0), "unit": "points/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "bf16+f32", "data": "synthetic",
            "config": {"workload": "learned_train_16x63^3", "batch": B, "grid": f"{n}^3",
                       "network": "3x3x3 conv 1->16->16->1, ReLU", "loss_power": 2,
                       "flops_per_point_fwd": NET_FLOPS_FWD, "final_loss": float(hist[-1]),
                       "l2": "activations 16 x 4.0M points x 2 B = 128 MB per layer, at the L2 size; no flush"},
            "roofline": roof, "kernels": kernels,
            "e2e": {"value": pts / (e2e_ms / 1000.0), "unit": "points/s", "h2d_bytes_per_step": 2 * pts * 4 + B * 4,
                    "d2h_bytes_per_step": 8, "ms_per_step": e2e_ms},
            "gpu_launches": launches, "clocks": clocks}
    if rank == 0 and world == 1 and not args.no_cpu_baseline and not args.quick:
        from oracle import learned as N
        rng = np.random.default_rng(3)
        nn = 24
        xs, ts = rng.standard_normal((nn, nn, nn)), rng.standard_normal((nn, nn, nn))
        prm = N.init_params(5)
        t0 = time.perf_counter()
        reps = 0
        while time.perf_counter() - t0 < 10.0:
            N.loss_and_grads(prm, [xs], [ts], [0.15], 2)
            reps += 1
        sec = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": reps * nn ** 3 / sec, "unit": "points/s", "cores": 1, "kind": "oracle",
                                "sample": f"{reps} FP64 numpy forward+backward passes on one {nn}^3 grid"}
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_learned_deploy(args):
    """The learned-correction workload: train the 3-layer 3x3x3 BF16 convolutional
    correction network (16 channels, ReLU) on error/residual pairs of the sub-step
    problems of 3D heat on 127^3 with Gaussian-random-field initial values (length
    scale 0.1, seeds 5, 6, ...), then deploy it in two-level PFASST on 255^3 / 127^3,
    16 slices, 5/3 Gauss-Lobatto nodes, one V(2,1) red-black cycle per sub-step, mixed
    precision, with the plain V-cycle kept on every level where the measured contraction
    does not drop.  Pairs: the library's FP64 multigrid solves each sub-step
    (I - c Lap_h) u = u0 to 1e-12; its initial error u* - u0 after one red-black sweep is
    the target, the scaled residual the input (pfasst_mg_net_substep_pairs); cut into
    32^3 crops.  value = DOF-sweeps/s of the deployed solver to the residual the plain
    solver reaches in 10 iterations (the same metric as the 3D workload); the plain
    solver's value and the error of both against the per-mode collocation solution of the
    sine-mode initial value of the 3D workload are in `config`."""
    import math
    import torch
    import paper_1407_6486_gb300 as pmg
    from paper_1407_6486_gb300 import _build, inputs

    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    _build.build()
    pmg.load()
    # ---- training pairs: 127^3 GRF fields, kappa over the deployment's operators
    ng, gb, crop = 127, 8, 32
    fields = args.learned_fields
    rng = np.random.default_rng(5)
    t0 = time.perf_counter()
    gen = pmg.NetTrainer(gb, ng)
    offs = [0, 32, 64, ng - crop]
    xs, ts, ks = [], [], []
    u0d = torch.empty((gb, ng ** 3), dtype=torch.float64, device="cuda")
    xg = torch.empty((gb, ng ** 3), dtype=torch.float32, device="cuda")
    tg = torch.empty_like(xg)
    for f0 in range(0, fields, gb):
        kap = rng.uniform(0.03, 1.0 / 6.0 - 1e-3, gb).astype(np.float32)
        for b in range(gb):
            u0d[b] = torch.from_numpy(inputs.gaussian_random_field(ng, 0.1, 5 + f0 + b))
        gen.substep_pairs(u0d, kap, xg, tg)
        xv, tv = xg.view(gb, ng, ng, ng), tg.view(gb, ng, ng, ng)
        for b in range(gb):
            for oz in offs:
                for oy in offs:
                    for ox in offs:
                        xs.append(xv[b, oz:oz + crop, oy:oy + crop, ox:ox + crop].reshape(-1))
                        ts.append(tv[b, oz:oz + crop, oy:oy + crop, ox:ox + crop].reshape(-1))
                        ks.append(kap[b])
    gen.close()
    X, T, K = torch.stack(xs), torch.stack(ts), np.array(ks, dtype=np.float32)
    del xs, ts
    torch.cuda.synchronize()
    pair_s = time.perf_counter() - t0
    # ---- training on the GPU: Adam on batches of 16 crops, power-1 loss (scaled residual)
    npairs, tb = X.shape[0], 16
    hold = torch.arange(npairs - 64, npairs, device="cuda")
    tr = pmg.NetTrainer(tb, crop)
    t1 = time.perf_counter()
    hist = []
    for ep in range(args.learned_epochs):
        perm = torch.randperm(npairs - 64, device="cuda", generator=torch.Generator(device="cuda").manual_seed(ep))
        for i in range(0, npairs - 64 - tb + 1, tb):
            idx = perm[i:i + tb]
            hist.append(tr.step(X[idx].contiguous(), T[idx].contiguous(), K[idx.cpu().numpy()], power=1,
                                lr=2e-3 if ep == 0 else 1e-3))
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t1
    prm = tr.params()
    held = [tr.gradients(X[hold[j:j + tb]].contiguous().cpu().numpy(), T[hold[j:j + tb]].contiguous().cpu().numpy(),
                         K[hold[j:j + tb].cpu().numpy()], power=1)[0] for j in range(0, 64, tb)]
    held_zero = float(0.5 * (X[hold].double() ** 2).mean())  # the same loss with no correction (y = 0)
    tr.close()
    del X, T
    torch.cuda.empty_cache()
    # ---- deployment: 255^3 / 127^3, 16 slices, one V-cycle per sub-step, mixed
    wl = inputs.heat3d_c3(n=255, slices=16)
    wl.vcycles = 1
    u0 = torch.tensor(wl.u0(), device="cuda")
    n, h = wl.n, 1.0 / (wl.n + 1)
    xg1 = np.arange(1, n + 1) * h
    want = np.zeros((n, n, n))
    for k, a in zip(wl.modes, wl.amps):
        z = wl.dt * wl.nu * sum((2 * math.cos(kk * math.pi * h) - 2) / h ** 2 for kk in k)
        want += a * _pade(z, wl.fine_nodes) ** wl.slices * np.einsum(
            "k,j,i->kji", np.sin(k[2] * np.pi * xg1), np.sin(k[1] * np.pi * xg1), np.sin(k[0] * np.pi * xg1))
    out = torch.empty(n ** 3, dtype=torch.float64, device="cuda")
    opts = dict(smoother=1, omega=1.0, vcycles=1, precision=1)
    rows, target, k_ref = {}, None, None
    for name in ("plain", "net"):
        s = pmg.PFASSTSolver(3, n, 5, 3, wl.slices, wl.nu, wl.dt, **opts)
        rho = None
        if name == "net":  # levels kept only where the handle's own PFASST residual drops
            s.set_initial(u0)
            rho = s.set_smoother_net(prm, min_n=15, calibrate=2)
        if target is None:
            s.set_initial(u0)
            _, k_ref, r10 = s.iterate(10, 0.0)
            target = float(f"{r10 * 1.01:.4e}")
        for _ in range(max(args.warmup, 1)):
            s.set_initial(u0)
            s.iterate(60, target)
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ms, its = [], []
        for _ in range(args.steps):
            ev0.record()
            s.set_initial(u0)
            rc, it, res = s.iterate(60, target)
            ev1.record()
            torch.cuda.synchronize()
            ms.append(ev0.elapsed_time(ev1))
            its.append(it)
        pmg.pfasst_mg_get_solution(s.h, wl.slices - 1, 4, out)
        err = float(np.abs(out.cpu().numpy().reshape(n, n, n) - want).max() / np.abs(want).max())
        dof = n ** 3 * 4 * wl.slices * k_ref
        rows[name] = {"ms_per_step": statistics.median(ms), "iterations": its[-1], "final_residual": res,
                      "reached": rc == pmg.PMG_OK, "dof_sweeps_per_s": dof / (statistics.median(ms) / 1000.0),
                      "rel_error_vs_collocation": err}
        if rho is not None:
            rows[name].update({"calibration_residual_plain": rho[0], "calibration_residual_net": rho[1],
                               "levels_kept_mask": rho[2],
                               "calibration": "fine collocation residual after 3 PFASST iterations, plain vs "
                                              "with each level added (finest first)"})
        s.close()
        torch.cuda.empty_cache()
    net, plain = rows["net"], rows["plain"]
    line = {"metric": "DOF-sweeps/s", "value": net["dof_sweeps_per_s"], "unit": "DOF-sweeps/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": net["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "bf16+f32+f64", "data": "synthetic",
            "config": {"workload": "learned_heat3d_n255_pfasst5x3_P16_1vc",
                       "training": {"pairs": int(npairs), "fields": fields, "field": "127^3 GRF, length scale 0.1",
                                    "crop": "32^3", "epochs": args.learned_epochs, "steps": len(hist),
                                    "final_loss": float(np.mean(hist[-20:])), "held_out_loss": float(np.mean(held)),
                                    "held_out_loss_without_correction": held_zero,
                                    "pair_seconds": pair_s, "train_seconds": train_s},
                       "K_ref": k_ref, "residual_target": target, "with_network": net, "plain_vcycle": plain,
                       "gain_vs_plain": net["dof_sweeps_per_s"] / plain["dof_sweeps_per_s"],
                       "l2": "working set ~27 GB per solver, far above L2; no flush"},
            "gpu_launches": None}
    if rank == 0:
        print(json.dumps(line), flush=True)


def _pade(z, s):
    """Diagonal (s-1, s-1) Pade approximant of exp(z): the Gauss-Lobatto collocation step."""
    import math
    N = s - 1
    c = [math.factorial(2 * N - j) * math.factorial(N) / (math.factorial(2 * N) * math.factorial(j)
                                                           * math.factorial(N - j)) for j in range(N + 1)]
    return sum(c[j] * z ** j for j in range(N + 1)) / sum(c[j] * (-z) ** j for j in range(N + 1))


def run_compare(args):
    """Solver comparison (a GPU analogue of the paper's full-solve PFASST / ISDC / MLSDC
    table, Sec. 4.2.1): 3D heat nu = 0.5 on 127^3 (coarse 63^3), dt = 0.002, 16 slices,
    16 sine modes (seed 6486), 5/3 Gauss-Lobatto nodes, red-black V(2,1).  Every variant
    integrates the block [0, 16 dt] until the collocation residual of every slice is
    <= 1e-9: PFASST with 2 V-cycles per sub-step (mixed and FP64) or with sub-steps solved
    to 1e-12 (FP64), and the serial methods one slice after another: MLSDC (two levels,
    2 V-cycles), ISDC (one level, 2 V-cycles) and ISDC with full solves.  Reported per
    variant: time, iterations, fine sweeps, final residual, and the max error of the end
    value against the serial collocation solution (Pade^16 per sine mode)."""
    import math
    import torch
    import paper_1407_6486_gb300 as pmg
    from paper_1407_6486_gb300 import _build, inputs

    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    _build.build()
    pmg.load()
    wl = inputs.heat3d_c3(n=127, slices=16)
    tol, maxit = 1e-9, 400
    n, h = wl.n, 1.0 / (wl.n + 1)
    x = np.arange(1, n + 1) * h
    want = np.zeros((n, n, n))
    for k, a in zip(wl.modes, wl.amps):
        z = wl.dt * wl.nu * sum((2 * math.cos(kk * math.pi * h) - 2) / h ** 2 for kk in k)
        want += a * _pade(z, wl.fine_nodes) ** wl.slices * np.einsum(
            "k,j,i->kji", np.sin(k[2] * np.pi * x), np.sin(k[1] * np.pi * x), np.sin(k[0] * np.pi * x))
    u0 = torch.tensor(wl.u0(), device="cuda")
    variants = [("pfasst_2vc_mixed", 2, 16, dict(vcycles=2, precision=1)),
                ("pfasst_2vc_fp64", 2, 16, dict(vcycles=2, precision=0)),
                ("pfasst_full_fp64", 2, 16, dict(vcycles=0, precision=0, mg_tol=1e-12)),
                ("mlsdc_2vc_mixed", 2, 1, dict(vcycles=2, precision=1)),
                ("isdc_2vc_mixed", 1, 1, dict(vcycles=2, precision=1)),
                ("isdc_full_fp64", 1, 1, dict(vcycles=0, precision=0, mg_tol=1e-12))]
    rows = []
    for name, nl, P, opts in variants:
        s = pmg.PFASSTSolver(3, n, wl.fine_nodes, wl.coarse_nodes if nl == 2 else 0, P, wl.nu, wl.dt, nlevels=nl,
                             smoother=1, omega=1.0, **opts)
        out = torch.empty(n ** 3, dtype=torch.float64, device="cuda")

        def solve():
            if P == wl.slices:
                s.set_initial(u0)
                rc, it, res = s.iterate(maxit, tol)
                return it, it * P, res, rc == pmg.PMG_OK
            u, its, ok, res = u0, 0, True, 0.0
            for _ in range(wl.slices):
                s.set_initial(u)
                rc, it, r = s.iterate(maxit, tol)
                its, ok, res = its + it, ok and rc == pmg.PMG_OK, max(res, r)
                pmg.pfasst_mg_get_solution(s.h, 0, wl.fine_nodes - 1, out)
                u = out.clone()
            return its, its, res, ok

        solve()  # warm-up (graph capture, caches)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        its, sweeps, res, ok = solve()
        torch.cuda.synchronize()
        sec = time.perf_counter() - t0
        end = (out if P == 1 else pmg.pfasst_mg_get_solution(s.h, P - 1, wl.fine_nodes - 1, out)).cpu().numpy()
        err = float(np.abs(end.reshape(n, n, n) - want).max() / np.abs(want).max())
        rows.append({"variant": name, "seconds": sec, "iterations": its, "fine_sweeps": sweeps,
                     "final_residual": res, "reached_1e-9": ok, "rel_error_vs_collocation": err})
        s.close()
        torch.cuda.empty_cache()
    best = min((r for r in rows if r["reached_1e-9"]), key=lambda r: r["seconds"], default=rows[0])
    dofs = n ** 3 * (wl.fine_nodes - 1)
    line = {"metric": "seconds to collocation residual 1e-9", "value": best["seconds"], "unit": "s", "n_gpus": world,
            "steps": 1, "warmup": 1, "ms_per_step": best["seconds"] * 1000, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": "heat3d_n127_compare_P16", "grid": "127^3/63^3", "slices": wl.slices,
                       "nodes": "5/3 Gauss-Lobatto", "best": best["variant"],
                       "dof_sweeps_per_fine_sweep_of_one_slice": dofs, "variants": rows,
                       "l2": "not flushed between variants (each variant's state is hundreds of MB to GB)"},
            "gpu_launches": None}
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_heat1d(args):
    """The 1D configuration: heat u_t = u_xx on 127 points, u0 = sin(pi x) + 0.5 sin(3 pi x),
    single-level SDC with 3 Gauss-Lobatto nodes, dt = 0.01 to T = 0.1 (10 steps), each step
    swept until its collocation residual is <= 1e-9 (at most 50 sweeps), sub-steps solved by
    2 V(2,1) cycles of weighted Jacobi (2/3) down to 3 points, FP64.  A latency-bound case:
    time and sweeps/s only, no roofline.  The error of the end value against the discrete
    solution of the semi-discrete problem (Pade(2,2) per sine mode) is reported too."""
    import math
    import torch
    import paper_1407_6486_gb300 as pmg
    from paper_1407_6486_gb300 import _build, inputs

    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    _build.build()
    pmg.load()
    wl = inputs.heat1d_c1()
    tail = dict(vcycle_tail=args.vcycle_tail) if args.vcycle_tail >= 0 else {}
    s = pmg.PFASSTSolver(1, wl.n, wl.fine_nodes, 0, 1, wl.nu, wl.dt, nlevels=1, smoother=wl.smoother,
                         omega=wl.omega, vcycles=wl.vcycles, precision=wl.precision, **tail)
    u0 = torch.tensor(wl.u0(), device="cuda")
    out = torch.empty(wl.n, dtype=torch.float64, device="cuda")

    def solve():
        u, sweeps = u0, 0
        for _ in range(wl.steps):
            s.set_initial(u)
            rc, it, res = s.iterate(wl.iterations, 1e-9)
            sweeps += it
            pmg.pfasst_mg_get_solution(s.h, 0, wl.fine_nodes - 1, out)
            u = out.clone()
        return sweeps, u

    for _ in range(max(args.warmup, 1)):
        solve()
    torch.cuda.synchronize()
    times, sweeps = [], 0
    l0 = s.launches()
    cp, cf = sample_clocks_start()
    for _ in range(max(args.steps, 1)):
        t0 = time.perf_counter()
        sweeps, u = solve()
        torch.cuda.synchronize()
        times.append(time.perf_counter() - t0)
    clocks = sample_clocks_stop(cp, cf, local)
    launches = (s.launches() - l0) // max(args.steps, 1)
    sec = min(times)
    h = 1.0 / (wl.n + 1)
    x = np.arange(1, wl.n + 1) * h
    want = np.zeros(wl.n)
    for k, a in zip(wl.modes, wl.amps):
        z = wl.dt * wl.nu * (2 * math.cos(k[0] * math.pi * h) - 2) / h ** 2
        want += a * _pade(z, wl.fine_nodes) ** wl.steps * np.sin(k[0] * math.pi * x)
    err = float(np.abs(u.cpu().numpy() - want).max())
    dof_sweeps = wl.n * (wl.fine_nodes - 1) * sweeps
    line = {"metric": "DOF-sweeps/s", "value": dof_sweeps / sec, "unit": "DOF-sweeps/s", "n_gpus": world,
            "steps": len(times), "warmup": max(args.warmup, 1), "ms_per_step": 1000 * sec, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": wl.name, "sweeps_to_1e-9_over_10_steps": sweeps, "sweeps_per_s": sweeps / sec,
                       "max_error_vs_collocation": err, "timing": "wall clock of the 10-step solve, best of the runs",
                       "l2": "127 points: the whole state stays in L2 and L1 (latency-bound; no flush)"},
            "gpu_launches": launches, "clocks": clocks}
    s.close()
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # the FP64 oracle runs the same 10-step solve (single-level SDC, sweeps to 1e-9)
        import oracle as O
        cores = O.set_threads(1)
        o = O.PFASST(1, wl.n, wl.fine_nodes, 2, 1, wl.nu, wl.dt,
                     O.MGParams(smoother=wl.smoother, omega=wl.omega, vcycles=wl.vcycles), nlevels=1)
        ctimes = []
        for _ in range(3):
            u, osweeps = wl.u0(), 0
            t0 = time.perf_counter()
            for _ in range(wl.steps):
                o.set_initial(u)
                it, _ = o.run(wl.iterations, 1e-9)
                osweeps += it
                u = o.end_value()
            ctimes.append(time.perf_counter() - t0)
        csec = min(ctimes)
        line["cpu_baseline"] = {"value": wl.n * (wl.fine_nodes - 1) * osweeps / csec, "unit": "DOF-sweeps/s",
                                "cores": cores, "kind": "oracle",
                                "sample": f"the whole 10-step solve ({osweeps} sweeps), best of 3, {1000 * csec:.1f} ms",
                                "nproc": os.cpu_count(), "cpu_model": cpu_model()}
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_weak3(args):
    """Three-level PFASST (Sec. 2.4 with a middle level).  Part 1, the weak-scaling runs
    of Sec. 4.2.2 on the GPU: 1D heat, k = nu = T = 1, N_x = N_t = N parallel steps
    (N = 32 .. 1024), 3 uniform nodes on levels 0 and 1, backward Euler on level 2,
    two V(2,2) Gauss-Seidel cycles, FP64; per N the iteration at which the PDE error of
    the last step first comes within 1.6x of its level after 20 iterations, and the time
    per iteration.  Part 2: the 3D workload (255^3, 32 slices, 5/3 Gauss-Lobatto nodes,
    mixed precision) with two levels against three (5/3/3 and 5/3/2, level 2 on 63^3): time
    and iterations to the collocation residual that two levels reach in 10 iterations."""
    import math
    import torch
    import paper_1407_6486_gb300 as pmg
    from paper_1407_6486_gb300 import _build, inputs

    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    _build.build()
    pmg.load()
    weak = []
    for N in (32, 64, 128, 256, 512, 1024):
        n, P, dt = N - 1, N, 1.0 / N
        x = np.arange(1, n + 1) / (n + 1)
        pde = math.exp(-math.pi ** 2) * np.sin(np.pi * x)
        s = pmg.PFASSTSolver(1, n, 3, 3, P, 1.0, dt, nlevels=3, coarsest_nodes=2, family=1, smoother=1, omega=1.0,
                             nu1=2, nu2=2, vcycles=2)
        u0 = torch.tensor(np.sin(np.pi * x), device="cuda")
        out = torch.empty(n, dtype=torch.float64, device="cuda")
        s.set_initial(u0)
        s.iterate(1, 0.0)  # warm-up: graph capture
        s.set_initial(u0)
        errs, secs = [], 0.0
        for _ in range(20):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            s.iterate(1, 0.0)
            torch.cuda.synchronize()
            secs += time.perf_counter() - t0
            pmg.pfasst_mg_get_solution(s.h, P - 1, 2, out)
            errs.append(float(np.abs(out.cpu().numpy() - pde).max()))
        reach = next(k + 1 for k, e in enumerate(errs) if e <= 1.6 * errs[-1])
        weak.append({"N": N, "slices": P, "iterations_to_error_level": reach, "error_level": errs[-1],
                     "ms_per_iteration": secs / 20 * 1000})
        s.close()
    wl = inputs.heat3d_c3()
    u0 = torch.tensor(wl.u0(), device="cuda")
    three, target = [], None
    for nl, s2 in ((2, 0), (3, 3), (3, 2)):
        s = pmg.PFASSTSolver(3, wl.n, 5, 3, wl.slices, wl.nu, wl.dt, nlevels=nl, coarsest_nodes=s2,
                             smoother=1, omega=1.0, vcycles=2, precision=1)
        s.set_initial(u0)
        _, _, r10 = s.iterate(10, 0.0)  # warm-up; two levels fix the target
        if target is None:
            target = 1.01 * r10
        s.set_initial(u0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rc, it, res = s.iterate(60, target)
        torch.cuda.synchronize()
        sec = time.perf_counter() - t0
        three.append({"levels": nl, "nodes": "5/3" if nl == 2 else f"5/3/{s2}", "seconds": sec, "iterations": it,
                      "final_residual": res, "target": target, "reached": rc == pmg.PMG_OK})
        s.close()
        torch.cuda.empty_cache()
    best = min(three, key=lambda r: r["seconds"])
    line = {"metric": "seconds to the two-level 10-iteration residual", "value": best["seconds"], "unit": "s",
            "n_gpus": world,
            "steps": 1, "warmup": 1, "ms_per_step": best["seconds"] * 1000, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": "heat3d_n255_P32_two_vs_three_levels", "best_levels": best["levels"],
                       "three_vs_two": three, "weak_scaling_1d_three_levels": weak,
                       "l2": "not flushed (state of GBs per solve)"},
            "gpu_launches": None}
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_order4(args):
    """The three discretisations of the paper's 3D study (Sec. 4.2.1): u_t = nu Lap u on the
    unit cube, nu = 1/3, u0 = sin(pi x) sin(pi y) sin(pi z), T = 1, uniform nodes:
      2/2: 127^3, 2nd-order stencil, 128 steps, midpoint + right node (M = 2), coarse
           backward Euler on 63^3;
      2/4: 127^3, 2nd-order stencil, 24 steps, M = 4 (fourth order), coarse backward Euler;
      4/4: 31^3, 4th-order stencil, 24 steps, M = 4, coarse 15^3 with the 2nd-order
           stencil and backward Euler.
    Each runs as PFASST with up to 32 steps batched on the GPU per block (the paper's
    largest number of time ranks; 128 steps = 4 blocks one after another) and as serial
    ISDC (one step after another), with two V(2,2) red-black Gauss-Seidel cycles per
    sub-step in mixed precision, until the collocation residual of every step is <= 1e-9
    (the paper's tolerance).  Reported: time, iterations, and the max error of the final
    value against the analytical solution exp(-pi^2) sin sin sin."""
    import math
    import torch
    import paper_1407_6486_gb300 as pmg
    from paper_1407_6486_gb300 import _build, inputs

    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    _build.build()
    pmg.load()
    nu, T, tol, maxit = 1.0 / 3.0, 1.0, 1e-9, 200
    configs = [("2/2", 127, 2, 128, 3), ("2/4", 127, 2, 24, 5), ("4/4", 31, 4, 24, 5)]
    rows = []
    only = args.order4_only.split(",") if args.order4_only else None
    for name, n, order, steps, nodes in configs:
        if only and name not in only:
            continue
        x = np.arange(1, n + 1) / (n + 1)
        s1 = np.sin(np.pi * x)
        u0 = np.einsum("k,j,i->kji", s1, s1, s1).reshape(-1)
        exact = math.exp(-3 * math.pi ** 2 * nu * T) * u0
        u0d = torch.tensor(u0, device="cuda")
        out = torch.empty(n ** 3, dtype=torch.float64, device="cuda")
        dt = T / steps
        # PFASST with the coarse level's sub-steps solved like the fine level's (two V-cycles),
        # by six V-cycles, or to the tolerance (coarse_vcycles 0), and serial ISDC
        methods = [("pfasst", -1), ("pfasst", 6), ("pfasst", 0), ("isdc", -1)] if name == "2/2" else \
            [("pfasst", -1), ("isdc", -1)]
        for method, cvc in methods:
            P, nl = (min(steps, 32), 2) if method == "pfasst" else (1, 1)
            s = pmg.PFASSTSolver(3, n, nodes, 2 if nl == 2 else 0, P, nu, dt, nlevels=nl, family=1, order=order,
                                 smoother=1, omega=1.0, nu1=2, nu2=2, vcycles=2, precision=1, coarse_vcycles=cvc)

            def solve():
                # blocks of P steps; each block starts from the previous block's end value
                u, its, ok, res = u0d, 0, True, 0.0
                for _ in range(steps // P):
                    s.set_initial(u)
                    rc, it, r = s.iterate(maxit, tol)
                    its, ok, res = its + it, ok and rc == pmg.PMG_OK, max(res, r)
                    pmg.pfasst_mg_get_solution(s.h, P - 1, nodes - 1, out)
                    u = out.clone()
                return its, res, ok

            solve()  # warm-up: graph capture, autotuned kernels
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            its, res, ok = solve()
            torch.cuda.synchronize()
            sec = time.perf_counter() - t0
            err = float(np.abs(out.cpu().numpy() - exact).max())
            rows.append({"config": name, "method": method, "coarse_vcycles": "as fine (2)" if cvc < 0 else
                         ("solved to 1e-12" if cvc == 0 else cvc) if method == "pfasst" else None,
                         "grid": f"{n}^3", "stencil_order": order, "steps": steps,
                         "steps_per_block": P, "nodes": nodes, "seconds": sec, "iterations": its, "final_residual": res,
                         "reached_1e-9": ok, "max_error_vs_exact": err})
            s.close()
            torch.cuda.empty_cache()
    best = min((r for r in rows if r["reached_1e-9"]), key=lambda r: r["seconds"], default=rows[0])
    line = {"metric": "seconds to collocation residual 1e-9", "value": best["seconds"], "unit": "s", "n_gpus": world,
            "steps": 1, "warmup": 1, "ms_per_step": best["seconds"] * 1000, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": "heat3d_sinsinsin_T1_three_discretisations", "best": best["config"] + " " +
                       best["method"], "runs": rows, "l2": "not flushed between runs"},
            "gpu_launches": None}
    if rank == 0:
        print(json.dumps(line), flush=True)


RES_TOL = 0.01  # relative tolerance on the FP64 path's residual (the bench's "fixed residual")


def run_ours(args):
    import torch
    import paper_1407_6486_gb300 as pmg

    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_1407_6486_gb300 import _build
    if rank == 0:
        _build.build()
    if world > 1:
        torch.distributed.barrier()
    pmg.load()
    wl = make_workload(args.workload)
    if args.quick and args.iters > 0:
        wl.iterations = args.iters
    if args.vcycles >= 0:
        wl.vcycles = args.vcycles
    if args.precision >= 0:
        wl.precision = args.precision
    stream = torch.cuda.current_stream()
    u0 = wl.u0()
    u0_dev = torch.tensor(u0, device="cuda")
    common = dict(smoother=wl.smoother, omega=wl.omega, vcycles=wl.vcycles, interp_order=4)
    # the measured variant's coarse-level V-cycles (the FP64 reference keeps the workload's)
    variant = dict(coarse_vcycles=args.coarse_vcycles) if args.coarse_vcycles >= 0 else {}
    if args.vcycle_tail >= 0:
        variant["vcycle_tail"] = args.vcycle_tail

    fp64_ms, fp64_runs = None, []
    r_ref = None
    if args.quick:
        k_ref, target = wl.iterations, 0.0
    else:
        # calibration: plain FP64 GPU path, the workload's iteration count -> residual target
        ref = pmg.PFASSTSolver(wl.dim, wl.n, wl.fine_nodes, wl.coarse_nodes, wl.slices, wl.nu, wl.dt,
                               nlevels=wl.nlevels, precision=0, **common)
        ref.set_initial(u0_dev)
        _, k_ref, r_ref = ref.iterate(wl.iterations, 0.0)
        # the same residual to RES_TOL: FP32 V-cycles perturb U at the FP32 rounding level
        # (~1e-7 |U|), which moves a residual of ~1e-4 |U| by ~0.1 %
        target = float(f"{r_ref * (1.0 + RES_TOL):.4e}")
        # the plain FP64 path to that target (same schedule, graphs): its iteration count is
        # K_ref; when the measured variant is not itself FP64 it is timed over repeated steps
        # (median and spread), after one untimed step
        ref.set_initial(u0_dev)
        _, k_ref, _ = ref.iterate(4 * wl.iterations, target)
        if wl.precision != 0:
            fp64_runs = []
            for _ in range(args.fp64_steps):
                torch.cuda.synchronize()
                f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                f0.record(stream)
                ref.set_initial(u0_dev)
                ref.iterate(4 * wl.iterations, target)
                f1.record(stream)
                torch.cuda.synchronize()
                fp64_runs.append(f0.elapsed_time(f1))
            fp64_ms = statistics.median(fp64_runs) if fp64_runs else None
        ref.close()
        del ref
        torch.cuda.empty_cache()

    s = pmg.PFASSTSolver(wl.dim, wl.n, wl.fine_nodes, wl.coarse_nodes, wl.slices, wl.nu, wl.dt,
                         nlevels=wl.nlevels, precision=wl.precision, **common, **variant)
    maxit = wl.iterations if args.quick else 4 * wl.iterations
    if args.tma:
        for lev in range(8):
            for narrow in (0, 1):
                try:
                    pmg.pfasst_mg_set_tuning(s.h, lev, narrow, args.tma, 32, 512)
                except pmg.PMGError:
                    pass
    if args.pin_tuning:
        # level:narrow:variant:param:threads entries (the tuning_codes of an earlier bench line)
        for item in args.pin_tuning.split():
            lev, narrow, fz, prm, thr = (int(v) for v in item.split(":"))
            pmg.pfasst_mg_set_tuning(s.h, lev, narrow, fz, prm, thr)
    tuning, codes = [], []

    def kind_of(fz, prm, thr):
        return {0: f"point x{prm}", 1: f"fused z{prm or 32} x{thr}", 2: f"tma z{prm}", 3: f"tma4 z{prm}"}.get(fz, "?")
    for lev in range(8):
        try:
            tw, tn = pmg.pfasst_mg_tuning(s.h, lev, 0), pmg.pfasst_mg_tuning(s.h, lev, 1)
            codes += [f"{lev}:0:{tw[0]}:{tw[1]}:{tw[2]}", f"{lev}:1:{tn[0]}:{tn[1]}:{tn[2]}"]
            wide, narrow = kind_of(*tw), kind_of(*tn)
            # the batch of all slices, and (after "|") single grids where that differs
            tuning.append(f"L{lev}:{wide}" + (f"|{narrow}" if narrow != wide else ""))
        except pmg.PMGError:
            break

    def step():
        s.set_initial(u0_dev)
        return s.iterate(maxit, target)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    launches0 = s.launches()
    # inputs larger than L2 (the 3D workload) need no flush; otherwise a 512 MB buffer is
    # rewritten between timed steps, outside the timed intervals
    flush = None if (wl.dim == 3 and wl.n >= 255) else torch.empty(1 << 27, dtype=torch.float32, device="cuda")
    cp, cf = sample_clocks_start()
    iters, step_ms = [], []
    torch.cuda.synchronize()
    for _ in range(args.steps):
        if flush is not None:
            flush.fill_(1.0)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        rc, it, res = step()
        ev1.record(stream)
        iters.append((rc, it, res))
        torch.cuda.synchronize()
        step_ms.append(ev0.elapsed_time(ev1))
    clocks = sample_clocks_stop(cp, cf, local)
    launches = s.launches() - launches0
    ms_total = sum(step_ms)
    # per-kernel CUDA-event times come from separate profiled steps of the same workload
    # after the timed region (an event pair around every launch on the fine grid, or around
    # every launch), so that the headline time carries no profiling overhead
    prof_steps = max(1, min(args.prof_steps, args.steps))
    pmg.pfasst_mg_profile(s.h, True, 0 if args.profile_all else wl.dofs)
    torch.cuda.synchronize()
    p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    p0.record(stream)
    for _ in range(prof_steps):
        if flush is not None:
            flush.fill_(1.0)
        step()
    p1.record(stream)
    torch.cuda.synchronize()
    prof_ms = p0.elapsed_time(p1) / prof_steps
    stats = pmg.pfasst_mg_profile_read(s.h)
    pmg.pfasst_mg_profile(s.h, False, 0)
    if args.profile_all:
        tot = sum(d["ms"] for d in stats)
        for d in sorted(stats, key=lambda d: -d["ms"]):
            print(f"{d['kernel']:>18} n={d['n']:>4} prec={d['precision']} launches/step={d['launches'] / prof_steps:8.0f} "
                  f"ms/step={d['ms'] / prof_steps:9.2f} share={d['ms'] / tot:6.1%}", file=sys.stderr)
    stats = [d for d in stats if d["n"] == wl.n]
    dof_sweeps = wl.dofs * (wl.fine_nodes - 1) * wl.slices * k_ref
    ms, value = job_time_and_value(ms_total / args.steps, dof_sweeps, world)

    # end to end through the C ABI with host buffers (h2d of u0, d2h of the end value)
    e2e_steps = 0 if args.quick else args.steps
    u0_host = torch.tensor(u0).pin_memory()
    out_host = torch.empty(wl.dofs, dtype=torch.float64).pin_memory()
    out_np = out_host.numpy()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        pmg.pfasst_mg_set_initial(s.h, u0_host.numpy())
        s.iterate(maxit, target)
        pmg.pfasst_mg_get_solution(s.h, wl.slices - 1, wl.fine_nodes - 1, out_np)
    torch.cuda.synchronize()
    e2e_ms, e2e_value = job_time_and_value(1000 * (time.perf_counter() - t0) / max(e2e_steps, 1), dof_sweeps, world)

    # roofline of the dominant kernel (by summed launch time on the fine grid): HBM for
    # the stencils / node mixes, the FP64 ALU for kernels bound by the FP64 pipe, against
    # the FP64 FMA rate the library's probe kernel measures on this GPU (best of 5)
    peak, peak_kind = measured_peak_gbs()
    fp64_peak = pmg.pfasst_mg_fp64_peak(5)

    def roof_of(d):
        flops = algo_fp64_flops_per_point(d["kernel"], wl.fine_nodes, wl.coarse_nodes)
        sec = d["ms"] / 1000.0
        tpp = traffic_for(d["kernel"], d["n"])
        traffic = (tpp * d["points"] / d["launches"]) if tpp is not None else None
        if flops > 0:
            achieved = flops * d["points"] / sec / 1e9
            return {"bound": "alu", "achieved": achieved, "peak": fp64_peak,
                    "unit": "GFLOP/s", "frac": achieved / fp64_peak, "traffic": traffic,
                    "kernel": d["kernel"], "grid": d["n"], "launches": d["launches"],
                    "avg_launch_ms": d["ms"] / d["launches"], "algo_fp64_flops_per_point": flops,
                    "peak_source": "measured: FP64 FMA probe kernel (pfasst_mg_fp64_peak, best of 5 launches "
                                   "of ~60 ms, every SM)",
                    "fp64_nominal_gflops": FP64_NOMINAL_GFLOPS}
        ts = 4 if d["precision"] == 1 else 8
        bpp = algo_bytes_per_point(d["kernel"], ts, wl.fine_nodes, wl.coarse_nodes)
        achieved = bpp * d["points"] / sec / 1e9
        return {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": traffic,
                "kernel": d["kernel"], "grid": d["n"], "launches": d["launches"],
                "avg_launch_ms": d["ms"] / d["launches"], "algo_bytes_per_point": bpp,
                "peak_source": f"{peak_kind} hbm_gbs"}

    dom = max(stats, key=lambda d: d["ms"]) if stats else None
    roof = roof_of(dom) if dom else None
    hbm_stats = [d for d in stats if algo_fp64_flops_per_point(d["kernel"]) == 0 and algo_bytes_per_point(d["kernel"], 4) > 0]
    roof_hbm = roof_of(max(hbm_stats, key=lambda d: d["ms"])) if hbm_stats else None
    line = {
        "metric": "DOF-sweeps/s", "value": value, "unit": "DOF-sweeps/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64" if wl.precision == 1 else "f64", "data": "synthetic",
        "config": {"workload": wl.name, "grid": f"{wl.n}^{wl.dim}/{(wl.n - 1) // 2}^{wl.dim}",
                   "slices": wl.slices, "nodes": f"{wl.fine_nodes}/{wl.coarse_nodes} Gauss-Lobatto",
                   "smoother": "V(2,1) " + ("red-black Gauss-Seidel" if wl.smoother == 1 else "Jacobi 2/3"),
                   "vcycles": wl.vcycles, "coarse_vcycles": args.coarse_vcycles if args.coarse_vcycles >= 0 else wl.vcycles,
                   "vcycle_tail": "auto" if args.vcycle_tail < 0 else args.vcycle_tail,
                   "precision": "FP32 V-cycles, FP64 SDC/FAS" if wl.precision else "FP64",
                   "K_ref": k_ref, "residual_target": target, "residual_tolerance": RES_TOL,
                   "fp64_residual_at_K_ref": r_ref, "iterations": [it for _, it, _ in iters],
                   "final_residual": iters[-1][2], "parallelism": f"replicas x{world}" if world > 1 else "1 GPU",
                   "l2": "working set > 60 GB, far above the 129 MB L2; no flush" if flush is None
                   else "L2 flushed (512 MB write) before every timed step, outside the timed interval",
                   "autotuned_smoothers": " ".join(tuning),
                   "tuning_codes": " ".join(codes[:-2]),  # (the exact coarsest level has no smoother)
                   "ms_per_step_median": statistics.median(step_ms),
                   "ms_per_step_min_max": [min(step_ms), max(step_ms)],
                   "fp64_plain_ms_per_step": fp64_ms,
                   "fp64_plain_repeats": len(fp64_runs),
                   "fp64_plain_ms_min_max": [min(fp64_runs), max(fp64_runs)] if fp64_runs else None,
                   "speedup_vs_fp64_plain": (fp64_ms / statistics.median(step_ms)) if fp64_ms else None},
        "roofline": roof,
        "roofline_hbm_kernel": roof_hbm,
        "kernels": sorted(({"kernel": d["kernel"], "n": d["n"], "ms_per_step": d["ms"] / prof_steps,
                            "launches_per_step": d["launches"] / prof_steps} for d in stats),
                          key=lambda d: -d["ms_per_step"])[:8],
        "kernel_timing": {"profiled_steps": prof_steps, "profiled_ms_per_step": prof_ms,
                          "how": "CUDA events around every fine-grid launch on the library's stream, in "
                                 "separate steps after the timed region"},
        "e2e": None if e2e_steps == 0 else {
            "value": e2e_value, "unit": "DOF-sweeps/s",
            "h2d_bytes_per_step": wl.dofs * 8, "d2h_bytes_per_step": wl.dofs * 8, "ms_per_step": e2e_ms},
        "gpu_launches": launches,
        "clocks": clocks,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline and not args.quick:
        orc = OracleSample(wl, args.ref_slices)
        v, tsec, cores = orc.sample()
        line["cpu_baseline"] = {"value": v, "unit": "DOF-sweeps/s", "cores": cores, "kind": "oracle",
                                "sample": f"one FP64 oracle PFASST iteration on {args.ref_slices} of the "
                                          f"{wl.slices} slices ({tsec:.1f} s)",
                                "nproc": os.cpu_count(), "cpu_model": cpu_model()}
        if args.single_thread_baseline:
            v1, t1, _ = orc.sample(threads=1)
            line["cpu_baseline"]["single_thread"] = {
                "value": v1, "unit": "DOF-sweeps/s", "cores": 1,
                "sample": f"the next oracle PFASST iteration on the same slice, one thread ({t1:.1f} s)"}
    s.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="heat3d",
                    choices=["heat3d", "heat3d-small", "heat3d-mid", "heat3d-255x4", "heat2d", "uneven", "learned-train", "learned",
                             "compare", "weak3", "order4", "heat1d"])
    ap.add_argument("--learned-fields", type=int, default=160,
                    help="learned: 127^3 GRF fields for the training pairs (64 crops each)")
    ap.add_argument("--learned-epochs", type=int, default=2)
    ap.add_argument("--quick", action="store_true",
                    help="profiling runs: no FP64 calibration (run the workload's iteration count), no e2e, "
                         "no CPU baseline")
    ap.add_argument("--ref-slices", type=int, default=1)
    ap.add_argument("--ref-threads", type=int, default=0,
                    help="--impl reference: oracle threads (0 = all host cores)")
    ap.add_argument("--single-thread-baseline", type=int, default=1,
                    help="1: also time one oracle iteration on one host thread")
    ap.add_argument("--fp64-steps", type=int, default=5,
                    help="timed repeats of the plain FP64 path (median reported)")
    ap.add_argument("--prof-steps", type=int, default=2,
                    help="profiled steps after the timed region (per-kernel CUDA-event times)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--iters", type=int, default=0, help="with --quick: PFASST iterations per step (default: workload's)")
    ap.add_argument("--vcycles", type=int, default=-1, help="override V-cycles per sub-step (0 = solve to 1e-12)")
    ap.add_argument("--precision", type=int, default=-1, help="override precision: 0 FP64, 1 mixed")
    ap.add_argument("--order4-only", default="", help="order4: comma-separated subset of 2/2,2/4,4/4")
    ap.add_argument("--coarse-vcycles", type=int, default=-1,
                    help="measured variant: V-cycles per coarse-level sub-step (-1: the workload's)")
    ap.add_argument("--vcycle-tail", type=int, default=-1,
                    help="1 = run the levels of a single-grid V-cycle that fit one CTA in one launch, 0 = per level "
                         "(-1: the library default)")
    ap.add_argument("--tma", type=int, nargs="?", const=3, default=0, choices=(0, 2, 3),
                    help="pin the TMA-staged sweep on every level that can run it (profiling runs): "
                         "2 = two x points per thread, 3 (bare flag) = four")
    ap.add_argument("--pin-tuning", default="",
                    help="pin the smoother variants ('level:narrow:variant:param:threads ...', the tuning_codes "
                         "of an earlier bench line), e.g. for an ncu run whose own autotuning ncu distorts")
    ap.add_argument("--profile-all", action="store_true",
                    help="time every launch (not only fine-grid ones) and print the breakdown to stderr")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "uneven":
        run_uneven(args)
    elif args.workload == "learned-train":
        run_learned(args)
    elif args.workload == "learned":
        run_learned_deploy(args)
    elif args.workload == "compare":
        run_compare(args)
    elif args.workload == "weak3":
        run_weak3(args)
    elif args.workload == "order4":
        run_order4(args)
    elif args.workload == "heat1d":
        run_heat1d(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
