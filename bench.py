"""Benchmark of the TWA trajectory planner on one GB300.

Headline: factor updates per second of one full TWA iteration (every
collision, kinetic, position and wall factor, then the consensus and dual
updates) on the p=1024, eta=16 random square with 4 walls: 8,380,416
collision + 16,384 kinetic + 65,536 wall + 2,048 position factors per
iteration.  A step is one iteration; every factor's minimizer plus its edge
updates counts as one update.  Also reported: the dense-state mode (every u
record streamed) against the HBM roofline, time to converge, the end-to-end
call with host buffers, and the FP64 oracle on the host.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank plans its own replica of the workload
(there is no exchange between instances); value is the sum over ranks.
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads  # noqa: E402

METRIC = "factor-updates/s and time-to-converge (1 GB300) vs FP64 CPU oracle; % HBM roofline"
UNIT = "factor-updates/s"

# DRAM traffic per launch (dram__bytes_read.sum + dram__bytes_write.sum) of
# the current pass-1 kernels on square1024_eta16 (gated: two launches of one
# capture, profiles/test_rows_kernel_square1024.md; dense: one single-pass
# capture of two launches, profiles/test_kernel_traffic_square1024.md).
TRAFFIC_SQUARE1024 = {"gated": 10.49e6, "dense": 486.32e6}
# Warp instructions executed per launch of the gated pass-1 kernel on
# square1024_eta16 (smsp__inst_executed.sum of a two-launch capture,
# profiles/test_rows_kernel_square1024.md): the work the issue-rate
# roofline divides by the kernel time.
WARP_INST_SQUARE1024 = {"gated": 7.017e6}


def factor_counts(inst):
    p, eta = inst.p, inst.eta
    return dict(coll=eta * p * (p - 1) // 2, kin=eta * p, wall=inst.n_walls * eta * p, pos=2 * p)


def dense_coll_bytes(inst):
    """Algorithmic HBM bytes of the collision test pass under the dense state
    model: per collision factor its 8-float u record read and written (64 B)
    plus 2 bits of activity (read and written)."""
    c = factor_counts(inst)
    return c["coll"] * 64 + c["coll"] * 2 / 8


def dense_bytes_per_iter(inst):
    """... plus per kinetic or wall factor a 4-float u read and written."""
    c = factor_counts(inst)
    return dense_coll_bytes(inst) + (c["kin"] + c["wall"]) * 32


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), float(d.get("sm_max_mhz", 2070.0)), "measured"
    except Exception:
        return 6800.0, 2070.0, "fallback"


def sm_count():
    import torch
    return int(torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count)


def issue_peak_g(sm_mhz):
    """Warp-instruction issue peak: SMs x 4 schedulers x one warp instruction
    per cycle each x SM clock, in G warp instructions per second."""
    return sm_count() * 4 * sm_mhz * 1e6 / 1e9


def host_cpu():
    """The host's logical core count and CPU model (lscpu / /proc/cpuinfo)."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if model is None:
        try:
            for line in open("/proc/cpuinfo"):
                if line.lower().startswith(("model name", "cpu part")):
                    model = line.split(":", 1)[1].strip()
                    break
        except Exception:
            pass
    return os.cpu_count() or 1, model or "unknown"


class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self, index):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(index), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.flush()
        self.f.seek(0)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f.read().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.f.name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": sorted(reasons),
                "samples": len(sm)}


def aggregate(ms_local, units_local, world, dist=None, device=None):
    """Whole-job numbers across ranks: the step time is the slowest rank's,
    the units are summed.  Returns (ms_per_step, total_units)."""
    if world == 1 or dist is None:
        return ms_local, units_local
    import torch
    t = torch.tensor([ms_local, units_local], dtype=torch.float64, device=device)
    mx = t.clone()
    dist.all_reduce(mx, op=dist.ReduceOp.MAX)
    sm = t.clone()
    dist.all_reduce(sm, op=dist.ReduceOp.SUM)
    return float(mx[0].item()), float(sm[1].item())


def _oracle_worker(args):
    """One process: the FP64 oracle, as it stands, on whole iterations of a
    named workload from its iterate `first`, for about budget_s seconds.
    Returns (iterations, seconds, active pairs of the timed iterations)."""
    name, first, budget_s = args
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    sys.path.insert(0, ROOT)
    import workloads as wl
    from oracle import twa
    inst = wl.by_name(name)
    prob = twa.Problem.from_instance(inst)
    st = twa.initial_state(prob)
    for _ in range(first):
        st, _ = twa.iterate(prob, st)
    n, act, t0 = 0, [], time.perf_counter()
    while True:
        st, info = twa.iterate(prob, st)
        n += 1
        act.append(int(info.active_coll.sum()))
        if time.perf_counter() - t0 >= budget_s:
            break
    return n, time.perf_counter() - t0, act


def cpu_baseline(inst, budget_s=20.0):
    """The FP64 oracle, as it stands, on this host: whole iterations of the
    same workload from its iterate 2 (an iteration's cost hardly depends on
    the iterate: the p(p-1)/2 x eta distance tests dominate it), first in one
    process, then in one process per host core at once (the oracle is
    single-threaded numpy, so all cores means that many oracle instances)."""
    import multiprocessing as mp
    from oracle import twa
    total = sum(factor_counts(inst).values())
    ncpu, model = host_cpu()
    n, dt, act = _oracle_worker((inst.name, 2, budget_s))
    out = {"value": total * n / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
           "cpu": model, "host_cores": ncpu,
           "sample": f"{n} full oracle iteration(s) of {inst.name} (iterations 3..{n + 2}), "
                     f"{dt:.1f} s, numpy FP64 single thread; active pairs "
                     f"{min(act)}..{max(act)}"}
    # all cores: one oracle process per core, spawned (this process holds a CUDA context)
    try:
        ctx = mp.get_context("spawn")
        with ctx.Pool(ncpu) as pool:
            res = pool.map(_oracle_worker, [(inst.name, 2, budget_s)] * ncpu)
        its = sum(r[0] for r in res)
        span = max(r[1] for r in res)
        out["all_cores"] = {"value": total * its / span, "unit": UNIT, "cores": ncpu,
                            "sample": f"{ncpu} oracle processes at once, {its} iterations in "
                                      f"{span:.1f} s (iterations 3.. of {inst.name} each)"}
    except Exception as e:  # memory or process limits of the host
        out["all_cores"] = {"unavailable": f"{type(e).__name__}: {e}"}
    # the oracle's own solve of the CPU-sized circle swap (time to converge)
    small = workloads.circle4()
    t0 = time.perf_counter()
    _, it, _ = twa.solve(twa.Problem.from_instance(small), small.tol, small.max_iter)
    out["time_to_converge_circle4_eta4"] = {"oracle_ms": 1e3 * (time.perf_counter() - t0),
                                            "iterations": it}
    return out


def run_reference(args, inst):
    """--impl reference: the FP64 oracle on the host cores, bounded."""
    if int(os.environ.get("RANK", "0")) != 0:
        return
    from oracle import twa
    prob = twa.Problem.from_instance(inst)
    st = twa.initial_state(prob)
    total = sum(factor_counts(inst).values())
    st, _ = twa.iterate(prob, st)  # one untimed warm-up iteration
    budget = 150.0
    times = []
    t_all = time.perf_counter()
    for _ in range(args.steps):
        t0 = time.perf_counter()
        st, _ = twa.iterate(prob, st)
        times.append(time.perf_counter() - t0)
        if time.perf_counter() - t_all > budget:
            break
    n = len(times)
    ms = 1e3 * sum(times) / n
    value = total / (ms / 1e3)
    ncpu, model = host_cpu()
    sample = (f"{n} of {args.steps} requested iterations of {inst.name} (capped at {budget:.0f} s) "
              f"after 1 untimed warm-up iteration; numpy FP64, single thread of {ncpu} ({model})")
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": n,
            "warmup": 1, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": inst.name, "p": inst.p, "eta": inst.eta,
                       "walls": inst.n_walls, "factors_per_step": total},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(_finite(line), allow_nan=False), flush=True)


def timed_iterations(pl, stream, steps, flush):
    """Each iteration timed alone with CUDA events on the planner's stream,
    L2 flushed (256 MB write) before it.  Returns ms per iteration."""
    import torch
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)]
    for k in range(steps):
        flush.fill_(float(k))
        ev[k][0].record(stream)
        pl.iterate(1)
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    return sum(a.elapsed_time(b) for a, b in ev) / steps


def by_iterate(pk, inst, flush, stream, points=(20, 1000, 10000, 100000), steps=10):
    """The same timed iteration (L2 flushed before each, CUDA events) at
    several points of one solve: the benchmark's iteration-20 state is the
    crowded start, where the last segment still spans each agent's whole
    path; later iterates are nearer the converged plan."""
    import torch
    out = {}
    with pk.Planner.from_instance(inst) as pl:
        done = 0
        for k in points:
            pl.iterate(k - done)
            done = k
            ms = timed_iterations(pl, stream, steps, flush)
            done += steps
            out[str(k)] = {"ms_per_step": ms, "active_coll": pl.info()["active_coll"]}
    return out


def kernel_times(pl, stream, steps, flush):
    """Average per-kernel ms over `steps` iterations (events inside the
    library, on the streams the kernels run on), L2 flushed before each."""
    import torch
    pl.profile_start()
    for k in range(steps):
        flush.fill_(float(k))
        pl.iterate(1)
    torch.cuda.synchronize()
    return pl.profile_stop()


def _plan_quality(pk, inst, pl):
    """Total kinetic cost (Eq. velo_cost_pair_wise) and the smallest pair and
    wall clearance ratios of the planner's current trajectory, from the FP64
    device check (plan_check)."""
    c = pl.check()
    return c["total_cost"], c["min_pair_clearance"], c["min_wall_clearance"]


def _solve_timed(pl):
    import torch
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    conv, it, res = pl.solve()
    torch.cuda.synchronize()
    return conv, it, res, 1e3 * (time.perf_counter() - t0)


# iteration caps and residual-check intervals of the time-to-converge runs:
# the p = 100 circle needs about 154,000 iterations, the p = 1024 square
# about 830,000
CONVERGE = {"circle4_eta4": (20000, 10), "circle100_eta8": (300000, 1000),
            "square1024_eta16": (1200000, 10000)}


def time_to_converge(pk, names):
    """plan_solve to the workload's tolerance (or its iteration cap) on the
    GPU, with the plan's cost and clearances from the FP64 device check; the
    p = 100 circle also with the rho warm-up of Section 4 (rho = eta p 1e-5
    for 20 iterations, then 1)."""
    out = {}
    runs = [(name, name, {}) for name in names]
    if "circle100_eta8" in names:
        inst = workloads.by_name("circle100_eta8")
        runs.append(("circle100_eta8_warmup", "circle100_eta8",
                     dict(rho0=1.0, warm_iters=20, warm_rho=inst.eta * inst.p * 1e-5)))
    for key, name, kw in runs:
        inst = workloads.by_name(name)
        cap, every = CONVERGE.get(name, (inst.max_iter, 10))
        with pk.Planner.from_instance(inst, max_iter=cap, check_every=every, **kw) as pl:
            conv, it, res, ms = _solve_timed(pl)
            chk = pl.check()
        out[key] = {"converged": conv, "iterations": it, "residual": res, "tol": inst.tol,
                    "check_every": every, "gpu_ms": ms, "total_cost": chk["total_cost"],
                    "min_clearance_ratio": chk["min_pair_clearance"],
                    "min_wall_clearance_ratio": chk["min_wall_clearance"],
                    "max_endpoint_error": chk["max_endpoint_error"],
                    "feasible": chk["min_pair_clearance"] >= 1 - 1e-4
                    and chk["min_wall_clearance"] >= 1 - 1e-4 and chk["max_endpoint_error"] <= 1e-6,
                    "factor_updates_per_s": sum(factor_counts(inst).values()) * it / (ms / 1e3)}
        if kw:
            out[key]["rho"] = kw
    return out


def modes(pk):
    """Rows f3 / f4 beside the plain solver on the same GPU: standard ADMM
    against TWA (Fig. 2-left's comparison), the feasibility problem against
    the energy problem (Section 4), a maximum-velocity limit, and recovery of
    a collision-free plan from an energy solve stopped early."""
    out = {}
    caps = {"circle4_eta4": (20000, 10), "circle100_eta8": (2000000, 5000)}
    for name in ("circle4_eta4", "circle100_eta8"):
        inst = workloads.by_name(name)
        cap, every = caps[name]
        rec = {}
        for label, kw in (("twa", {}), ("admm", {"flags": pk.PLAN_ADMM}),
                          ("feasibility", {"energy": False})):
            kw = dict(kw, max_iter=cap, check_every=every if label != "feasibility" else 10)
            with pk.Planner.from_instance(inst, **kw) as pl:
                conv, it, res, ms = _solve_timed(pl)
                cost, coll, _ = _plan_quality(pk, inst, pl)
            rec[label] = {"converged": conv, "iterations": it, "check_every": kw["check_every"],
                          "gpu_ms": ms, "total_cost": cost, "min_clearance_ratio": coll}
        if rec["twa"]["converged"] and rec["admm"]["converged"]:
            rec["admm_over_twa_iterations"] = rec["admm"]["iterations"] / rec["twa"]["iterations"]
        out[name] = rec
    inst = workloads.circle4()
    with pk.Planner.from_instance(inst, check_every=10, vmax=0.56) as pl:
        conv, it, res, ms = _solve_timed(pl)
        z = pl.trajectory().double()
        vmax_seen = float((z[:, 1:] - z[:, :-1]).norm(dim=-1).max())
        cost, coll, _ = _plan_quality(pk, inst, pl)
    out["circle4_vmax0.56"] = {"converged": conv, "iterations": it, "gpu_ms": ms,
                               "longest_segment": vmax_seen, "total_cost": cost,
                               "min_clearance_ratio": coll}
    inst = workloads.small_square(48, 8, 2)
    with pk.Planner.from_instance(inst, check_every=1) as pl:
        pl.iterate(300)
        _, before, _ = _plan_quality(pk, inst, pl)
        pl.set_energy(False)
        conv, it, res, ms = _solve_timed(pl)
        _, after, wall = _plan_quality(pk, inst, pl)
    out["recovery_square48"] = {"energy_iterations": 300, "clearance_before": before,
                                "feasibility_iterations": it - 300, "converged": conv,
                                "gpu_ms": ms, "clearance_after": after,
                                "wall_clearance_after": wall}
    return out


def local_planner(pk, p=32, epochs=150, step=0.1, advance=0.5):
    """Section 5's velocity-obstacle planner on a circle swap (CONF1) with
    the paper's symmetry breaking C_i = 1 + 0.001 i: per-epoch solve time and
    iterations until every agent is within 1e-3 of its destination."""
    import torch
    inst = workloads.circle_swap(p, 2, 0.05, 0.005, workloads.SEED_BASE + 5, name=f"vo_circle{p}")
    c = 1 + 0.001 * np.arange(p)
    # rho0 = 30 C' and dual step 0.5: every epoch converges (a sweep of rho0
    # in {10, 30, 100}, step in {0.05, 0.1}, alpha in {0.1, 0.5} on this swap)
    pl = pk.Planner.velocity_obstacle(inst.start, inst.goal, inst.radius, c, step, rho0=30.0,
                                      alpha=0.5, tol=1e-5, max_iter=8000, check_every=5)
    ms, its, conv_all = [], [], True
    md = float("inf")
    for e in range(epochs):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        conv, it, r, md = pl.vo_epoch(advance)
        ms.append(1e3 * (time.perf_counter() - t0))
        its.append(it)
        conv_all &= conv
        if md < 1e-3:
            break
    pl.close()
    q = lambda a, f: float(np.percentile(a, f))
    return {"workload": f"{inst.name}: p={p} circle swap, r=0.05, step {step}, advance {advance}",
            "epochs": len(ms), "arrived": md < 1e-3, "all_epochs_converged": conv_all,
            "epoch_ms": {"median": q(ms, 50), "p90": q(ms, 90), "max": max(ms)},
            "epoch_iterations": {"median": q(its, 50), "p90": q(its, 90), "max": max(its)}}


def batching(pk, n=512, tol_rel=1e-4, max_iter=20000, check_every=100):
    """Row f1: n uneven instances (p ~ U{8..256}, eta in {4, 8, 16}, circle
    swap or random square 50/50) solved as one batch (one launch per pass,
    CUDA graphs, autotuned launch shapes) against looping the plain solver
    over the same instances.  Equal accuracy: every member stops, in both
    arms, at the first residual check below tol_rel x its layout scale (or
    at max_iter), so both arms run each member for the same iterations."""
    import torch
    insts = workloads.batch_instances(n)
    for m in insts:
        L = max(1.0, float(np.abs(m.start).max()), float(np.abs(m.goal).max()))
        m.tol = tol_rel * L
        m.max_iter = max_iter
    factors = [sum(factor_counts(m).values()) for m in insts]
    # the autotuner's timing iterations are real iterations, so it tunes on a
    # throwaway batch of the same instances; the timed solve starts afresh
    with pk.PlannerBatch(insts, check_every=check_every) as B:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        choice = B.autotune(8)
        torch.cuda.synchronize()
        t_tune = time.perf_counter() - t0
    with pk.PlannerBatch(insts, check_every=check_every) as B:
        B.set_shape(**choice)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        its, res, nconv = B.solve()
        torch.cuda.synchronize()
        t_batch = time.perf_counter() - t0
    # the same instances, one plain planner at a time
    t_loop = 0.0
    its_loop, conv_loop = [], 0
    for m in insts:
        with pk.Planner.from_instance(m, check_every=check_every) as pl:
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            conv, it, r = pl.solve()
            torch.cuda.synchronize()
            t_loop += time.perf_counter() - t0
            its_loop.append(it)
            conv_loop += int(conv)
    upd = float(sum(f * i for f, i in zip(factors, its)))
    return {"workload": f"batch{n}: p ~ U{{8..256}}, eta in {{4,8,16}}, circle/square 50/50",
            "members": n, "tol": f"{tol_rel:g} x layout scale", "max_iter": max_iter,
            "check_every": check_every, "converged": nconv, "converged_loop": conv_loop,
            "iterations_total": int(sum(its)),
            "iterations_median": float(np.median(its)),
            "same_iterations_as_loop": its == its_loop,
            "batch_s": t_batch, "loop_s": t_loop, "speedup_vs_loop": t_loop / t_batch,
            "batch_factor_updates_per_s": upd / t_batch, "loop_factor_updates_per_s": upd / t_loop,
            "autotuned": choice, "autotune_s": t_tune}


def differentiation(pk, K=2000, reps=3):
    """Row f2: gradient of loss(z^K) = final kinetic energy + 10 x squared
    collision slack with respect to starts, goals, radii and cost weights
    through K unrolled iterations on the p = 256 circle swap (eta = 8,
    r = 0.02), against the plain solver running the same K iterations.  The
    forward keeps ceil(sqrt(K)) checkpoints; the backward replays each
    segment and runs the adjoint kernels.  Times are CUDA events on the
    planner's stream, best of reps."""
    import torch
    from paper_1311_4527_gb300 import losses
    inst = workloads.circle256()
    dev = torch.device("cuda")
    radius = torch.tensor(inst.radius, dtype=torch.float32, device=dev)
    cost = torch.tensor(inst.cost_w, dtype=torch.float32, device=dev)
    pl = pk.Planner.from_instance(inst)

    def timed(f):
        best = float("inf")
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            a.record()
            f()
            b.record()
            torch.cuda.synchronize()
            best = min(best, a.elapsed_time(b))
        return best

    t_plain = timed(lambda: (pl.reset(), pl.iterate(K)))
    t_unroll = timed(lambda: pl.unroll(K))
    z = pl.trajectory().requires_grad_(True)
    loss = losses.plan_loss(z, radius, cost)
    dz, = torch.autograd.grad(loss, z)
    t_back = timed(lambda: pl.backward(dz))
    gs, gg, gr, gc = pl.backward(dz)
    torch.cuda.synchronize()
    # translation equivariance: the position gradients sum to sum(dL/dz)
    resid = (gs.double().sum(0) + gg.double().sum(0) - dz.double().reshape(-1, 2).sum(0)).abs().max()
    pl.close()
    return {"workload": f"circle256_eta8: p=256 circle swap, r=0.02, eta=8, K={K} unrolled FP32 "
                        "iterations, loss = kinetic energy + 10 x squared collision slack",
            "checkpoint_every": int(math.ceil(math.sqrt(K))), "loss": float(loss.detach()),
            "plain_forward_ms": t_plain, "unroll_ms": t_unroll, "backward_ms": t_back,
            "forward_plus_backward_ms": t_unroll + t_back,
            "cost_vs_plain_forward": (t_unroll + t_back) / t_plain,
            "grad_norms": {"start": float(gs.norm()), "goal": float(gg.norm()),
                           "radius": float(gr.norm()), "cost": float(gc.norm())},
            "translation_identity_residual": float(resid) / max(float(dz.abs().sum()), 1e-30)}


def _finite(obj):
    """Non-finite floats (an unmeasured clearance, a residual that never
    came) as null, so that the line is strict JSON."""
    if isinstance(obj, float):
        return obj if math.isfinite(obj) else None
    if isinstance(obj, dict):
        return {k: _finite(v) for k, v in obj.items()}
    if isinstance(obj, (list, tuple)):
        return [_finite(v) for v in obj]
    return obj


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--mode", default="gated", choices=["gated", "dense"],
                    help="state mode of the headline measurement")
    ap.add_argument("--workload", default="square1024_eta16",
                    help="a named workload, or 'square' for a random square of --p agents")
    ap.add_argument("--p", type=int, default=768)
    ap.add_argument("--eta", type=int, default=16)
    ap.add_argument("--seed", type=int, default=7)
    ap.add_argument("--start-iter", type=int, default=20,
                    help="untimed iterations before warm-up (a mid-solve iterate)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--quick", action="store_true",
                    help="headline only: no dense companion, convergence or e2e legs")
    args = ap.parse_args()
    if args.workload == "square":
        inst = workloads.small_square(args.p, args.eta, seed=args.seed)
    else:
        inst = workloads.by_name(args.workload)
    if args.impl == "reference":
        return run_reference(args, inst)

    import torch
    import torch.distributed as dist
    import paper_1311_4527_gb300 as pk

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    warmup = max(3, args.warmup)
    hbm_peak, sm_max, peak_kind = peaks()
    c = factor_counts(inst)
    total = sum(c.values())
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def prepared(flags):
        pl = pk.Planner.from_instance(inst, flags=flags)
        pl.iterate(args.start_iter)
        for _ in range(warmup):
            pl.iterate(1)
        torch.cuda.synchronize()
        return pl

    head_flags = pk.PLAN_DENSE_STATE if args.mode == "dense" else 0
    pl = prepared(head_flags)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = Clocks(local)
    time.sleep(0.3)
    wall0 = time.perf_counter()
    ms_local = timed_iterations(pl, stream, args.steps, flush)
    wall = time.perf_counter() - wall0
    clk = clocks.stop()
    ms_step, units = aggregate(ms_local, total, world, dist if world > 1 else None, dev)
    if world > 1:
        dist.barrier()
    value = units / (ms_step / 1e3)
    kt = kernel_times(pl, stream, min(args.steps, 20), flush)
    info = pl.info()
    pl.close()

    def roofline_for(mode, ktimes):
        if mode == "dense":
            b = dense_coll_bytes(inst)
            t = ktimes["test"] / 1e3
            ach = b / t / 1e9
            traffic = TRAFFIC_SQUARE1024["dense"] if inst.name == "square1024_eta16" else None
            return {"bound": "hbm", "kernel": "test_kernel<dense> (with the kinetic and wall blocks)",
                    "achieved": ach,
                    "peak": hbm_peak, "unit": "GB/s", "frac": ach / hbm_peak, "traffic": traffic,
                    "peak_kind": f"{peak_kind} (copy bandwidth)",
                    "note": f"algorithmic bytes {b:.4g} per launch (64 B u record read+written "
                            f"and 2 bits per collision factor) / live kernel time "
                            f"{ktimes['test'] * 1e3:.1f} us"}
        # gated state: the bounding-circle filter leaves no per-factor bytes or
        # flops to speak of; the kernel is bound by warp-instruction issue
        t = ktimes["test"] / 1e3
        winst = WARP_INST_SQUARE1024["gated"] if inst.name == "square1024_eta16" else None
        pk_i = issue_peak_g(sm_max)
        ach = winst / t / 1e9 if winst else None
        own = TRAFFIC_SQUARE1024["gated"] if inst.name == "square1024_eta16" else None
        return {"bound": "issue", "kernel": "test_rows_kernel (gated; with the kinetic and wall blocks)",
                "achieved": ach, "peak": pk_i, "unit": "G warp-instructions/s",
                "frac": ach / pk_i if ach else None, "traffic": own,
                "peak_kind": f"derived: {sm_count()} SMs x 4 schedulers x 1 warp instruction/cycle "
                             f"x {sm_max:.0f} MHz",
                "note": f"{winst:.4g} warp instructions per launch (ncu) / live kernel time "
                        f"{ktimes['test'] * 1e3:.1f} us" if winst else "no instruction count for "
                        "this workload",
                "hbm_own_bytes_frac": (own / t / 1e9) / hbm_peak if own else None}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": inst.name, "p": inst.p, "eta": inst.eta, "walls": inst.n_walls,
                   "factors_per_step": total, "coll_factors": c["coll"], "kin_factors": c["kin"],
                   "wall_factors": c["wall"], "pos_factors": c["pos"], "mode": args.mode,
                   "parallelism": f"replicas{world}",
                   "l2": "flushed (256 MB write) before every timed iteration",
                   "start_iter": args.start_iter,
                   "active_coll_last": info["active_coll"], "active_wall_last": info["active_wall"]},
        "coll_factor_updates_per_s": c["coll"] * world / (ms_step / 1e3),
        "kernel_ms": kt,
        "wall_s": wall,
        "clocks": clk,
        "gpu_launches": 3 * args.steps,
        "roofline": roofline_for(args.mode, kt),
    }
    if not args.quick:
        # the other state mode, same workload, same timing rules
        other = "gated" if args.mode == "dense" else "dense"
        pl = prepared(pk.PLAN_DENSE_STATE if other == "dense" else 0)
        ms_o = timed_iterations(pl, stream, args.steps, flush)
        kt_o = kernel_times(pl, stream, min(args.steps, 20), flush)
        pl.close()
        ms_o, units_o = aggregate(ms_o, total, world, dist if world > 1 else None, dev)
        b = dense_bytes_per_iter(inst)
        line[other] = {"ms_per_step": ms_o, "value": units_o / (ms_o / 1e3), "kernel_ms": kt_o,
                       "roofline": roofline_for(other, kt_o),
                       "iteration_hbm_frac": (b / (ms_o / 1e3) / 1e9) / hbm_peak
                       if other == "dense" else None}
        # the other state mode's roofline, visible beside the headline's
        line["roofline"]["companion"] = dict(line[other]["roofline"], mode=other,
                                             iteration_hbm_frac=line[other]["iteration_hbm_frac"])

        # end to end through the C ABI with host buffers: new endpoints in,
        # one iteration, the trajectory back to pinned host memory
        pl = prepared(head_flags)
        # 200 steps of about 0.06 ms: the loop's timer resolution and a
        # stray host hiccup stay small against the total
        e2e_steps = 200
        # a control loop's buffers: pinned host memory, refilled in place
        # each step, held as numpy views
        start_h = torch.from_numpy(inst.start.astype(np.float32)).pin_memory().numpy()
        goal_h = torch.from_numpy(inst.goal.astype(np.float32)).pin_memory().numpy()
        z_h = torch.empty((inst.p, inst.eta + 1, 2), dtype=torch.float32).pin_memory().numpy()
        def e2e_loop(wait):
            # new endpoints in (checked on the device; with wait=False the
            # check's verdict is read by the trajectory readback), one
            # iteration, the trajectory back
            for _ in range(5):  # untimed: the first call builds the endpoint update's graph
                pl.set_endpoints(start_h, goal_h, wait=wait)
                pl.iterate(1)
                pl.trajectory_host(z_h)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for _ in range(e2e_steps):
                pl.set_endpoints(start_h, goal_h, wait=wait)
                pl.iterate(1)
                pl.trajectory_host(z_h)
            torch.cuda.synchronize()
            return 1e3 * (time.perf_counter() - t0) / e2e_steps

        e2e_sync_ms = e2e_loop(True)
        e2e_ms = e2e_loop(False)
        pl.close()
        e2e_ms, units_e = aggregate(e2e_ms, total, world, dist if world > 1 else None, dev)
        line["e2e"] = {"value": units_e / (e2e_ms / 1e3), "unit": UNIT,
                       "h2d_bytes_per_step": int(2 * inst.p * 2 * 4),
                       "d2h_bytes_per_step": int(inst.p * (inst.eta + 1) * 2 * 4),
                       "ms_per_step": e2e_ms,
                       "path": "plan_set_endpoints_async(host; the device check's verdict is read "
                               "at the readback) + plan_iterate(1) + plan_get_trajectory(host), "
                               "pinned buffers",
                       "ms_per_step_waiting_check": e2e_sync_ms}
    if rank == 0 and world == 1 and not args.quick:
        line["by_iterate"] = by_iterate(pk, inst, flush, stream)
        line["batching"] = batching(pk)
        line["differentiation"] = differentiation(pk)
        line["time_to_converge"] = time_to_converge(
            pk, ["circle4_eta4", "circle100_eta8", "square1024_eta16"])
        line["modes"] = modes(pk)
        line["local_planner"] = local_planner(pk)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(inst)
    if rank == 0:
        print(json.dumps(_finite(line), allow_nan=False), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
