"""Benchmark of the TMM year map (Metos3D, arXiv:1410.0204, Sections 3-4) on GB300.

One benchmark step = one model year: the year map phi over 2880 TMM steps on the
128 x 64 x 15 synthetic grid (52749 wet cells in 4448 columns, the size of the paper's
2.8125 degree runs), PO4-DOP model (2 tracers), FP64, inputs resident in HBM.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the CPU oracle (the FP64 C statement of the method the GPU path is
checked against) on the host cores instead.  For N > 1 (torchrun) every rank runs its own
replica of the year map (the method does not shard on one problem here; replicas only).
Rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import m3d_inputs as mi  # noqa: E402

WORKLOAD = "ndop_128x64x15"
METRIC = "model years/s & HBM roofline % of year map"
UNIT = "model years/s"


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    hbm, src = 6800.0, "fallback"
    try:
        with open(path) as f:
            d = json.load(f)
        hbm, src = float(d["hbm_gbs"]), "measured"
    except Exception:
        pass
    return hbm, src


# DRAM bytes (read + write) per launch of the year kernel on this workload, from ncu (see
# profiles/), with how they were obtained; None where no capture of the current kernel exists.
# Keys: (plan, tridiagonal implicit form, per-step explicit operators, kernel revision).
# The revision names the year kernel's code the capture was taken of; a changed kernel
# gets a new revision and no traffic until it is captured again.
# The counters are taken on the 64x32x8 grid (3.12 GB of step operators on the device):
# 3.126244 GB read + 4.13 MB written per launch, 1.0049x its step-operator bytes
# (3,115,008,000). The traffic is the step operators read once plus a few tens of MB, so
# it grows with the step-operator bytes, and is scaled to this workload's
# 16,793,763,840 by that ratio.
YEAR_KERNEL_REVISION = "per-warp-release"
TRAFFIC_PER_LAUNCH = {
    ("resident", True, True, "per-warp-release"): (
        round(16793763840 * (3126244000 + 4127744) / 3115008000),
        "ncu dram__bytes_read.sum + dram__bytes_write.sum of one launch on the 64x32x8 grid, "
        "scaled by the step-operator bytes (16.79 GB here vs 3.12 GB there)"),
}

# FP64 peak of the GPU per SM clock: ncu's sm__sass_thread_inst_executed_op_dfma_pred_on.sum.peak_sustained
# on GB300 is 304 thread-level DFMA per cycle (2 per SM), i.e. 608 FP64 flops per cycle.
FP64_FLOPS_PER_CLOCK = 304 * 2
# Nominal: the same at the maximum SM clock, 2.07 GHz (used where no clock was sampled).
FP64_PEAK_TFLOPS = FP64_FLOPS_PER_CLOCK * 2.07e9 / 1e12


def fp64_peak_tflops(sm_mhz):
    """FP64 peak at the SM clock sampled during the timed region (nominal clock if none)."""
    if not sm_mhz:
        return FP64_PEAK_TFLOPS, "ncu dfma peak_sustained (304/clk) x nominal 2070 MHz"
    return FP64_FLOPS_PER_CLOCK * float(sm_mhz) * 1e6 / 1e12, \
        "ncu dfma peak_sustained (304/clk) x sampled median SM clock %.0f MHz" % float(sm_mhz)


# FP64 flops per cell of the source terms, per member: (euphotic cell, aphotic cell).  A division
# counts as one flop here (the algorithmic count, not the instruction cost).
Q_FLOPS = {1: (12, 2), 2: (18, 6), 3: (30, 10), 5: (40, 30)}


def ensemble_flops_per_step(prob, members, executed=False):
    """FP64 flops of one ensemble step.  Algorithmic (the method's count): per explicit entry
    and per dense implicit block entry one FMA to interpolate and one per tracer, 2 + 2 W;
    the source terms per member and cell; the increment added to each tracer (2 W per cell).
    executed=True: what the kernel does, the implicit part as the Thomas solves of both months
    and their blend per cell and tracer (13 W) instead of the dense blocks."""
    W = sum(m.ntracer for m in members)
    L = prob.nlayer
    n_eu = int(np.minimum(L, 2).sum())
    q = sum(Q_FLOPS[m.ntracer][0] * n_eu + Q_FLOPS[m.ntracer][1] * (prob.n - n_eu) for m in members)
    implicit = 13 * prob.n * W if executed else prob.s_imp * (2 + 2 * W)
    return prob.nnz * (2 + 2 * W) + implicit + q + 2 * prob.n * W


def method_per_step(prob, ntr=2):
    """Algorithmic bytes and FP64 flops of one TMM step as the method states it, whatever form
    a kernel applies.  Bytes: the explicit values of two months and their column index per
    entry (2 x 8 + 4), the row pointers, the dense implicit blocks of two months (2 x 8 per
    block entry), the state read and written.  Flops: per explicit entry and per block entry
    one FMA to interpolate the months and one per tracer (2 + 2 ntr), and about 50 per
    euphotic cell and tracer for the source term."""
    n_eu = int(np.minimum(prob.nlayer, 2).sum())
    bytes_ = prob.nnz * (2 * 8 + 4) + 4 * (prob.n + 1) + prob.s_imp * 2 * 8 + ntr * prob.n * (8 + 8)
    flops = (prob.nnz + prob.s_imp) * (2 + 2 * ntr) + 50 * n_eu * ntr
    return bytes_, flops


def run_ensemble(prob, t_single_ndop, flush):
    """The batched 64-member ensemble (16 N, 32 N-DOP, 16 NPZD-DOP) against the same members
    run one at a time: N-DOP members by the single-context year map, N and NPZD-DOP members
    (which only ensembles run) as one-member ensembles."""
    import torch
    import paper_1410_0204_gb300 as m3d
    members = mi.make_ensemble()
    ens = m3d.Ensemble.from_problem(prob, members)
    Y0 = torch.from_numpy(np.vstack([mi.initial_state(prob, m.ntracer, mi.model_initial_values(m.model))
                                     for m in members])).cuda()
    Y1 = torch.empty_like(Y0)
    cpb, nw, ms_tune = ens.autotune(Y0, nsteps=20)

    def year_time(e, Y, Yo, reps):
        e.year_map(Y, Yo)
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            flush.fill_(1.0)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record()
            e.year_map(Y, Yo)
            b.record()
            b.synchronize()
            ts.append(a.elapsed_time(b) / 1e3)
        return sum(ts) / len(ts)

    t_ens = year_time(ens, Y0, Y1, 3)
    launches = ens.last_launch_count()
    ens.close()
    singles = {}
    for model in (mi.MODEL_N, mi.MODEL_NPZD):
        one = m3d.Ensemble.from_problem(prob, [mi.Member(model, mi.default_params(model))])
        y = torch.from_numpy(mi.initial_state(prob, one.width, mi.model_initial_values(model))).cuda()
        one.autotune(y, nsteps=10)
        singles[model] = year_time(one, y, torch.empty_like(y), 2)
        one.close()
    counts = {}
    for m in members:
        counts[m.model] = counts.get(m.model, 0) + 1
    t_seq = counts[mi.MODEL_N] * singles[mi.MODEL_N] + counts[mi.MODEL_NDOP] * t_single_ndop + \
        counts[mi.MODEL_NPZD] * singles[mi.MODEL_NPZD]
    flops = ensemble_flops_per_step(prob, members) * prob.nstep
    flops_x = ensemble_flops_per_step(prob, members, executed=True) * prob.nstep
    W = sum(m.ntracer for m in members)
    return {
        "workload": "64 members on %s: 16 N (1 tracer), 32 N-DOP (2), 16 NPZD-DOP (5), parameters within "
                    "+-50%% of the defaults; W = %d tracers in 5 lane groups" % (WORKLOAD, W),
        "member_years_per_s": len(members) / t_ens, "seconds_per_ensemble_year": t_ens,
        "cell_tracer_steps_per_s": prob.n * W * prob.nstep / t_ens,
        "tiling": {"cols_per_block": cpb, "warps_per_block": nw, "autotune_ms_per_step": ms_tune},
        "launches_per_year": launches,
        "roofline": {"bound": "alu", "achieved": flops / t_ens / 1e12, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                     "frac": flops / t_ens / 1e12 / FP64_PEAK_TFLOPS, "kernel": "k_ens_step (one launch per TMM step)",
                     "executed": {"achieved": flops_x / t_ens / 1e12, "frac": flops_x / t_ens / 1e12 / FP64_PEAK_TFLOPS,
                                  "implicit_form": "tridiagonal"}},
        "sequential_single_instance": {
            "seconds": t_seq, "n_years_per_s": 1.0 / singles[mi.MODEL_N], "ndop_years_per_s": 1.0 / t_single_ndop,
            "npzd_years_per_s": 1.0 / singles[mi.MODEL_NPZD],
            "how": "N-DOP: single-context year map (resident kernel); N and NPZD-DOP: one-member ensembles"},
        "speedup_vs_sequential": t_seq / t_ens,
    }


def executed_per_step(prob, ntr=2, tridiagonal=False, step_operators=False):
    """Bytes and FP64 flops of one TMM step as the year kernel carries it out.

    bytes: explicit values of two months (or, with per-step operators, the step's one
    interpolated matrix) and their column indices, row pointers, the implicit operator of
    two months (dense blocks: S_imp values each; tridiagonal form: three Thomas factors per
    cell each), and the state read and written once.
    flops: explicit part, one FMA per entry and tracer, plus one FMA per entry to
    interpolate the monthly matrices unless the per-step operators were built beforehand
    (once per context, not per year map); implicit part, the same per dense block entry, or
    per cell and tracer two Thomas solves (forward FMA, scaling multiply, backward FMA: 5
    flops each) and the interpolation (3 flops); the source term, ~20 flops per euphotic
    cell, ~8 per aphotic cell, plus adding the increment to every tracer.
    """
    n, nnz, s_imp = prob.n, prob.nnz, prob.s_imp
    imp_bytes = (2 * 3 * n * 8) if tridiagonal else s_imp * 2 * 8
    exp_values = 1 if step_operators else 2
    bytes_ = nnz * (exp_values * 8 + 4) + 4 * (n + 1) + imp_bytes + ntr * n * (8 + 8)
    L = prob.nlayer
    n_eu = int(np.minimum(L, 2).sum())
    imp_flops = (13 * ntr * n) if tridiagonal else s_imp * (2 + 2 * ntr)
    exp_flops = nnz * (2 * ntr if step_operators else 2 + 2 * ntr)
    flops = exp_flops + imp_flops + 20 * n_eu + 8 * (n - n_eu) + 2 * ntr * n
    return bytes_, flops


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        # nvidia-smi numbers GPUs in PCI order whatever CUDA_VISIBLE_DEVICES says: select the
        # GPU by the UUID of the CUDA device this process uses
        self.index = str(index)
        try:
            import torch
            uid = str(torch.cuda.get_device_properties(index).uuid)
            if uid and uid != "None":
                self.index = uid if uid.startswith(("GPU-", "MIG-")) else "GPU-" + uid
        except Exception:
            pass
        self.proc = None
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", self.index, "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        try:
            self.f.seek(0)
            rows = [r.split(",") for r in self.f.read().strip().splitlines() if r.strip()]
        except Exception:
            rows = []
        finally:
            try:
                os.unlink(self.f.name)
            except OSError:
                pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in rows if len(r) > 2]
        mx = [float(r[2]) for r in rows if len(r) > 2]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in rows:
            for k, nm in enumerate(names):
                if len(r) > 5 + k and r[5 + k].strip().lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(rows)}


def cpu_baseline(prob, seconds=12.0, max_steps=16 * 2880):
    """The CPU oracle as it stands, on all host cores, over a bounded sample of the workload:
    consecutive TMM steps of the year map for about `seconds`, at most 16 model years."""
    import oracle
    threads = oracle.set_threads(os.cpu_count() or 1)
    P = oracle.Problem(prob)
    u = mi.default_params_ndop()
    y = mi.initial_state(prob)
    t0 = time.perf_counter()
    steps = 0
    chunk = 24
    while steps < max_steps and time.perf_counter() - t0 < seconds:
        y = oracle.steps(P, steps % prob.nstep, chunk, y, u)
        steps += chunk
    dt = time.perf_counter() - t0
    oracle.set_threads(1)
    years = steps / prob.nstep
    # the oracle's plain single-threaded mode over a shorter sample
    y = mi.initial_state(prob)
    t1 = time.perf_counter()
    steps1 = 0
    while steps1 < max_steps and time.perf_counter() - t1 < seconds / 3:
        y = oracle.steps(P, steps1 % prob.nstep, chunk, y, u)
        steps1 += chunk
    dt1 = time.perf_counter() - t1
    return {"value": years / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": "%d consecutive TMM steps (%.2f model years) of the %s year map, FP64 C oracle, "
                      "%d OpenMP threads, %.1f s" % (steps, years, WORKLOAD, threads, dt),
            "single_thread": {"value": steps1 / prob.nstep / dt1, "unit": UNIT, "cores": 1,
                              "sample": "%d TMM steps, %.1f s" % (steps1, dt1)}}


def max_over_ranks(seconds, pg, device):
    """The slowest rank's time (every rank gets it); seconds unchanged without a process group."""
    if pg is None:
        return seconds
    import torch
    t = torch.tensor([seconds], dtype=torch.float64, device=device)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world, units_per_rank, seconds):
    """Units of all ranks per second of the slowest rank (weak scaling: every rank does the same work)."""
    return world * units_per_rank / seconds


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def workload_config(prob, world):
    """The bench line's `config`, the same for both arms."""
    return {"workload": WORKLOAD + " year map: PO4-DOP, 2 tracers, 2880 TMM steps per model year",
            "n": prob.n, "ncol": prob.ncol, "nnz": prob.nnz, "S_imp": prob.s_imp,
            "parallelism": "replicas" if world > 1 else "single",
            "l2": "flushed between timed iterations (256 MiB write); 12 months of matrices (~270 MB) exceed L2"}


def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return 0
    prob = mi.make_problem(WORKLOAD)
    import oracle
    threads = oracle.set_threads(os.cpu_count() or 1)
    P = oracle.Problem(prob)
    u = mi.default_params_ndop()
    y = mi.initial_state(prob)
    sample_steps = 288        # one tenth of a model year per benchmark step
    for _ in range(args.warmup):
        y = oracle.steps(P, 0, sample_steps, y, u)
    t0 = time.perf_counter()
    for k in range(args.steps):
        y = oracle.steps(P, (k * sample_steps) % prob.nstep, sample_steps, y, u)
    dt = time.perf_counter() - t0
    value = args.steps * sample_steps / prob.nstep / dt
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": workload_config(prob, args.gpus),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": "%d x %d TMM steps (each bench step 1/10 model year) of the %s year map"
                                       % (args.steps, sample_steps, WORKLOAD)},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import torch
    world, rank, local = dist_env()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU")
    torch.cuda.set_device(local)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        pg = dist
    import paper_1410_0204_gb300 as m3d

    prob = mi.make_problem(WORKLOAD)
    u_h = mi.default_params_ndop()
    y0_h = mi.initial_state(prob)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        ctx = m3d.Context.from_problem(prob, model=m3d.MODEL_NDOP, ntracer=2, nparam=7, stream=stream)
        tridiagonal = ctx.get_option(m3d.OPT_IMPLICIT_FORM) == m3d.IMPLICIT_TRIDIAGONAL
        plan = {m3d.PLAN_RESIDENT: "resident", m3d.PLAN_PERSISTENT: "persistent",
                m3d.PLAN_GRAPH: "graph"}[ctx.get_option(m3d.OPT_YEAR_PLAN)]
        y0 = torch.from_numpy(y0_h).cuda()
        u = torch.from_numpy(u_h).cuda()
        ya = torch.empty_like(y0)
        flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")   # > L2 (129 MB)
        for _ in range(max(args.warmup, 0)):
            ctx.year_map(y0, ya, u)
        torch.cuda.synchronize()
        if pg:
            pg.barrier()
        torch.cuda.synchronize()
        times = []
        launches = 0
        # the year kernel's own launch, timed by the library with CUDA events on its stream
        ctx.set_option(m3d.OPT_KERNEL_TIMING, 1)
        kernel_s, kernel_n = 0.0, 0
        with ClockSampler(local) as clocks:
            for _ in range(args.steps):
                flush.fill_(1.0)                       # L2 flushed between timed iterations
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                ctx.year_map(y0, ya, u)
                e1.record(stream)
                launches += ctx.last_launch_count()
                e1.synchronize()
                times.append(e0.elapsed_time(e1) / 1e3)
                kns = ctx.get_option(m3d.OPT_LAST_KERNEL_NS)
                if kns > 0:
                    kernel_s += kns * 1e-9
                    kernel_n += 1
        ctx.set_option(m3d.OPT_KERNEL_TIMING, 0)
        torch.cuda.synchronize()
        if pg:
            pg.barrier()
        total = max_over_ranks(sum(times), pg, "cuda")
        value = whole_job_rate(world, args.steps, total)

        # end to end through the C ABI with host buffers (pinned), copies inside the timed region
        y0_pin = torch.from_numpy(y0_h).pin_memory()
        y1_pin = torch.empty_like(y0_pin).pin_memory()
        u_pin = torch.from_numpy(u_h).pin_memory()
        ctx.year_map_host_ptr(y0_pin.data_ptr(), y1_pin.data_ptr(), u_pin.data_ptr())
        e2e_steps = max(1, min(args.steps, 5))
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            ctx.year_map_host_ptr(y0_pin.data_ptr(), y1_pin.data_ptr(), u_pin.data_ptr())
        e2e_dt = max_over_ranks(time.perf_counter() - t0, pg, "cuda")
        e2e_value = whole_job_rate(world, e2e_steps, e2e_dt)

        # the per-step explicit operators: their size, the time to build them, and the year
        # map with the kernel interpolating every entry itself instead (identical results)
        step_ops = bool(ctx.get_option(m3d.OPT_STEP_OPERATORS))
        stepops = {"on": step_ops}
        if step_ops:
            stepops["bytes"] = int(ctx.get_option(m3d.OPT_STEP_OPERATOR_BYTES))
            ctx.set_option(m3d.OPT_STEP_OPERATORS, 0)
            k = max(1, min(args.steps, 3))
            ctx.year_map(y0, ya, u)
            t_int = 0.0
            for _ in range(k):
                flush.fill_(1.0)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                ctx.year_map(y0, ya, u)
                e1.record(stream)
                e1.synchronize()
                t_int += e0.elapsed_time(e1) / 1e3
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ctx.set_option(m3d.OPT_STEP_OPERATORS, 1)
            stepops["build_s"] = time.perf_counter() - t0
            stepops["in_kernel_interpolation"] = {"value": k / t_int, "unit": UNIT, "ms_per_year": 1e3 * t_int / k,
                                                  "years": k}

        # cost of the adjoint year map (checkpoint every 240 steps) and of the tangent year map,
        # each relative to one year map, wall clock with the device synchronised on both sides
        costs = {}
        if not args.no_adjoint:
            ybar1 = torch.ones_like(y0)
            ybar0 = torch.empty_like(y0)
            v = torch.ones_like(y0)
            phi = torch.empty_like(y0)
            jv = torch.empty_like(y0)

            def wall(fn, k):
                fn()
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                for _ in range(k):
                    fn()
                torch.cuda.synchronize()
                return (time.perf_counter() - t0) / k

            k = max(1, min(args.steps, 3))
            t_fwd = wall(lambda: ctx.year_map(y0, ya, u), k)
            t_adj = wall(lambda: ctx.year_adjoint(y0, u, ybar1, ybar0, 240), k)
            t_all = wall(lambda: ctx.year_adjoint(y0, u, ybar1, ybar0, prob.nstep), k)
            t_tan = wall(lambda: ctx.year_tangent(y0, v, u, phi, jv), k)
            costs = {"forward_s": t_fwd, "adjoint_s": t_adj, "tangent_s": t_tan,
                     "adjoint_over_forward": t_adj / t_fwd, "tangent_over_forward": t_tan / t_fwd,
                     "ckpt_every": 240, "repeats": k,
                     "adjoint_includes": "forward sweep keeping 12 checkpoints, recomputation of each 240-step segment, reverse sweep",
                     "store_all": {"adjoint_s": t_all, "adjoint_over_forward": t_all / t_fwd,
                                   "state_bytes": int((prob.nstep + 1) * 2 * prob.n * 8),
                                   "how": "ckpt_every = nstep: one forward sweep keeps all 2881 states in HBM, no recomputation"}}

        ensemble = {}
        if not args.no_ensemble:
            ensemble = run_ensemble(prob, total / args.steps, flush)

        # Newton-Krylov periodic solve to ||phi(y) - y|| < 1e-8 from the constant initial state
        newton = {}
        if not args.no_newton:
            modes = [("fd", m3d.JV_FD)] + ([] if args.no_newton_tangent else [("tangent", m3d.JV_TANGENT)])
            for label, jv in modes:
                yN = torch.from_numpy(y0_h).cuda()
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                st, rep = ctx.newton_solve(yN, u, tol=1e-8, jv=jv)
                dt_n = time.perf_counter() - t0
                newton[label] = {"seconds": dt_n, "converged": bool(rep["converged"]), "residual": rep["residual"],
                                 "newton_steps": rep["newton_steps"], "krylov_iterations": rep["krylov_total"],
                                 "year_maps": rep["year_maps"], "tangent_maps": rep["tangent_maps"],
                                 "model_year_equivalents": rep["year_maps"] + rep["tangent_maps"],
                                 "krylov_per_newton_step": rep.get("krylov"), "residuals": rep.get("residuals"),
                                 "line_search_steps": rep.get("lambdas"), "forcing_terms": rep.get("etas"),
                                 "line_search_trials": rep.get("trials")}
        # spin-up to the Newton tolerance (the paper's comparison of Section 7), capped
        spinup = {}
        if args.spinup_years > 0:
            yS = torch.from_numpy(y0_h).cuda()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            res = ctx.spinup(yS, u, args.spinup_years, tol=1e-8)
            dt_s = time.perf_counter() - t0
            first_below = {}
            for thr in (1e-2, 1e-4, 1e-6, 1e-8):
                hit = np.nonzero(res < thr)[0]
                first_below["%g" % thr] = int(hit[0]) + 1 if hit.size else None
            spinup = {"seconds": dt_s, "years": int(res.size), "final_residual": float(res[-1]),
                      "reached_1e-8": bool(res[-1] < 1e-8), "years_to_reach": first_below, "cap": args.spinup_years}
        ctx.close()

    if rank != 0:
        if pg:
            pg.destroy_process_group()
        return 0
    hbm_peak, hbm_src = peaks()
    bytes_step, flops_step = method_per_step(prob)
    xbytes_step, xflops_step = executed_per_step(prob, tridiagonal=tridiagonal, step_operators=step_ops)
    t_year = total / args.steps
    t_kernel = kernel_s / max(kernel_n, 1) if kernel_n else t_year
    achieved_tf = flops_step * prob.nstep / t_year / 1e12
    achieved_gbs = bytes_step * prob.nstep / t_kernel / 1e9
    executed_tf = xflops_step * prob.nstep / t_kernel / 1e12
    clock = clocks.summary()
    fp64_peak, fp64_src = fp64_peak_tflops(clock.get("sm_mhz"))
    traffic, traffic_how = TRAFFIC_PER_LAUNCH.get((plan, tridiagonal, step_ops, YEAR_KERNEL_REVISION),
                                                  (None, None))
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * t_year, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(prob, world),
        "roofline": {"bound": "hbm", "achieved": achieved_gbs, "peak": hbm_peak, "unit": "GB/s",
                     "frac": achieved_gbs / hbm_peak, "peak_source": hbm_src + " (MEASURED_PEAKS hbm_gbs)"
                     if hbm_src == "measured" else "fallback 6.8 TB/s",
                     "traffic": traffic,
                     "traffic_unit": "DRAM bytes per launch (one model year), ncu",
                     "traffic_how": traffic_how,
                     "kernel": {"resident": "k_year_resident (one launch per model year)",
                                "persistent": "k_year (one launch per model year)",
                                "graph": "k_step (one launch per TMM step)"}[plan],
                     "kernel_ms": 1e3 * t_kernel, "kernel_launches_timed": kernel_n,
                     "bytes_per_step": bytes_step,
                     "bytes_note": ("algorithmic bytes of the method per TMM step: nnz (2 x 8 + 4) + 4 (n + 1) + "
                                    "S_imp 2 x 8 + ntr n (8 + 8), x 2880 steps per launch"),
                     "plan": plan, "implicit_form": "tridiagonal" if tridiagonal else "dense"},
        "fp64": {"bound": "alu", "unit": "TFLOP/s", "peak": fp64_peak, "peak_source": fp64_src,
                 "executed": {"flops_per_step": xflops_step, "bytes_per_step": xbytes_step,
                              "achieved": executed_tf, "frac": executed_tf / fp64_peak},
                 "note": ("FP64 flops the kernel executes (Thomas form of the implicit part; with per-step "
                          "explicit operators no interpolation in the kernel) per kernel time"),
                 "method_flops_per_step": flops_step},
        "dram_measured": ({"gbs": traffic / t_kernel / 1e9, "frac": traffic / t_kernel / 1e9 / hbm_peak,
                           "note": "ncu DRAM bytes of one launch / kernel time"} if traffic else None),
        "step_operators": stepops,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(y0_h.nbytes + u_h.nbytes),
                "d2h_bytes_per_step": int(y0_h.nbytes)},
        "throughput": {"cell_tracer_steps_per_s": value * prob.n * 2 * prob.nstep,
                       "unit": "wet cells x tracers x TMM steps per second"},
        "gpu_launches": launches,
        "clocks": clock,
        "newton": newton,
        "adjoint": costs,
        "ensemble": ensemble,
    }
    if spinup:
        line["spinup"] = spinup
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(prob)
    print(json.dumps(line), flush=True)
    if pg:
        pg.destroy_process_group()
    return 0


def run_profile_steps(nsteps):
    """A short run for profilers: set up the benchmark workload and run nsteps single TMM steps."""
    import torch
    import paper_1410_0204_gb300 as m3d
    prob = mi.make_problem(WORKLOAD)
    ctx = m3d.Context.from_problem(prob, model=m3d.MODEL_NDOP, ntracer=2, nparam=7)
    y = torch.from_numpy(mi.initial_state(prob)).cuda()
    u = torch.from_numpy(mi.default_params_ndop()).cuda()
    yn = torch.empty_like(y)
    for j in range(nsteps):
        ctx.step(j, y, yn, u)
        y, yn = yn, y
    torch.cuda.synchronize()
    ctx.close()
    print(json.dumps({"profile_steps": nsteps, "workload": WORKLOAD}))
    return 0


def run_profile_years(nyears, grid, plan=None):
    """A short run for profilers: nyears year maps on `grid`, by the context's own year plan or
    by the persistent one (`plan="persistent"`: the kernel that streams every step's matrices
    from HBM, as on grids whose tiles do not fit in shared memory)."""
    import torch
    import paper_1410_0204_gb300 as m3d
    prob = mi.make_problem(grid)
    ctx = m3d.Context.from_problem(prob, model=m3d.MODEL_NDOP, ntracer=2, nparam=7)
    if plan == "persistent":
        if ctx.get_option(m3d.OPT_STEP_OPERATORS):
            ctx.set_option(m3d.OPT_STEP_OPERATORS, 0)
        ctx.set_option(m3d.OPT_YEAR_PLAN, m3d.PLAN_PERSISTENT)
    y = torch.from_numpy(mi.initial_state(prob)).cuda()
    u = torch.from_numpy(mi.default_params_ndop()).cuda()
    yn = torch.empty_like(y)
    for _ in range(nyears):
        ctx.year_map(y, yn, u)
        y, yn = yn, y
    torch.cuda.synchronize()
    out = {"profile_years": nyears, "grid": grid, "plan": ctx.get_option(m3d.OPT_YEAR_PLAN),
           "step_operator_bytes": ctx.get_option(m3d.OPT_STEP_OPERATOR_BYTES)}
    ctx.close()
    print(json.dumps(out))
    return 0


def run_scale_1deg(args):
    """The 1-degree grid (360 x 180 x 23, 700,000 cells): the single-context N-DOP year map and
    the 16-member NPZD-DOP ensemble year map, each timed with CUDA events over whole years."""
    import torch
    import paper_1410_0204_gb300 as m3d
    t_start = time.perf_counter()

    def progress(what):
        sys.stderr.write("[scale-1deg %7.1f s] %s\n" % (time.perf_counter() - t_start, what))
        sys.stderr.flush()

    name = "npzd_360x180x23"
    prob = mi.make_problem(name)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    def timed(fn, reps):
        fn()
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            flush.fill_(1.0)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record()
            fn()
            b.record()
            b.synchronize()
            ts.append(a.elapsed_time(b) / 1e3)
        return sum(ts) / len(ts)

    reps = max(1, min(args.steps, 3))
    ctx = m3d.Context.from_problem(prob, model=m3d.MODEL_NDOP, ntracer=2, nparam=7)
    plan = {m3d.PLAN_RESIDENT: "resident", m3d.PLAN_PERSISTENT: "persistent",
            m3d.PLAN_GRAPH: "graph"}[ctx.get_option(m3d.OPT_YEAR_PLAN)]
    y0 = torch.from_numpy(mi.initial_state(prob)).cuda()
    u = torch.from_numpy(mi.default_params_ndop()).cuda()
    ya = torch.empty_like(y0)
    t_single = timed(lambda: ctx.year_map(y0, ya, u), reps)
    progress("single-context year map")
    # the adjoint (streaming sweep on this grid), checkpoint every 480 steps, wall clock
    yb0 = torch.empty_like(y0)
    ybar1 = torch.ones_like(y0)
    ctx.year_adjoint(y0, u, ybar1, yb0, 480)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ctx.year_adjoint(y0, u, ybar1, yb0, 480)
    torch.cuda.synchronize()
    t_adj = time.perf_counter() - t0
    progress("single-context adjoint")
    adj_plan = {m3d.PLAN_RESIDENT: "resident", m3d.PLAN_PERSISTENT: "streaming"}.get(
        ctx.get_option(m3d.OPT_ADJOINT_PLAN), "none")
    # the tangent year map (phi and phi' v in one pass), CUDA events
    v = torch.ones_like(y0)
    phi, jv = torch.empty_like(y0), torch.empty_like(y0)
    t_tan = timed(lambda: ctx.year_tangent(y0, v, u, phi, jv), reps)
    progress("single-context tangent")
    tridiagonal = ctx.get_option(m3d.OPT_IMPLICIT_FORM) == m3d.IMPLICIT_TRIDIAGONAL
    ctx.close()
    _, flops_single = method_per_step(prob)
    _, xflops_single = executed_per_step(prob, tridiagonal=tridiagonal)
    members = mi.make_ensemble(((mi.MODEL_NPZD, 16),), seed=1410)
    ens = m3d.Ensemble.from_problem(prob, members)
    Y0 = torch.from_numpy(np.vstack([mi.initial_state(prob, 5, mi.model_initial_values(mi.MODEL_NPZD))
                                     for _ in members])).cuda()
    Y1 = torch.empty_like(Y0)
    cpb, nw, ms = ens.autotune(Y0, nsteps=5)
    progress("ensemble autotune")
    t_ens = timed(lambda: ens.year_map(Y0, Y1), reps)
    progress("ensemble year map")
    # the ensemble's derivatives: one tangent-ensemble year map (phi and phi' v of all 16 members:
    # one Krylov iteration of all members' Newton-Krylov solves), the reverse sweep (checkpoint
    # every 480 steps), and a bounded batched Newton-Krylov run (tangent products) from a state
    # spun up for a few years
    deriv = {}
    if not args.no_adjoint:
        tan = m3d.Ensemble.from_problem(prob, members, tangent=True)
        tan.set_tiling(*ens.get_tiling())
        V = torch.from_numpy(np.random.default_rng(5).standard_normal(tuple(Y0.shape))).cuda()
        YV = torch.cat([Y0, V])
        t_etan = timed(lambda: tan.year_map(YV, torch.empty_like(YV)), 1)
        progress("tangent-ensemble year map")
        Wb = torch.ones_like(Y0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ens.year_adjoint(Y0, Wb, torch.empty_like(Y0), ckpt_every=480)
        torch.cuda.synchronize()
        t_eadj = time.perf_counter() - t0
        progress("ensemble reverse sweep")
        Ys = Y0.clone()
        for _ in range(args.scale_spinup_years):
            ens.year_map(Ys, Ys)
        torch.cuda.synchronize()
        progress("spin-up")
        t0 = time.perf_counter()
        st, reps_n = ens.newton_solve(Ys, prob.vol, tangent_ensemble=tan, tol=1e-8, jv=m3d.JV_TANGENT,
                                      max_newton=args.scale_newton_steps, max_krylov=args.scale_krylov,
                                      restart=args.scale_krylov)
        torch.cuda.synchronize()
        t_newton = time.perf_counter() - t0
        progress("ensemble Newton-Krylov")
        tan.close()
        deriv = {"tangent_year_map_s": t_etan, "tangent_over_forward": t_etan / t_ens,
                 "adjoint_s": t_eadj, "adjoint_over_forward": t_eadj / t_ens, "ckpt_every": 480,
                 "newton": {"seconds": t_newton, "spinup_years_before": args.scale_spinup_years,
                            "max_newton": args.scale_newton_steps, "max_krylov": args.scale_krylov,
                            "krylov_iterations_all_members": max(r["krylov_total"] for r in reps_n),
                            "tangent_year_maps": reps_n[0]["tangent_maps"], "year_maps": reps_n[0]["year_maps"],
                            "residual0": [r["residual0"] for r in reps_n], "residual": [r["residual"] for r in reps_n],
                            "seconds_per_krylov_iteration": t_newton / max(1, max(r["krylov_total"] for r in reps_n)),
                            "how": "every member's Newton-Krylov in lockstep, one tangent-ensemble year map per Krylov "
                                   "iteration of all 16 members, bounded (max_newton, max_krylov)"}}
    ens.close()
    f_ens = ensemble_flops_per_step(prob, members) * prob.nstep
    line = {"metric": METRIC, "value": 1.0 / t_single, "unit": UNIT, "n_gpus": 1, "steps": reps,
            "higher_is_better": True, "dtype": "f64", "data": "synthetic",
            "config": {"workload": name + " year map: PO4-DOP, 2 tracers, 2880 TMM steps per model year",
                       "n": prob.n, "ncol": prob.ncol, "nnz": prob.nnz, "S_imp": prob.s_imp, "plan": plan,
                       "implicit_form": "tridiagonal" if tridiagonal else "dense"},
            "roofline": {"bound": "alu", "achieved": flops_single * prob.nstep / t_single / 1e12,
                         "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                         "frac": flops_single * prob.nstep / t_single / 1e12 / FP64_PEAK_TFLOPS,
                         "executed": {"achieved": xflops_single * prob.nstep / t_single / 1e12,
                                      "frac": xflops_single * prob.nstep / t_single / 1e12 / FP64_PEAK_TFLOPS}},
            "adjoint": {"seconds": t_adj, "adjoint_over_forward": t_adj / t_single, "ckpt_every": 480,
                        "sweep": adj_plan},
            "tangent": {"seconds": t_tan, "tangent_over_forward": t_tan / t_single},
            "ensemble": {"workload": "16 NPZD-DOP members (5 tracers), parameters within +-50% of the defaults",
                         "member_years_per_s": len(members) / t_ens, "seconds_per_ensemble_year": t_ens,
                         "derivatives": deriv,
                         "tiling": {"cols_per_block": cpb, "warps_per_block": nw, "autotune_ms_per_step": ms},
                         "roofline": {"bound": "alu", "achieved": f_ens / t_ens / 1e12, "peak": FP64_PEAK_TFLOPS,
                                      "unit": "TFLOP/s", "frac": f_ens / t_ens / 1e12 / FP64_PEAK_TFLOPS}}}
    print(json.dumps(line), flush=True)
    return 0


def run_profile_ensemble(nsteps):
    """A short run for profilers: the 64-member ensemble on the benchmark grid, nsteps steps."""
    import torch
    import paper_1410_0204_gb300 as m3d
    prob = mi.make_problem(WORKLOAD)
    members = mi.make_ensemble()
    ens = m3d.Ensemble.from_problem(prob, members)
    Y0 = torch.from_numpy(np.vstack([mi.initial_state(prob, m.ntracer, mi.model_initial_values(m.model))
                                     for m in members])).cuda()
    ens.set_tiling(1, 5)                 # the autotuner's usual choice on this grid
    ens.steps(0, nsteps, Y0, torch.empty_like(Y0))
    torch.cuda.synchronize()
    ens.close()
    print(json.dumps({"profile_ensemble_steps": nsteps, "workload": WORKLOAD, "members": len(members)}))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-newton", action="store_true", help="skip the Newton-Krylov solve timing")
    ap.add_argument("--no-adjoint", action="store_true", help="skip the adjoint/tangent cost timing")
    ap.add_argument("--no-ensemble", action="store_true", help="skip the batched ensemble timing")
    ap.add_argument("--spinup-years", type=int, default=0,
                    help="also time a spin-up of up to this many years to ||phi(y) - y|| < 1e-8 (e.g. 3000)")
    ap.add_argument("--no-newton-tangent", action="store_true",
                    help="skip the Newton-Krylov solve with tangent Jacobian-vector products")
    ap.add_argument("--profile-steps", type=int, default=0,
                    help="only run this many single TMM steps of the workload (for profilers)")
    ap.add_argument("--profile-ensemble-steps", type=int, default=0,
                    help="only run this many steps of the 64-member ensemble (for profilers)")
    ap.add_argument("--profile-years", type=int, default=0,
                    help="only run this many year maps (for profilers) on --profile-grid")
    ap.add_argument("--profile-grid", default=WORKLOAD, help="grid of --profile-years")
    ap.add_argument("--profile-plan", default=None, choices=["persistent"],
                    help="year plan of --profile-years (default: the context's own)")
    ap.add_argument("--scale-1deg", action="store_true",
                    help="time the 1-degree grid (single context and 16-member ensemble) instead")
    ap.add_argument("--scale-spinup-years", type=int, default=2,
                    help="--scale-1deg: years of spin-up before the bounded ensemble Newton-Krylov run")
    ap.add_argument("--scale-newton-steps", type=int, default=1,
                    help="--scale-1deg: Newton steps of the bounded ensemble Newton-Krylov run")
    ap.add_argument("--scale-krylov", type=int, default=4,
                    help="--scale-1deg: Krylov iterations per Newton step of that run")
    args = ap.parse_args()
    if args.scale_1deg:
        return run_scale_1deg(args)
    if args.profile_ensemble_steps:
        return run_profile_ensemble(args.profile_ensemble_steps)
    if args.profile_steps:
        return run_profile_steps(args.profile_steps)
    if args.profile_years:
        return run_profile_years(args.profile_years, args.profile_grid, args.profile_plan)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
