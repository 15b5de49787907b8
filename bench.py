#!/usr/bin/env python3
"""Benchmark of the AIRG solve phase: DOFs solved per second to rtol 1e-10.

Default workload (`--workload c3`): the 4096x4096 upwind advection problem
(seeded direction, inflow values U[0,1], coarse polynomial order 30,
truncation tolerance 1e-2), 16.8M DOFs, the per-GPU size class of the paper's
runs (Sec. 3).  A step is one complete solve (FP64 FGMRES preconditioned by
AIRG V-cycles, Sec. 2-3 of arXiv 2508.17517) from x0 = 0 with the hierarchy
set up once beforehand (the paper times the second solve).  `value` = DOFs
solved per second with the FP64 V-cycle, timed on the device with CUDA
events around each solve, L2 flushed between steps; `mixed` (FP32 V-cycle
inside the FP64 outer iteration) and `mixed_bf16r` (the same with the
restrictor stored in bfloat16) are timed the same way on the same right-hand
side, with their error against the FP64 solution and the exact solution.
`e2e` repeats the solves through the C ABI with host buffers, copies
included.  The roofline entry times its kernel group alone with CUDA events
(airg_profile_group) after a first pass has ranked the groups.

  python bench.py [--gpus N] [--steps K] [--warmup W]
                  [--workload c3|c1|c2|c3_fp64|c3_fp32|c3_bf16|c4a|c4a_fp64|c4a_bf16|c4b]
  python bench.py --impl reference ...   (the CPU oracle as the reference arm)
  python bench.py --sweep coarse-order|smoother|cases|readings   (one JSON line of study rows)
"""
import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")
os.environ.setdefault("OMP_NUM_THREADS", "1")
os.environ.setdefault("MKL_NUM_THREADS", "1")

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "DOFs solved/s to rtol 1e-10 (mixed vs FP64 on GPU); V-cycle HBM GB/s vs peak"
L2_FLUSH_BYTES = 256 << 20
# bench workload name -> synthetic workload name (c3 is the paired FP64 / mixed run)
SINGLE = {"c1": "c1", "c2": "c2", "c3_fp64": "c3_fp64", "c3_fp32": "c3", "c3_bf16": "c3_bf16",
          "c4a": "c4a", "c4a_fp64": "c4a_fp64", "c4a_bf16": "c4a_bf16", "c4b": "c4b"}
# side of the lower-left corner of the 4096^2 grid that the CPU oracle solves
# as its bounded sample (upwind dependence makes the corner a closed problem)
CORNER = 1024


def parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="c3", choices=["c3"] + sorted(SINGLE))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--problems", type=int, default=None,
                    help="number of grids of the many-grid workload (a smaller case of it, for profiling)")
    ap.add_argument("--grid", type=int, default=None,
                    help="grid side of a single-problem workload (a smaller case of the same kind, "
                         "for profiling)")
    ap.add_argument("--sweep", choices=["coarse-order", "smoother", "cases", "readings"], default=None,
                    help="instead of the throughput line, one JSON line with a row per setting: "
                         "coarse-order = the coarse polynomial order / truncation study of Sec. 3.1; "
                         "smoother = matrix-free polynomial vs assembled Eq. 8 smoother (Sec. 2.2) and F vs FC/FCF "
                         "smoothing (Sec. 2); "
                         "cases = hard direction (Sec. 3.3.2) and rectangular domain (Sec. 3.4); "
                         "readings = R drop tolerance and DDC settings against levels and complexities")
    return ap.parse_args(argv)


def dist_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def max_over_ranks(value, world, device=None):
    """Max of a float over the ranks of the default process group."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ----------------------------------------------------------- clock sampling --
class Clocks:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.3)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
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
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": sorted(reasons),
                "samples": len(sm)}


# --------------------------------------------------------------- workloads --
def problem_and_rhs(w, G, torch):
    """Operator and the right-hand sides b (n, or k x n for k > 1) on the device."""
    from synthetic import velocity
    vx, vy = velocity(w["theta"])
    prob = G.airg_problem_advection2d(w["nx"], w["ny"], vx, vy)
    k = w["n_rhs"]
    g = torch.tensor(w["g"] if k > 1 else w["g"][0], device="cuda")
    s = None
    if w["s"] is not None:
        s = torch.tensor(w["s"] if k > 1 else w["s"][0], device="cuda")
    b = G.airg_assemble_rhs_advection2d(prob, g, s)
    return prob, b


def reference_sample(args):
    """The workload the CPU oracle times, and what it is.  For the 4096^2
    workloads the oracle's setup alone would take many minutes, so its sample
    is the CORNER x CORNER lower-left corner of the same problem (a closed
    sub-problem with the same direction, inflow values and options); other
    workloads are sampled whole."""
    from synthetic import corner, workload
    name = "c3_fp64" if args.workload == "c3" else SINGLE[args.workload]
    w = workload(name, n=args.grid)
    if w.get("n_rhs", 1) != 1 or "problems" in w:
        return w, None
    if w["nx"] * w["ny"] > CORNER * CORNER:
        return corner(w, CORNER), "the %dx%d lower-left corner of the workload" % (CORNER, CORNER)
    return w, "the workload"


def cpu_oracle_solve(w, steps, warmup, min_seconds=0.0):
    """Times the oracle's solve (after an untimed oracle setup) of workload
    w: `steps` solves, more while their total stays below `min_seconds`;
    returns (DOFs/s, per-step seconds, oracle iterations, setup seconds)."""
    from oracle import airg as O
    from synthetic import velocity
    vx, vy = velocity(w["theta"])
    po = O.advection_2d(w["nx"], w["ny"], vx, vy)
    opts = O.Options(**{k: v for k, v in w["opts"].items() if k != "precision"})
    t0 = time.perf_counter()
    Ho = O.setup(po.A, opts)
    setup_s = time.perf_counter() - t0
    s = w["s"][0] if w["s"] is not None else [0.0] * po.A.n_rows
    bo = O.assemble_rhs(po, w["g"][0], s)
    for _ in range(warmup):
        O.solve(Ho, po.A, bo, rtol=w["rtol"])
    ts, its = [], 0
    while len(ts) < steps or sum(ts) < min_seconds:
        t0 = time.perf_counter()
        _, info = O.solve(Ho, po.A, bo, rtol=w["rtol"])
        ts.append(time.perf_counter() - t0)
        its = info.iterations
    n = po.A.n_rows
    return n * len(ts) / sum(ts), ts, its, setup_s


def cpu_exact(w, repeats=3):
    """The exact discrete solution of workload w by substitution in upwind
    order (Sec. 1.1), the O(n) serial solver of this lower-triangular system
    that the paper sets against multigrid because it does not parallelise.
    Oracle code, one core.  Returns (u*, DOFs/s of the best of `repeats`,
    seconds)."""
    from oracle import airg as O
    from synthetic import velocity
    vx, vy = velocity(w["theta"])
    po = O.advection_2d(w["nx"], w["ny"], vx, vy)
    s = w["s"][0] if w["s"] is not None else [0.0] * po.A.n_rows
    bo = O.assemble_rhs(po, w["g"][0], s)
    order = O.sweep_order(po)
    best, u = math.inf, None
    for _ in range(repeats):
        t0 = time.perf_counter()
        u = O.sweep_solve(po.A, bo, order)
        best = min(best, time.perf_counter() - t0)
    return u, po.A.n_rows / best, best


def cpu_baseline_entry(args, min_seconds=10.0):
    """The oracle on its bounded sample: setup untimed, then at least
    `min_seconds` of solves."""
    ws, what = reference_sample(args)
    if what is None:
        return None
    cv, ts, its, setup_s = cpu_oracle_solve(ws, 1, 0, min_seconds=min_seconds)
    return {"value": cv, "unit": "DOF/s", "cores": 1, "kind": "oracle",
            "sample": "%s (%d DOFs; oracle setup untimed, %.0f s): %d full solves to rtol %g, "
                      "%d iterations each, %.1f s in total" % (what, ws["nx"] * ws["ny"], setup_s, len(ts),
                                                               ws["rtol"], its, sum(ts))}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    ws, what = reference_sample(args)
    if what is None:
        print(json.dumps({"impl": "reference", "unavailable": "the oracle has no solve of this batched workload"}))
        return
    t0 = time.time()
    value, ts, its, setup_s = cpu_oracle_solve(ws, args.steps, args.warmup)
    from synthetic import workload
    full = workload("c3_fp64" if args.workload == "c3" else SINGLE[args.workload])
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "DOF/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * sum(ts) / len(ts), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": full["desc"], "n": full["nx"] * full["ny"], "nrhs": 1, "rtol": full["rtol"]},
        "cpu_baseline": {"value": value, "unit": "DOF/s", "cores": 1, "kind": "oracle",
                         "sample": "each step one full oracle solve of %s (%d DOFs, %d iterations; "
                                   "single-threaded C kernels + numpy, FP64), setup untimed (%.0f s)"
                                   % (what, ws["nx"] * ws["ny"], its, setup_s)},
        "e2e": {"value": value, "unit": "DOF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "wall_s": time.time() - t0,
    }
    print(json.dumps(line))


def run_gpu_multi(args):
    """Workload of many separate grids of uneven size (one hierarchy each):
    `value` from the default form, each lockstep FGMRES iteration of all
    problems as one graph of per-problem branches; `worklist_form` times the
    same solves with each iteration as one persistent work-list launch."""
    import torch
    rank, world, local_rank, dev = _dist_setup(torch)
    import paper_2508_17517_gb300 as G
    from synthetic import velocity, workload
    G.lib()
    w = workload(args.workload, n=args.problems)
    csrs, bs = [], []
    for p in w["problems"]:
        vx, vy = velocity(p["theta"])
        pg = G.airg_problem_advection2d(p["nx"], p["ny"], vx, vy)
        csrs.append((pg["rowptr"], pg["col"], pg["val"]))
        bs.append(G.airg_assemble_rhs_advection2d(pg, torch.tensor(p["g"], device="cuda")))
    ntot = sum(p["nx"] * p["ny"] for p in w["problems"])
    t0 = time.perf_counter()
    B = G.airg_setup_batch(csrs, G.airg_options_default(**w["opts"]))
    setup_s = time.perf_counter() - t0
    xs = [torch.zeros_like(b) for b in bs]
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    peak, peak_kind = measured_peaks()

    def timed(form, steps, warmup, label):
        os.environ["AIRG_MULTI"] = form
        for _ in range(warmup):
            for x in xs:
                x.zero_()
            G.airg_solve_batch(B, bs, xs, rtol=w["rtol"])
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        _barrier(world, torch)
        total_ms, its, launches = 0.0, [], 0
        torch.cuda.nvtx.range_push(label)
        for _ in range(steps):
            flush.zero_()
            for x in xs:
                x.zero_()
            ev0.record(stream)
            _, infos = G.airg_solve_batch(B, bs, xs, rtol=w["rtol"])
            ev1.record(stream)
            ev1.synchronize()
            total_ms += ev0.elapsed_time(ev1)
            its.append(max(i.iterations for i in infos))
            launches += sum(i.kernel_launches for i in infos)
            assert all(i.converged for i in infos)
        torch.cuda.nvtx.range_pop()
        _barrier(world, torch)
        return total_ms, its, launches

    def iteration_roofline(form, steps):
        """Event-timed iteration launches of one form (one pair per launch)."""
        os.environ["AIRG_MULTI"] = form
        G.airg_batch_profile(B, True)
        tot = 0.0
        for _ in range(steps):
            flush.zero_()
            for x in xs:
                x.zero_()
            t, _, _ = timed(form, 1, 0, "iteration timing")
            tot += t
        ms, nl, nb = G.airg_batch_profile_read(B)
        G.airg_batch_profile(B, False)
        gbs = nb / (ms / 1e3) / 1e9
        return {"kernel": {"worklist": "k_worklist (all problems' iteration, one launch)",
                           "graph": "iteration graph (per-problem branches)"}[form],
                "bound": "hbm", "launches": nl, "avg_launch_us": 1e3 * ms / nl,
                "algorithmic_bytes_per_launch": nb / nl, "share": ms / tot,
                "achieved": gbs, "peak": peak, "unit": "GB/s", "frac": gbs / peak, "peak_source": peak_kind,
                "timing": "each iteration launch between CUDA events on the batch stream, %d solves" % steps}

    clk = Clocks(local_rank)
    clk.start()
    t_wall0 = time.perf_counter()
    total_ms, its, launches = timed("graph", args.steps, args.warmup, "timed")
    wall_s = time.perf_counter() - t_wall0
    g_ms, g_its, g_launches = timed("worklist", args.steps, args.warmup, "work-list form")
    clocks = clk.stop()
    t_max = max_over_ranks(total_ms, world, dev)
    g_max = max_over_ranks(g_ms, world, dev)
    value = world * ntot * args.steps / (t_max / 1e3)
    os.environ["AIRG_MULTI"] = "graph"
    bh = [b.cpu().pin_memory() for b in bs]
    xh = [torch.zeros_like(b).pin_memory() for b in bh]
    G.airg_solve_batch(B, bh, xh, rtol=w["rtol"])     # warm-up of the host path (staging buffers)
    e2e_s = 0.0
    for _ in range(args.steps):
        for x in xh:
            x.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        G.airg_solve_batch(B, bh, xh, rtol=w["rtol"])
        e2e_s += time.perf_counter() - t0
    e2e_max = max_over_ranks(e2e_s, world, dev)
    roof = iteration_roofline("graph", args.steps)
    g_roof = iteration_roofline("worklist", args.steps)
    os.environ.pop("AIRG_MULTI", None)
    if rank == 0:
        print(json.dumps({
            "metric": METRIC, "value": value, "unit": "DOF/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": w["desc"], "n": ntot, "problems": len(bs), "rtol": w["rtol"],
                       "l2": "flushed (256 MiB write) between timed steps"},
            "iterations_per_solve": statistics.median(its), "setup_s": setup_s,
            "e2e": {"value": world * ntot * args.steps / e2e_max, "unit": "DOF/s",
                    "h2d_bytes_per_step": 16 * ntot, "d2h_bytes_per_step": 8 * ntot},
            "roofline": roof,
            "worklist_form": {"value": world * ntot * args.steps / (g_max / 1e3), "unit": "DOF/s",
                           "ms_per_step": g_max / args.steps, "iterations_per_solve": statistics.median(g_its),
                           "gpu_launches": g_launches, "roofline": g_roof},
            "cpu_baseline": None, "clocks": clocks, "gpu_launches": launches, "wall_s_timed": wall_s}))
    _dist_end(world)


# Arithmetic peaks from unit counts and the nominal 2070 MHz SM clock of the
# GB300 (152 SMs): 2 FP64 FMA per clock per SM (1.26 TFLOP/s; an FMA-chain
# probe measured 1.20), 128 FP32 FMA per clock per SM (80.5 TFLOP/s).
SM_COUNT, SM_GHZ = 152, 2.07
ALU_PEAK_TFLOPS = {"f64": 2 * 2 * SM_COUNT * SM_GHZ / 1e3, "f32": 2 * 128 * SM_COUNT * SM_GHZ / 1e3}
VCYCLE_KINDS = ("restrict", "f_residual", "f_smoother", "coarse_newton")


KERNEL_SECTION = (b"// ------------------------------------------------------- V-cycle kernels --",
                  b"// ------------------------------------- coarse steps with x in shared memory --")


def kernel_source_hash():
    """Short hash of the solve's row kernels: the V-cycle kernel section of
    solve.cu (between its two section markers; the whole file if they are
    missing) and solve_internal.cuh.  A DRAM-traffic figure measured on
    other kernel source no longer applies; host-side edits elsewhere in
    solve.cu leave it valid."""
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2508_17517_gb300", "csrc")
    with open(os.path.join(d, "solve.cu"), "rb") as fh:
        src = fh.read()
    i0, i1 = src.find(KERNEL_SECTION[0]), src.find(KERNEL_SECTION[1])
    h.update(src[i0:i1] if 0 <= i0 < i1 else src)
    with open(os.path.join(d, "solve_internal.cuh"), "rb") as fh:
        h.update(fh.read())
    return h.hexdigest()[:12]


def measured_traffic(workload, kind, level, alg_bytes=None):
    """DRAM bytes per launch of a (kind, level) group from the committed ncu
    summary (profiles/coarse_newton_traffic.md), taken on the current kernel
    source and on the same operator (algorithmic bytes per launch within 1%
    of `alg_bytes` when given); (bytes, source hash) or (None, reason)."""
    path = os.path.join(ROOT, "profiles", "coarse_newton_traffic.md")
    src = kernel_source_hash()
    if not os.path.exists(path):
        return None, "no ncu traffic summary"
    for line in open(path):
        cells = [c.strip() for c in line.strip().strip("|").split("|")]
        if len(cells) >= 8 and cells[0] == workload and cells[1] == kind and cells[2] == str(level):
            if cells[3] != src:
                return None, "ncu traffic was measured on kernel source %s, not the current %s" % (cells[3], src)
            try:
                alg, traffic = float(cells[5]), float(cells[6])
            except ValueError:
                return None, "unreadable traffic entry"
            if alg_bytes is not None and abs(alg - alg_bytes) > 0.01 * alg_bytes:
                return None, ("ncu traffic was measured on an operator of %.4g algorithmic bytes per launch, "
                              "not the current %.4g" % (alg, alg_bytes))
            return traffic, src
    return None, "no ncu traffic entry for this kernel group and workload"


def solve_timed(G, torch, h, b, x, rtol, flush, steps, label="timed"):
    """`steps` solves from x0 = 0, L2 flushed before each; device time of
    each solve by CUDA events on the launching stream.  Returns (total ms,
    iterations per solve, kernel launches, last info)."""
    stream = torch.cuda.current_stream()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    total_ms, its, launches, info = 0.0, [], 0, None
    torch.cuda.nvtx.range_push(label)     # lets a profiler take the timed solves alone
    for _ in range(steps):
        flush.zero_()
        x.zero_()
        ev0.record(stream)
        _, info = G.airg_solve(h, b, x, rtol=rtol)
        ev1.record(stream)
        ev1.synchronize()
        total_ms += ev0.elapsed_time(ev1)
        its.append(info.iterations)
        launches += info.kernel_launches
        assert info.converged and info.rel_residual <= rtol, (info.converged, info.rel_residual)
    torch.cuda.nvtx.range_pop()
    return total_ms, its, launches, info


def roofline_groups(G, torch, h, b, x, rtol, flush, levels):
    """Pass 1: every solve kernel timed with its own event pair (one solve);
    ranks the (kind, level) groups.  Per-kernel events inflate the small
    kernels, so these shares only rank."""
    G.airg_profile(h, True)
    flush.zero_()
    x.zero_()
    G.airg_solve(h, b, x, rtol=rtol)
    torch.cuda.synchronize()
    prof = G.airg_profile_read(h)
    per_level = G.airg_profile_read_level(h, levels)
    G.airg_profile(h, False)
    return prof, per_level


def group_timed(G, torch, h, b, x, rtol, flush, steps, kind, level, levels):
    """Pass 2: only the launches of one (kind, level) group are timed (one
    event pair per V-cycle for a V-cycle group).  Returns the group's (ms,
    launches, bytes, flops) over `steps` solves and the ms per solve of that
    instrumented pass."""
    G.airg_profile_group(h, kind, level)
    tot, _, _, _ = solve_timed(G, torch, h, b, x, rtol, flush, steps, label="group timing")
    per = G.airg_profile_read_level(h, levels).get((kind, level))
    G.airg_profile(h, False)
    return per, tot / steps


def dominant_group(per_level):
    """The (kind, level) group with the largest time of the ranking pass."""
    return max(per_level.items(), key=lambda kv: kv[1][0])[0]


def roofline_from(prof, per_level, group, steps, ms_per_step, inst_ms, peak, peak_kind, vcycle_dtype="f64"):
    """Roofline entry of one kernel group (host logic).  prof / per_level:
    the ranking pass (per kind; per (kind, level): ms, launches, bytes[,
    flops]); group: (ms, launches, bytes, flops) of the dominant group timed
    alone over `steps` solves; ms_per_step: the uninstrumented solve time;
    inst_ms: the solve time of the pass that timed the group.  The group's
    arithmetic intensity I (flops / algorithmic byte) decides the bound: HBM
    when peak_BW * I is below the arithmetic peak of its precision, else the
    ALU (the FP64 rate of this part is low enough to bind the FP64 dot
    products).  `share` = the group's device time per solve over
    ms_per_step."""
    kinds = {k: v for k, v in prof.items() if v[1] > 0}
    tot = sum(v[0] for v in kinds.values())
    dk, dl = dominant_group(per_level)
    ms, nl, nb, nf = group
    dtype = vcycle_dtype if dk in VCYCLE_KINDS else "f64"
    gbs = nb / (ms / 1e3) / 1e9
    tflops = nf / (ms / 1e3) / 1e12
    fpeak = ALU_PEAK_TFLOPS[dtype]
    intensity = nf / nb if nb else 0.0
    alu_bound = peak * 1e9 * intensity > fpeak * 1e12
    top = sorted(per_level.items(), key=lambda kv: -kv[1][0])[:8]
    entry = {"kernel": "%s (level %d)" % (dk, dl), "dtype": dtype,
             "launches": nl, "avg_launch_us": 1e3 * ms / nl, "algorithmic_bytes_per_launch": nb / nl,
             "flops_per_launch": nf / nl,
             "share": (ms / steps) / ms_per_step,
             "group_ms_per_step": ms / steps,
             "timing": "group timed alone with CUDA events (one pair per V-cycle), %d solves; "
                       "that pass ran at %.3f ms per solve against %.3f uninstrumented"
                       % (steps, inst_ms, ms_per_step),
             "hbm": {"achieved": gbs, "peak": peak, "unit": "GB/s", "frac": gbs / peak},
             "alu": {"achieved": tflops, "peak": fpeak, "unit": "TFLOP/s", "frac": tflops / fpeak,
                     "peak_source": "unit counts x nominal clock"},
             "ranking_pass": {
                 "note": "one solve with an event pair around every kernel (inflates small kernels)",
                 "kernel_share": {k: round(v[0] / tot, 4) for k, v in kinds.items()},
                 "top_launch_groups": [{"kernel": k, "level": l, "share": round(v[0] / tot, 4),
                                        "gbs": round(v[2] / (v[0] / 1e3) / 1e9, 1),
                                        "avg_us": round(1e3 * v[0] / v[1], 2)} for (k, l), v in top]}}
    if alu_bound:
        entry.update({"bound": "alu", "achieved": tflops, "peak": fpeak, "unit": "TFLOP/s",
                      "frac": tflops / fpeak, "peak_source": "unit counts x nominal clock"})
    else:
        entry.update({"bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s", "frac": gbs / peak,
                      "peak_source": peak_kind})
    return entry


def roofline_entry(G, torch, h, b, x, rtol, flush, steps, levels, ms_per_step, peak, peak_kind,
                   vcycle_dtype="f64", workload_key=None):
    """Roofline of the dominant kernel group of a solve: ranked by one
    per-kernel-event solve, then timed alone over `steps` solves."""
    prof, per_level = roofline_groups(G, torch, h, b, x, rtol, flush, levels)
    dk, dl = dominant_group(per_level)
    group, inst_ms = group_timed(G, torch, h, b, x, rtol, flush, steps, dk, dl, levels)
    entry = roofline_from(prof, per_level, group, steps, ms_per_step, inst_ms, peak, peak_kind, vcycle_dtype)
    traffic, src = (measured_traffic(workload_key, dk, dl, entry["algorithmic_bytes_per_launch"])
                    if workload_key else (None, "not captured"))
    entry["traffic"] = traffic
    if traffic is not None:
        entry["traffic_source"] = ("ncu dram__bytes_read.sum + dram__bytes_write.sum per launch "
                                   "(kernel source %s)" % src)
    else:
        entry["traffic_source"] = src
    return entry


def _dist_setup(torch):
    rank, world, local_rank = dist_env()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    return rank, world, local_rank, dev


def _barrier(world, torch):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()


def _dist_end(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()


def e2e_timed(G, torch, h, b, rtol, flush, steps):
    """Seconds of `steps` solves through the C ABI with pinned host buffers:
    the copies of b and x in and of x out are inside the call."""
    bh = b.cpu().pin_memory()
    xh = torch.zeros_like(bh).pin_memory()
    G.airg_solve(h, bh, xh, rtol=rtol)     # warm-up of the host path (staging buffers)
    torch.cuda.synchronize()
    e2e_s = 0.0
    for _ in range(steps):
        flush.zero_()
        torch.cuda.synchronize()
        xh.zero_()
        t0 = time.perf_counter()
        G.airg_solve(h, bh, xh, rtol=rtol)
        e2e_s += time.perf_counter() - t0
    return e2e_s


def row_kernel_choices(G, h):
    """What the setup's per-operator timing picked, one short string per
    operator the solve keeps: warps per slice (w), slices per warp or loads
    in flight per lane (r), own or resident grid, index and value bytes per
    entry ('+base': 16-bit offsets from each slice's smallest column)."""
    out = {}
    for lev, name, d in G.airg_row_kernel_choices(h):
        out["L%d %s" % (lev, name)] = "%dw r%d %s i%d%s v%d, %d rows x %.1f" % (
            d["warps_per_slice"], d["r"], "resident" if d["resident_grid"] else "own", d["index_bytes"],
            "+base" if d["slice_bases"] else "", d["value_bytes"], d["n_rows"],
            d["nnz"] / max(d["n_rows"], 1))
    return out


def hierarchy_entry(sinfo, G=None, h=None):
    e = {"levels": sinfo["levels"], "coarse_rows": sinfo["n"][-1],
         "cycle_complexity": sinfo["cycle_complexity"], "storage_complexity": sinfo["storage_complexity"],
         "vcycle_algorithmic_bytes": sinfo["bytes_per_vcycle"],
         "setup_ms": sinfo["setup_ms"],
         "setup_breakdown_ms": {k: round(v, 2) for k, v in sinfo["setup_breakdown_ms"].items()},
         "setup_exact_dots": sinfo["exact_dots"]}
    if h is not None:
        e["row_kernels"] = row_kernel_choices(G, h)
    return e


def run_gpu(args):
    """One single-problem workload (c1, c2, c3_fp64, c3_fp32, c3_bf16, c4a...)."""
    import torch
    rank, world, local_rank, dev = _dist_setup(torch)
    import paper_2508_17517_gb300 as G
    from synthetic import workload
    G.lib()
    w = workload(SINGLE[args.workload], n=args.grid)
    k = w["n_rhs"]
    n = w["nx"] * w["ny"]
    prob, b = problem_and_rhs(w, G, torch)
    opts = G.airg_options_default(**w["opts"])
    torch.cuda.nvtx.range_push("setup")
    h = G.airg_setup(prob["rowptr"], prob["col"], prob["val"], opts)
    torch.cuda.nvtx.range_pop()
    sinfo = G.airg_setup_info(h)
    x = torch.zeros_like(b)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    for _ in range(args.warmup):
        x.zero_()
        G.airg_solve(h, b, x, rtol=w["rtol"])
    clk = Clocks(local_rank)
    _barrier(world, torch)
    clk.start()
    t_wall0 = time.perf_counter()
    total_ms, its, launches, _ = solve_timed(G, torch, h, b, x, w["rtol"], flush, args.steps)
    _barrier(world, torch)
    wall_s = time.perf_counter() - t_wall0
    clocks = clk.stop()
    t_max = max_over_ranks(total_ms, world, dev)
    value = world * n * k * args.steps / (t_max / 1e3)
    e2e_max = max_over_ranks(e2e_timed(G, torch, h, b, w["rtol"], flush, args.steps), world, dev)
    e2e = {"value": world * n * k * args.steps / e2e_max, "unit": "DOF/s",
           "h2d_bytes_per_step": 2 * 8 * n * k, "d2h_bytes_per_step": 8 * n * k}
    peak, peak_kind = measured_peaks()
    vdt = "f32" if w["opts"].get("precision", 0) in (1, 2) else "f64"
    roofline = roofline_entry(G, torch, h, b, x, w["rtol"], flush, args.steps, sinfo["levels"],
                              t_max / args.steps, peak, peak_kind, vdt,
                              args.workload if args.grid is None else "%s@%d" % (args.workload, args.grid))
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline_entry(args)
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "DOF/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": t_max / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": {0: "f64", 1: "f32/f64", 2: "bf16/f32/f64"}[w["opts"].get("precision", 0)],
            "data": "synthetic",
            "config": {"workload": w["desc"], "n": n, "nrhs": k, "rtol": w["rtol"],
                       "l2": "flushed (256 MiB write) between timed steps"},
            "parallelism": "replicas" if world > 1 else "single",
            "iterations_per_solve": statistics.median(its),
            # DOFs x V-cycles per second, the paper's per-V-cycle rate (Sec. 3.2)
            "dofs_per_s_per_vcycle": value * statistics.median(its),
            "hierarchy": hierarchy_entry(sinfo, G, h),
            "e2e": e2e, "roofline": roofline, "cpu_baseline": cpu, "clocks": clocks,
            "gpu_launches": launches, "wall_s_timed": wall_s,
        }
        print(json.dumps(line))
    _dist_end(world)


def rel_err(a, b):
    import torch
    return float(torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b))


def run_gpu_pair(args):
    """The metric's own comparison on the 4096^2 workload: the FP64 V-cycle
    solve (`value`) against the FP32 V-cycle (`mixed`) and FP32 with a
    bfloat16 restrictor (`mixed_bf16r`), all inside the FP64 outer
    iteration, on the same operator and right-hand side, each to rtol 1e-10
    in the true FP64 residual."""
    import torch
    rank, world, local_rank, dev = _dist_setup(torch)
    import paper_2508_17517_gb300 as G
    from synthetic import workload
    G.lib()
    arms = [("value", workload("c3_fp64")), ("mixed", workload("c3")), ("mixed_bf16r", workload("c3_bf16"))]
    w = arms[0][1]
    n = w["nx"] * w["ny"]
    rtol = w["rtol"]
    prob, b = problem_and_rhs(w, G, torch)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    peak, peak_kind = measured_peaks()
    res = {}
    clk = Clocks(local_rank)
    clk_started = False
    for key, wa in arms:
        h = G.airg_setup(prob["rowptr"], prob["col"], prob["val"], G.airg_options_default(**wa["opts"]))
        sinfo = G.airg_setup_info(h)
        x = torch.zeros_like(b)
        for _ in range(args.warmup):
            x.zero_()
            G.airg_solve(h, b, x, rtol=rtol)
        _barrier(world, torch)
        if not clk_started:
            clk.start()
            clk_started = True
        t_wall0 = time.perf_counter()
        total_ms, its, launches, info = solve_timed(G, torch, h, b, x, rtol, flush, args.steps)
        _barrier(world, torch)
        wall_s = time.perf_counter() - t_wall0
        t_max = max_over_ranks(total_ms, world, dev)
        e2e_max = max_over_ranks(e2e_timed(G, torch, h, b, rtol, flush, args.steps), world, dev)
        vdt = "f32" if wa["opts"].get("precision", 0) in (1, 2) else "f64"
        roof = roofline_entry(G, torch, h, b, x, rtol, flush, args.steps, sinfo["levels"], t_max / args.steps,
                              peak, peak_kind, vdt, {"value": "c3_fp64", "mixed": "c3_fp32",
                                                     # bf16 R changes no coarse operator: the FP32
                                                     # captures apply where the operator's bytes match
                                                     "mixed_bf16r": "c3_fp32"}[key])
        x.zero_()
        _, info = G.airg_solve(h, b, x, rtol=rtol)
        res[key] = dict(value=world * n * args.steps / (t_max / 1e3), ms=t_max / args.steps,
                        its=statistics.median(its), launches=launches, wall_s=wall_s, x=x.clone(),
                        rel_residual=info.rel_residual, hier=hierarchy_entry(sinfo, G, h), roofline=roof,
                        e2e=world * n * args.steps / e2e_max)
        G.airg_free(h)
        del x
        torch.cuda.empty_cache()
    clocks = clk.stop()
    x64 = res["value"]["x"]
    cpu, exact = None, None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline_entry(args)
        u, sv, sts = cpu_exact(w, repeats=1)
        ut = torch.tensor(u, device=dev)
        exact = {k: rel_err(r["x"], ut) for k, r in res.items()}
        exact["sweep"] = {"value": sv, "unit": "DOF/s", "cores": 1, "seconds": sts,
                          "kind": "exact substitution in upwind order (serial; context, not a baseline)"}
    if rank == 0:
        v = res["value"]

        def arm(key):
            r = res[key]
            return {"value": r["value"], "unit": "DOF/s", "dtype": {"mixed": "f32/f64", "mixed_bf16r": "bf16/f32/f64"}[key],
                    "ms_per_step": r["ms"], "iterations_per_solve": r["its"],
                    "speedup_vs_fp64": r["value"] / v["value"],
                    "rel_residual": r["rel_residual"],
                    "rel_err_vs_fp64_solution": rel_err(r["x"], x64),
                    "rel_err_vs_exact": exact[key] if exact else None,
                    "e2e": {"value": r["e2e"], "unit": "DOF/s"},
                    "gpu_launches": r["launches"], "hierarchy": r["hier"], "roofline": r["roofline"]}
        line = {
            "metric": METRIC, "value": v["value"], "unit": "DOF/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": v["ms"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": w["desc"], "n": n, "nrhs": 1, "rtol": rtol,
                       "l2": "flushed (256 MiB write) between timed steps"},
            "parallelism": "replicas" if world > 1 else "single",
            "iterations_per_solve": v["its"], "dofs_per_s_per_vcycle": v["value"] * v["its"],
            "rel_residual": v["rel_residual"],
            "rel_err_vs_exact": exact["value"] if exact else None,
            "hierarchy": v["hier"],
            "e2e": {"value": v["e2e"], "unit": "DOF/s", "h2d_bytes_per_step": 16 * n, "d2h_bytes_per_step": 8 * n},
            "roofline": v["roofline"],
            "mixed": arm("mixed"), "mixed_bf16r": arm("mixed_bf16r"),
            "cpu_baseline": cpu, "clocks": clocks, "gpu_launches": v["launches"], "wall_s_timed": v["wall_s"],
        }
        if exact:
            line["context_sweep"] = exact["sweep"]
        print(json.dumps(line))
    _dist_end(world)


def _sweep_row(G, torch, prob, b, opts, args):
    """Setup then median device time of `steps` solves to rtol 1e-10."""
    stream = torch.cuda.current_stream()
    t0 = time.perf_counter()
    h = G.airg_setup(prob["rowptr"], prob["col"], prob["val"], opts)
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t0
    info = G.airg_setup_info(h)
    x = torch.zeros_like(b)
    for _ in range(args.warmup):
        x.zero_()
        G.airg_solve(h, b, x, rtol=1e-10)
    times, its = [], []
    for _ in range(args.steps):
        x.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        _, si = G.airg_solve(h, b, x, rtol=1e-10)
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
        its.append(si.iterations)
    solve_ms = statistics.median(times)
    nit = statistics.median(its)
    return {"levels": info["levels"], "coarse_rows": info["n"][-1], "truncated": info["truncated"],
            "grid_complexity": round(sum(info["n"]) / info["n"][0], 3),
            "cycle_complexity": round(info["cycle_complexity"], 2),
            "storage_complexity": round(info["storage_complexity"], 2),
            "setup_s": round(setup_s, 3), "iterations": nit, "solve_ms": round(solve_ms, 3),
            "ms_per_iteration": round(solve_ms / max(nit, 1), 3),
            "dof_per_s_per_vcycle": info["n"][0] * nit / (solve_ms / 1e3)}


def run_sweep(args):
    """One GPU, theta = pi/4 on a 4096^2 grid (16.8M DOFs, the per-GPU size
    class of the paper's studies), inflow g = 1, smoother order 6, rtol 1e-10.
    coarse-order (Sec. 3.1): m_c in {5, 10, 30, 100} with truncation at
    alpha_trunc = 0.1 on every level vs no truncation, FP64.  smoother
    (Sec. 2.2): the matrix-free GMRES polynomial vs the assembled
    fixed-sparsity matrix of Eq. 8, F-point vs FC and FCF smoothing
    (Sec. 2, Sec. 3.3.2), and the GMRES (AIRG) vs Neumann (nAIR, Sec.
    3.3.1) polynomial, FP64 and FP32 V-cycles, m_c = 30 with truncation at
    1e-2.  Solve times are the median of `steps` device-timed
    solves after `warmup` untimed ones."""
    import torch
    torch.cuda.set_device(0)
    import paper_2508_17517_gb300 as G
    G.lib()
    if args.sweep == "cases":
        run_cases(G, torch, args)
        return
    if args.sweep == "readings":
        run_readings(G, torch, args)
        return
    n = 4096
    th = math.pi / 4
    vx, vy = math.cos(th), math.sin(th)
    prob = G.airg_problem_advection2d(n, n, vx, vy)
    g = torch.ones(prob["inflow"].numel(), dtype=torch.float64, device="cuda")
    b = G.airg_assemble_rhs_advection2d(prob, g)
    rows = []
    if args.sweep == "coarse-order":
        for mc in (5, 10, 30, 100):
            for trunc in (0.1, 0.0):
                r = _sweep_row(G, torch, prob, b, G.airg_options_default(coarse_poly_order=mc, trunc_rtol=trunc), args)
                rows.append(dict({"coarse_order": mc, "truncation": trunc}, **r))
    else:
        P, A, GM, NE = G.AIRG_SMOOTH_POLYNOMIAL, G.AIRG_SMOOTH_ASSEMBLED, G.AIRG_INVERSE_GMRES, G.AIRG_INVERSE_NEUMANN
        settings = [(P, G.AIRG_SMOOTH_F, GM), (A, G.AIRG_SMOOTH_F, GM), (P, G.AIRG_SMOOTH_FC, GM),
                    (P, G.AIRG_SMOOTH_FCF, GM), (A, G.AIRG_SMOOTH_FC, GM), (P, G.AIRG_SMOOTH_F, NE)]
        for prec in (G.AIRG_FP64, G.AIRG_MIXED_FP32):
            for sm, stype, inv in settings:
                opts = G.airg_options_default(coarse_poly_order=30, trunc_rtol=1e-2, precision=prec, smoother=sm,
                                              smooth_type=stype, inverse_type=inv)
                r = _sweep_row(G, torch, prob, b, opts, args)
                rows.append(dict({"precision": "f64" if prec == G.AIRG_FP64 else "f32",
                                  "smoother": "polynomial" if sm == P else "assembled",
                                  "points": ("f", "fc", "fcf")[stype],
                                  "inverse": "gmres (AIRG)" if inv == GM else "neumann (nAIR)"},
                                 **r))
    print(json.dumps({"sweep": args.sweep, "grid": "%dx%d" % (n, n), "theta": "pi/4", "g": 1.0,
                      "rtol": 1e-10, "steps": args.steps, "warmup": args.warmup, "rows": rows}))


def run_readings(G, torch, args):
    """Which reading of the unstated parameters drives the cycle complexity:
    the R drop tolerance r_drop (reading R8) and DDC on / off (ddc_its 2 /
    0, reading R4) on the 1024^2 workload (seeded direction, m_c = 30,
    truncation 1e-2; with --grid N, the N^2 grid of the 4096^2 workload's
    family as well), FP64, rtol 1e-10.  Each row splits the
    cycle complexity into the part of the levels (restriction, residual,
    smoother) and that of the coarse Newton polynomial, whose SpMVs on the
    coarsest operator are counted from its roots (a real root one SpMV, a
    conjugate pair two, the last root one less)."""
    from synthetic import velocity, workload
    rows = []
    for name in ("c2", "c3_fp64") if args.grid else ("c2",):
        w = workload(name, n=args.grid if name == "c3_fp64" else None)
        vx, vy = velocity(w["theta"])
        prob = G.airg_problem_advection2d(w["nx"], w["ny"], vx, vy)
        b = G.airg_assemble_rhs_advection2d(prob, torch.tensor(w["g"][0], device="cuda"))
        for ddc in (2, 0):
            # from the largest tolerance down; r_drop = 0 (no drop) fills the
            # coarse operators so much that a 1024^2 setup did not finish in 30 min
            for rd in (5e-2, 2e-2, 1e-2, 5e-3):
                opts = dict(w["opts"], r_drop=rd, ddc_its=ddc)
                t0 = time.perf_counter()
                h = G.airg_setup(prob["rowptr"], prob["col"], prob["val"], G.airg_options_default(**opts))
                torch.cuda.synchronize()
                setup_s = time.perf_counter() - t0
                info = G.airg_setup_info(h)
                L = info["levels"] - 1
                roots = G.airg_export_vector(h, L, 3).reshape(-1, 2)
                nsp = sum((0 if i + 1 == len(roots) else 1) if im == 0.0 else (1 if i + 1 == len(roots) else 2)
                          for i, (_, im) in enumerate(roots))
                cc_coarse = nsp * info["nnz_a"][L] / info["nnz_a"][0]
                x = torch.zeros_like(b)
                times, its = [], []
                for k in range(args.warmup + args.steps):
                    x.zero_()
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record()
                    _, si = G.airg_solve(h, b, x, rtol=1e-10)
                    e1.record()
                    e1.synchronize()
                    if k >= args.warmup:
                        times.append(e0.elapsed_time(e1))
                        its.append(si.iterations)
                rows.append({"workload": name, "r_drop": rd, "ddc_its": ddc, "levels": info["levels"],
                             "coarse_rows": info["n"][L],
                             "coarse_nnz_per_row": round(info["nnz_a"][L] / max(info["n"][L], 1), 1),
                             "cycle_complexity": round(info["cycle_complexity"], 2),
                             "cc_coarse": round(cc_coarse, 2),
                             "cc_levels": round(info["cycle_complexity"] - cc_coarse, 2),
                             "storage_complexity": round(info["storage_complexity"], 2),
                             "iterations": statistics.median(its), "solve_ms": round(statistics.median(times), 3),
                             "setup_s": round(setup_s, 2)})
                G.airg_free(h)
        del prob, b
        torch.cuda.empty_cache()
    print(json.dumps({"sweep": "readings", "rtol": 1e-10, "steps": args.steps, "warmup": args.warmup,
                      "rows": rows}))


def run_cases(G, torch, args):
    """The paper's two other single-direction studies at one GPU's share:
    the hard direction v = (sqrt(2/3), sqrt(1/3)) with strong threshold 0.4
    on 2896^2 (Sec. 3.3.2), and the 500 x 26000 rectangle at theta = pi/4
    with coarse order 10 (Sec. 3.4).  FP64, g = 1, s = 0, rtol 1e-10."""
    from synthetic import velocity, workload
    rows = []
    for name in ("hard", "rect"):
        w = workload(name)
        vx, vy = velocity(w["theta"])
        prob = G.airg_problem_advection2d(w["nx"], w["ny"], vx, vy)
        b = G.airg_assemble_rhs_advection2d(prob, torch.tensor(w["g"][0], device="cuda"))
        r = _sweep_row(G, torch, prob, b, G.airg_options_default(**w["opts"]), args)
        rows.append(dict({"case": name, "workload": w["desc"]}, **r))
        del prob, b
        torch.cuda.empty_cache()
    print(json.dumps({"sweep": "cases", "rtol": 1e-10, "steps": args.steps, "warmup": args.warmup,
                      "rows": rows}))


def main(argv=None):
    args = parse(argv)
    if args.sweep:
        run_sweep(args)
    elif args.impl == "reference":
        run_reference(args)
    elif args.workload == "c4b":
        run_gpu_multi(args)
    elif args.workload == "c3":
        run_gpu_pair(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
