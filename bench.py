"""Benchmark: RVE realizations per second (both correctors + A_hom each).

Workload (the method at scale): L = 32 unit cells per axis, h = 1/16
(512 x 512 nodes, 262,144 unknowns per corrector), contrast 10, 717 square
inclusions of side 1 (density 0.7), PCG to a true relative residual of 1e-10,
seeded synthetic realizations (seed 0, indices 0..999 cycled).  One step =
field generation + both corrector solves + A_hom for a batch of B
realizations (default 1000: the whole seeded set of the workload in one
step) through the C ABI, mixed precision (FP32 stencil / transforms /
vectors, FP64 dots and true-residual refinement, double-word A_hom).  The
per-step working set (~17 GB at B = 1000) is far larger than L2.

Timing: K steps between CUDA events on the launching stream (the headline
`value`, no per-launch instrumentation); the same K steps again with every
pipeline launch bracketed by CUDA events give the per-kernel times of the
roofline; `e2e` runs K steps through rve_homogenize_host (host descriptors
in, host A_hom out).  Also reported: the FP64 fused path and the plain FP64
path on a small sample, the oracle on the host cores (all cores, and one
thread), and the per-entry A_hom error of the first 125 realizations of the
first timed batch against the FP64 oracle.  The batched form rides along:
`uneven_4096` holds a short run (at most 4 steps) of the uneven workload
below, the same object `--workload uneven_4096` prints in full.

    python bench.py [--gpus N --steps K --warmup W --batch B] [--impl reference]
    python bench.py --workload cubes_L4    # the 3D extension (one JSON line too)
    python bench.py --workload uneven_4096 # 4096 uneven realizations, persistent + graph
    python bench.py --workload large_L256  # 2048^2, contrast 100, mixed; statistics
    python bench.py --workload adjoint_L64 # 1024^2, contrast 100, FP64, A_hom + gradient

The 3D workload (`--workload cubes_L4`): L = 4, h = 1/16 (64^3 nodes), 45
unit cubes (density 0.7 per unit volume), contrast 10, three correctors per
realization by the mixed-precision 3D solver to a true relative residual of
1e-10, 3x3 A_hom; one step = field + correctors + A_hom for 256
realizations (67 M nodes, ~17 GB of state).

The uneven workload (`--workload uneven_4096`): 4096 realizations with L
drawn from {8, 16, 32, 64} at h = 1/8 and contrast from {10, 100}; one step
= one execution of a captured plan (field, the correctors' fused kernels in
a conditional while node, A_hom), tile shapes from the autotuner; the same
plan as one persistent launch is timed beside it.
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

METRIC = "RVE realizations/s (2 correctors each) at ≤1e-7 A_hom rel. error; HBM % of peak"
UNIT = "realizations/s"
WORKLOAD = dict(name="plain_L32", L=32, m0=16, contrast=10.0, tol=1e-10, realizations=1000)
CONFIG_DESC = ("L=32, h=1/16 (512x512 nodes, 262144 unknowns per corrector), contrast 10, "
               "717 inclusions of side 1 (density 0.7), PCG tol 1e-10 on the true residual")

# Algorithmic bytes per node (both correctors, float2 = 8 B per node pair) of
# the fused pipeline kernels, per realization-step.  ITER: S reads zhat,
# p_old, x and writes p_new, q, x; U reads rt (the row transform of r) and q
# and writes rt; C reads rt and writes zhat.  REFINE: R reads u (double word,
# 16 B), x, p and writes q; U reads u, x, p, q and writes u, x, rt; C as in
# ITER.  The coefficient bitmask adds 1/8 B per node to R and S.
BYTES_PER_NODE = {
    "refine": {"iter": 0.0, "refine": 16 + 8 + 8 + 8 + 0.125},
    "stencil": {"iter": 6 * 8 + 0.125, "refine": 0.0},
    "update_row": {"iter": 3 * 8, "refine": 16 + 8 + 8 + 8 + 16 + 8 + 8},
    "column": {"iter": 2 * 8, "refine": 2 * 8},
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=8)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--batch", type=int, default=None,
                    help="realizations per step and GPU (default: the workload's own)")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="plain_L32",
                    choices=["plain_L32", "cubes_L4", "uneven_4096", "large_L256", "adjoint_L64"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the FP64 comparison arms")
    return ap.parse_args()


def descs(start: int, count: int):
    from paper_1903_12227_gb300 import workloads
    return [workloads.realization(WORKLOAD["L"], WORKLOAD["m0"], WORKLOAD["contrast"], 0,
                                  (start + k) % WORKLOAD["realizations"]) for k in range(count)]


# ----------------------------------------------------------------- clocks --
class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self, index: int):
        import tempfile
        self.index = index
        self.proc = None
        # samples go to a temporary file; their summary goes into the JSON line
        self.path = os.path.join(tempfile.gettempdir(), f"rve_bench_clocks_{os.getpid()}_{index}.csv")

    def start(self):
        os.makedirs(os.path.dirname(self.path), exist_ok=True)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index),
                 "--query-gpu=index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as fh:
            lines = fh.readlines()
        try:
            os.remove(self.path)
        except OSError:
            pass
        for line in lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for name, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------ CPU oracle --
def cpu_oracle_rate(indices, threads: int = 0):
    """Oracle (as it stands) on the host cores for the given realization
    indices: realizations/s, threads used, A, seconds."""
    import oracle
    from paper_1903_12227_gb300 import workloads
    ds = [workloads.realization(WORKLOAD["L"], WORKLOAD["m0"], WORKLOAD["contrast"], 0, int(k))
          for k in indices]
    t0 = time.perf_counter()
    A, it, used = oracle.solve_batch(ds, tol=WORKLOAD["tol"], threads=threads)
    dt = time.perf_counter() - t0
    return len(ds) / dt, used, A, dt


def per_entry_error(A, ref):
    """Error of A [N,2,2] against ref per entry (a11, a12, a21, a22), each
    |dA_ij| / max(|ref_11|, |ref_22|) of its realization: max and mean."""
    import numpy as np
    A = np.asarray(A).reshape(-1, 2, 2)
    ref = np.asarray(ref).reshape(-1, 2, 2)
    sc = np.maximum(np.abs(ref[:, 0, 0]), np.abs(ref[:, 1, 1]))[:, None]
    e = (np.abs(A - ref).reshape(-1, 4)) / sc
    return {"entries": ["a11", "a12", "a21", "a22"], "max": e.max(axis=0).tolist(),
            "mean": e.mean(axis=0).tolist(), "max_all": float(e.max()), "count": int(len(A))}


# Thread instructions per node of the double-word true-residual pass
# (k_fused_R): ncu instruction count of a refining launch divided by its
# nodes, for the first refinement of a solve (r = f) and the later ones
# (profiles/k_fused_R_refine_plain_L32_32copies.md).
REFINE_INST_PER_NODE = 485.4
REFINE_FIRST_INST_PER_NODE = 95.9


def refine_alu(prof, refines, reals, nodes, clk):
    """Instruction-issue roofline of the double-word true-residual pass: its
    thread instructions (per node, measured by ncu, times the nodes of the
    refinements run) over its CUDA-event time, against 152 SMs x 4 schedulers
    x 32 lanes x the measured SM clock."""
    launches = prof["refine"]["launches"]
    if launches == 0 or refines == 0:
        return None
    # every step launches the refine kernel; only refining realizations work
    # in it, and idle launches return at once (their time is included)
    ms = prof["refine"]["ms"]
    mhz = clk.get("sm_mhz") or 2070.0
    peak_inst = 152 * 4 * 32 * mhz * 1e6   # thread instructions/s
    work = nodes * (REFINE_INST_PER_NODE * (refines - reals) + REFINE_FIRST_INST_PER_NODE * reals)
    return {"bound": "alu", "unit": "thread instructions/s",
            "inst_per_node": REFINE_INST_PER_NODE,
            "inst_per_node_first": REFINE_FIRST_INST_PER_NODE,
            "achieved": work / (ms / 1e3), "peak": peak_inst,
            "frac": work / (ms / 1e3) / peak_inst,
            "peak_source": "152 SMs x 4 schedulers x 32 lanes x measured SM clock",
            "note": "time includes the idle launches of non-refining steps"}


def graph_plan(args, rve, torch, np, dev, stream, ds, A_first):
    """K executions of a plan of the first timed batch (field + solve + A_hom
    captured once as a CUDA graph, the solve as the fused kernels in a
    conditional while node), timed like `value`."""
    opts = rve.make_opts(precision=rve.MIXED, tol=WORKLOAD["tol"], path=rve.PATH_FUSED)
    plan = rve.Plan(ds, opts, device=dev)
    for _ in range(args.warmup):
        plan.execute()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        A, _ = plan.execute()
    ev1.record(stream)
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    diff = float(np.abs(A.cpu().numpy().reshape(-1, 4) - A_first.cpu().numpy().reshape(-1, 4)).max())
    plan.close()
    return {"value": len(ds) * args.steps / (ms / 1e3), "unit": UNIT,
            "ms_per_step": ms / args.steps, "a_hom_max_abs_diff_vs_value_path": diff,
            "api": "rve_plan_create / rve_plan_execute (one CUDA graph per step, no host "
                   "synchronisation inside the solve)"}


def e2e_host(args, rve, torch, dev):
    """End to end through rve_homogenize_host over the same K steps: host
    descriptors copied in, field + solve + A_hom, A_hom and the solver report
    copied back to host memory, every step inside the timed region."""
    B = args.batch
    opts = rve.make_opts(precision=rve.MIXED, tol=WORKLOAD["tol"])
    b0 = rve.Batch(descs(0, B))
    ws_h = rve.workspace(rve.lib().rve_homogenize_workspace_size(b0.ptr, b0.count,
                                                                 rve.ctypes.byref(opts)), dev)
    for k in range(args.warmup):
        rve.homogenize_host(descs(B * k, B), opts, ws=ws_h)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(args.steps):
        rve.homogenize_host(descs(B * (args.warmup + k), B), opts, ws=ws_h)
    dt = time.perf_counter() - t0
    del ws_h
    return {"value": args.steps * B / dt, "unit": UNIT,
            "h2d_bytes_per_step": B * 48, "d2h_bytes_per_step": B * (32 + 40),
            "api": "rve_homogenize_host (host descriptors in, host A_hom and solver report out)",
            "steps": args.steps}


def run_reference(args):
    """The oracle arm: each step solves one realization per host thread."""
    import oracle
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    oracle.build()
    cores = os.cpu_count() or 1
    per_step = cores
    times = []
    used = cores
    for k in range(args.warmup + args.steps):
        ds = descs(k * per_step, per_step)
        t0 = time.perf_counter()
        _, _, used = oracle.solve_batch(ds, tol=WORKLOAD["tol"], threads=cores)
        dt = time.perf_counter() - t0
        if k >= args.warmup:
            times.append(dt)
    total = sum(times)
    value = per_step * args.steps / total
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "impl": "reference",
           "config": {"workload": f"{WORKLOAD['name']}: {CONFIG_DESC}",
                      "realizations_per_step": per_step},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": used, "kind": "oracle",
                            "sample": f"{per_step} realizations per step (one per host thread)"},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


# -------------------------------------------------------------- GPU arm --
# The translation unit of the fused 2D pipeline kernels and the headers it
# includes: the recorded DRAM traffic stays valid while these are unchanged.
PIPELINE_SOURCES = ("rve_solver.cu", "rve_colsolve.cuh", "rve_common.cuh", "rve_device.cuh",
                    "rve_internal.h")


def source_hash() -> str:
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1903_12227_gb300", "csrc")
    for f in PIPELINE_SOURCES:
        h.update(open(os.path.join(csrc, f), "rb").read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel: str):
    """Per-node DRAM traffic of `kernel` from the committed ncu summary, if it
    was measured on the current sources (else None)."""
    path = os.path.join(ROOT, "profiles", "dram_traffic_k_fused_S_U_C_plain_L32_batch128.json")
    try:
        rec = json.load(open(path))
    except (OSError, ValueError):
        return None
    if rec.get("source_hash") != source_hash():
        return None
    return rec.get("bytes_per_node", {}).get(kernel)


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0}, "fallback"


def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_1903_12227_gb300 import rve

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream()
    B = args.batch
    opts = rve.make_opts(precision=rve.MIXED, tol=WORKLOAD["tol"])
    # each rank owns its own realization indices (weak scaling, no collective
    # on the data path)
    base = rank * B * (args.steps + args.warmup)
    probe = rve.Batch(descs(0, B))
    ws = rve.workspace(rve.workspace_size(probe, opts), dev)
    mask = torch.empty(probe.words, dtype=torch.int32, device=dev)
    u = torch.empty(probe.nodes, 2, dtype=torch.float64, device=dev)
    info = torch.empty(B * rve.INFO_BYTES, dtype=torch.uint8, device=dev)
    nb_hom = rve.workspace_size(probe, rve.make_opts())
    ws_hom = ws if ws.numel() >= nb_hom else rve.workspace(nb_hom, dev)
    A_out = torch.empty(B, 4, dtype=torch.float64, device=dev)
    L = rve.lib()

    def step(k: int):
        b = rve.Batch(descs(base + k * B, B))
        rve.check(L.rve_gen_field(b.ptr, b.count, rve._ptr(mask), rve._stream(stream)))
        rve.check(L.rve_solve_correctors(b.ptr, b.count, rve._ptr(mask), None,
                                         rve.ctypes.byref(opts), rve._ptr(u), rve._ptr(info),
                                         rve._ptr(ws), ws.numel(), rve._stream(stream)))
        rve.check(L.rve_a_hom(b.ptr, b.count, rve._ptr(mask), None, opts.scheme, opts.precision,
                              rve._ptr(u), rve._ptr(A_out), None, None, rve._ptr(ws_hom),
                              ws_hom.numel(), rve._stream(stream)))
        return b

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
            torch.cuda.synchronize()

    for k in range(args.warmup):
        step(k)
    barrier()

    def timed_loop(first: int, profile: bool):
        """K steps between CUDA events on the launching stream (barrier and
        synchronize on both sides); returns (ms, launches, infos, As, clocks)."""
        rve.launch_count()
        rve.profile_enable(profile)
        rve.profile_read()
        clocks = Clocks(local)
        clocks.start()
        infos, As = [], []
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier()
        ev0.record(stream)
        for k in range(args.steps):
            step(first + k)
            infos.append(info.clone())
            As.append(A_out.clone())
        ev1.record(stream)
        barrier()
        clk = clocks.stop()
        prof = rve.profile_read() if profile else None
        rve.profile_enable(False)
        return ev0.elapsed_time(ev1), rve.launch_count(), infos, As, clk, prof

    # the headline: plain timed steps, no per-launch profiling events
    t0 = time.perf_counter()
    elapsed_ms, launches, infos, As, clk, _ = timed_loop(args.warmup, False)
    wall = time.perf_counter() - t0
    # the same steps again with every pipeline launch bracketed by events:
    # the per-kernel times of the roofline
    prof_ms, _, pinfos, _, _, prof = timed_loop(args.warmup, True)
    if world > 1:
        t = torch.tensor([elapsed_ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        elapsed_ms = float(t.item())
    total_real = B * args.steps * world
    value = total_real / (elapsed_ms / 1e3)

    info_d = [d for t in infos for d in rve.info_to_dicts(t, B)]
    pinfo_d = [d for t in pinfos for d in rve.info_to_dicts(t, B)]
    A_all = torch.cat(As).cpu().numpy().reshape(-1, 2, 2)
    statuses = sorted({d["status"] for d in info_d})
    nodes = 512 * 512

    # roofline of the dominant fused kernel (CUDA events on the launching
    # stream over the profiled repeat): algorithmic bytes / average launch
    peaks, peak_src = measured_peaks()
    peak = float(peaks.get("hbm_gbs", 6800.0))
    steps_iter = sum(d["steps"] for d in pinfo_d)
    refines = sum(d["refinements"] for d in pinfo_d)

    def kernel_rate(kind):
        bpn = BYTES_PER_NODE[kind]
        alg = nodes * (steps_iter * bpn["iter"] + refines * bpn["refine"])
        nl = max(prof[kind]["launches"], 1)
        avg_s = prof[kind]["ms"] / 1e3 / nl
        return alg / nl, avg_s, (alg / nl) / avg_s / 1e9 if avg_s > 0 else 0.0

    dom = max(("stencil", "update_row", "column"), key=lambda k: prof[k]["ms"])
    bytes_per_launch, avg_launch_s, achieved = kernel_rate(dom)
    tr = ncu_traffic(dom)   # per node of an ITER step
    launches_dom = max(prof[dom]["launches"], 1)
    traffic = None if tr is None else tr * nodes * steps_iter / launches_dom
    # the refine pass is bound by FP32 issue, not HBM: its operation count
    # per node against the FP32 rate of the measured clock
    rk = refine_alu(prof, refines, len(pinfo_d), nodes, clk)
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": traffic, "kernel": dom,
                "peak_source": f"hbm_gbs of {peak_src}", "bytes_per_launch": bytes_per_launch,
                "avg_launch_us": avg_launch_s * 1e6,
                "per_kernel_gbs": {k: kernel_rate(k)[2] for k in BYTES_PER_NODE},
                "per_kernel_frac": {k: kernel_rate(k)[2] / peak for k in BYTES_PER_NODE},
                "refine_alu": rk,
                "profiled_ms_per_step": prof_ms / args.steps,
                "time_share": {k: prof[k]["ms"] / max(sum(prof[j]["ms"] for j in prof), 1e-9)
                               for k in prof}}

    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": elapsed_ms / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f32 vectors + f64 dots/refinement/A_hom (mixed)", "data": "synthetic",
           "config": {"workload": f"{WORKLOAD['name']}: {CONFIG_DESC}", "batch_per_gpu": B,
                      "realizations_per_step": B * world, "l2": "inputs larger than L2 "
                      f"(~{B * 262144 * 64 / 1e9:.0f} GB working set per step, 129 MB L2)",
                      "precision": "mixed"},
           "roofline": roofline, "gpu_launches": launches,
           "clocks": clk,
           "solver": {"statuses": statuses,
                      "mean_steps": sum(d["steps"] for d in info_d) / len(info_d),
                      "mean_iters": float(np.mean([max(d["iters"]) for d in info_d])),
                      "mean_refinements": sum(d["refinements"] for d in info_d) / len(info_d),
                      "max_relres": float(max(max(d["relres"]) for d in info_d))},
           "a_hom_stats": {"mean": A_all.mean(axis=0).tolist(),
                           "var": A_all.var(axis=0, ddof=1).tolist(), "count": len(A_all)},
           "wall_s": wall}
    if rank == 0:
        # end to end through the host-buffer entry point over the same K steps
        out["e2e"] = e2e_host(args, rve, torch, dev)
    if world == 1:
        # the same step as one captured CUDA graph (rve_plan_execute): the
        # solve's fused kernels inside a conditional while node, so the host
        # never waits on the device between steps
        out["graph_plan"] = graph_plan(args, rve, torch, np, dev, stream,
                                       descs(base + args.warmup * B, B), As[0])

    if rank == 0 and not args.no_extras:
        out.update(extras(args, rve, torch, np, dev, stream))
        if "fp64_plain" in out:
            out["speedup_vs_fp64_plain"] = value / out["fp64_plain"]["value"]
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # the oracle on the realizations of the first timed batch: the first
        # 32 timed on all host cores (the baseline), the rest for the
        # per-entry error of the mixed path against the FP64 oracle
        first = [(args.warmup * B + k) % WORKLOAD["realizations"] for k in range(min(B, 125))]
        k0 = min(32, B)
        rate, cores, A_cpu, dt = cpu_oracle_rate(first[:k0])
        out["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
                               "sample": f"{k0} realizations (indices {first[0]}..{first[k0 - 1]}) "
                                         f"of the same workload, one per host thread ({dt:.1f} s)"}
        rate1, _, _, dt1 = cpu_oracle_rate(first[:1], threads=1)
        out["cpu_baseline_1thread"] = {"value": rate1, "unit": UNIT, "cores": 1, "kind": "oracle",
                                       "sample": f"1 realization (index {first[0]}), one thread "
                                                 f"({dt1:.1f} s)"}
        if len(first) > k0:
            _, _, A_rest, _ = cpu_oracle_rate(first[k0:])
            A_cpu = np.concatenate([A_cpu, A_rest])
        A_gpu = As[0].cpu().numpy().reshape(-1, 2, 2)[:len(first)]
        out["a_hom_err_vs_oracle"] = per_entry_error(A_gpu, A_cpu)
        out["a_hom_err_vs_oracle"]["sample"] = (f"{len(first)} realizations (the first of the "
                                                f"first timed batch), mixed precision vs the "
                                                f"FP64 oracle")
    if world == 1 and not args.no_extras:
        # the batched form beside the headline: 4096 uneven realizations, one
        # captured graph per step (tiles from the autotuner), and the same
        # plan as one persistent launch; a few steps (the full line is
        # --workload uneven_4096)
        sub = argparse.Namespace(steps=min(args.steps, 4), warmup=3,
                                 no_cpu_baseline=args.no_cpu_baseline)
        try:
            un = uneven_line(sub)
            out["uneven_4096"] = {k: un[k] for k in (
                "value", "unit", "steps", "warmup", "ms_per_step", "config", "roofline",
                "persistent_plan", "e2e", "solver", "clocks", "cpu_baseline",
                "a_hom_err_vs_oracle") if k in un}
        except Exception as exc:   # reported, not hidden: the headline stands
            out["uneven_4096"] = {"error": f"{type(exc).__name__}: {exc}"}
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


CUBES = dict(name="cubes_L4", L=4, m0=16, contrast=10.0, tol=1e-10, batch=256)
CUBES_METRIC = "3D RVE realizations/s (3 correctors each, mixed precision, true residual <= 1e-10)"
CUBES_DESC = ("L=4, h=1/16 (64^3 nodes, 262144 unknowns per corrector), contrast 10, 45 unit "
              "cubes (density 0.7), PCG tol 1e-10 on the true residual, 3x3 A_hom")
# Algorithmic bytes per unit-node (a unit = one corrector pair of a
# realization) of one launch of each 3D kernel kind in the mixed solve:
# FP32 stencil 17 (x, cells, y); line pass 18 on average (16, the last of
# four also reads r); z solve 16; vector steps 36 on average (axpy 48, xpby
# 24); true residual in double words 81 (the split of u into double words:
# u in, 16-byte words out; the residual pass: words, f, cells in, r out).
CUBES_BYTES = {"stiffness": 17.0, "lines": 18.0, "zsolve": 16.0, "vector": 36.0, "scalar": 0.0,
               "resid64": 81.0}


def cubes_descs(start: int, count: int):
    from paper_1903_12227_gb300 import workloads
    return [workloads.realization3(CUBES["L"], CUBES["m0"], CUBES["contrast"], 0, start + k)
            for k in range(count)]


def cpu_oracle_rate_cubes(count: int):
    """The 3D oracle as it stands, one realization per host thread (the C
    oracle runs with the GIL released): realizations/s, threads, A."""
    import concurrent.futures as cf

    import numpy as np

    import oracle
    oracle.build()
    ds = cubes_descs(0, count)
    t0 = time.perf_counter()
    with cf.ThreadPoolExecutor(max_workers=count) as ex:
        res = list(ex.map(lambda d: oracle.solve_realization3(d, tol=CUBES["tol"], want_u=False), ds))
    dt = time.perf_counter() - t0
    return count / dt, count, np.array([r["A_energy"] for r in res]), dt


def run_cubes(args):
    """The 3D extension: batches of 64^3 realizations through the rve3 C ABI."""
    import numpy as np
    import torch

    from paper_1903_12227_gb300 import rve, rve3

    if int(os.environ.get("WORLD_SIZE", "1")) > 1:
        raise SystemExit("--workload cubes_L4 runs on one GPU")
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", "0")))
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream()
    B = args.batch or CUBES["batch"]
    opts = rve3.make_opts3(precision=rve.MIXED, tol=CUBES["tol"])
    probe = rve3.Batch3(cubes_descs(0, B))
    L3 = rve3.lib()
    ws = rve.workspace(rve3.workspace_size3(probe), dev)
    mask = torch.empty(probe.nodes, dtype=torch.uint8, device=dev)
    u = torch.empty(probe.nodes, 3, dtype=torch.float64, device=dev)
    info = torch.empty(B * rve3.INFO3_BYTES, dtype=torch.uint8, device=dev)
    A_out = torch.empty(B, 9, dtype=torch.float64, device=dev)

    def step(k: int):
        b = rve3.Batch3(cubes_descs(k * B, B))
        s = rve._stream(stream)
        rve.check(L3.rve3_gen_field(b.ptr, b.count, rve._ptr(mask), s))
        rve.check(L3.rve3_solve_correctors(b.ptr, b.count, rve._ptr(mask), None,
                                           rve3.ctypes.byref(opts), rve._ptr(u), rve._ptr(info),
                                           rve._ptr(ws), ws.numel(), s))
        rve.check(L3.rve3_a_hom(b.ptr, b.count, rve._ptr(mask), None, opts.scheme, rve._ptr(u),
                                rve._ptr(A_out), None, rve._ptr(ws), ws.numel(), s))

    for k in range(args.warmup):
        step(k)
    torch.cuda.synchronize()
    rve.launch_count()
    rve.profile_enable(True)
    rve3.profile_read()
    clocks = Clocks(dev.index)
    clocks.start()
    infos, As = [], []
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record(stream)
    for k in range(args.steps):
        step(args.warmup + k)
        infos.append(info.clone())
        As.append(A_out.clone())
    ev1.record(stream)
    torch.cuda.synchronize()
    elapsed_ms = ev0.elapsed_time(ev1)
    clk = clocks.stop()
    prof = rve3.profile_read()
    rve.profile_enable(False)
    launches = rve.launch_count()
    value = B * args.steps / (elapsed_ms / 1e3)
    info_d = [d for t in infos for d in rve3.decode_info(t)]
    A_all = torch.cat(As).cpu().numpy().reshape(-1, 3, 3)

    # roofline of the dominant kernel kind: algorithmic bytes of the unit-
    # nodes its launches worked on / the average CUDA-event launch time; a
    # launch covers every unit, but blocks of converged units return at once,
    # so the unit-nodes are the units' CG steps (FP32 stencil launches) x n^3
    n3 = (CUBES["L"] * CUBES["m0"]) ** 3
    unit_steps = sum(max(d["iters"][0], d["iters"][1]) + d["iters"][2] for d in info_d)
    peaks, peak_src = measured_peaks()
    peak = float(peaks.get("hbm_gbs", 6800.0))

    def rate(kind, unit_nodes):
        ms, cnt = prof[kind]
        if cnt == 0 or ms <= 0:
            return 0.0, 0.0, 0.0
        per_launch = CUBES_BYTES[kind] * unit_nodes / cnt
        avg_s = ms / 1e3 / cnt
        return per_launch, avg_s, per_launch / avg_s / 1e9

    # unit-node counts per kind: one stencil, four line passes, one z solve,
    # two vector launches per unit CG step
    per_kind_nodes = {"stiffness": unit_steps * n3, "lines": 4 * unit_steps * n3,
                      "zsolve": unit_steps * n3, "vector": 2 * unit_steps * n3, "scalar": 0,
                      "resid64": sum(max(d["refinements"] - 2, 0) for d in info_d) * n3}
    dom = max(("stiffness", "lines", "zsolve", "vector"), key=lambda k: prof[k][0])
    bpl, avg_s, achieved = rate(dom, per_kind_nodes[dom])
    total_ms = max(sum(v[0] for v in prof.values()), 1e-9)
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": None, "kernel": dom,
                "peak_source": f"hbm_gbs of {peak_src}", "bytes_per_launch": bpl,
                "avg_launch_us": avg_s * 1e6,
                "per_kernel_gbs": {k: rate(k, per_kind_nodes[k])[2] for k in CUBES_BYTES},
                "time_share": {k: prof[k][0] / total_ms for k in prof}}
    out = {"metric": CUBES_METRIC, "value": value, "unit": UNIT, "n_gpus": 1,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": elapsed_ms / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f32 vectors + f64 dots/refinement/A_hom (mixed)", "data": "synthetic",
           "config": {"workload": f"{CUBES['name']}: {CUBES_DESC}", "batch_per_gpu": B,
                      "l2": "inputs larger than L2 (~17 GB of state per step)",
                      "precision": "mixed"},
           "roofline": roofline, "gpu_launches": launches, "clocks": clk,
           "solver": {"statuses": sorted({d["status"] for d in info_d}),
                      "mean_iters": float(np.mean([np.mean(d["iters"]) for d in info_d])),
                      "mean_refinements": float(np.mean([d["refinements"] for d in info_d])),
                      "max_relres": float(max(max(d["relres"]) for d in info_d))},
           "a_hom_stats": {"mean_diag": float(np.mean(A_all.diagonal(axis1=1, axis2=2))),
                           "std_diag": float(np.std(A_all.diagonal(axis1=1, axis2=2))),
                           "count": len(A_all)}}
    # end to end: host descriptors in, host A_hom out, the copies in the timing
    t0 = time.perf_counter()
    n_e2e = 2
    for k in range(n_e2e):
        step(args.warmup + args.steps + k)
        A_host = A_out.cpu()
    dt = time.perf_counter() - t0
    out["e2e"] = {"value": n_e2e * B / dt, "unit": UNIT, "h2d_bytes_per_step": B * 48,
                  "d2h_bytes_per_step": B * 72,
                  "api": "rve3_gen_field + rve3_solve_correctors + rve3_a_hom (host descriptors, "
                         "A_hom copied to the host)"}
    del A_host
    if not args.no_cpu_baseline:
        cores = min(os.cpu_count() or 1, 16)
        rate_cpu, used, A_cpu, dt = cpu_oracle_rate_cubes(cores)
        out["cpu_baseline"] = {"value": rate_cpu, "unit": UNIT, "cores": used, "kind": "oracle",
                               "sample": f"{used} realizations (indices 0..{used - 1}) of the same "
                                         f"workload, one per host thread ({dt:.1f} s)"}
        # the same realizations on the GPU, against the oracle
        ds = cubes_descs(0, used)
        m = rve3.gen_field(ds, device=dev)
        ug, _ = rve3.solve(ds, mask=m, opts=opts)
        Ag = rve3.a_hom(ds, ug, mask=m).cpu().numpy()
        sc = np.abs(A_cpu.diagonal(axis1=1, axis2=2)).max(axis=1)
        out["a_hom_max_rel_err_vs_oracle"] = float((np.abs(Ag - A_cpu).max(axis=(1, 2)) / sc).max())
    print(json.dumps(out), flush=True)


UNEVEN_DESC = ("4096 realizations, L uniform in {8,16,32,64}, h=1/8 (64^2 .. 512^2 nodes), "
               "contrast uniform in {10,100}, round(0.7 L^2) inclusions of side 1, "
               "mixed precision, PCG tol 1e-10 on the true residual; the whole pipeline (field, "
               "solve, A_hom) as one captured CUDA graph per step, autotuned tiles")


def run_uneven(args):
    print(json.dumps(uneven_line(args)), flush=True)


def uneven_line(args) -> dict:
    """The batched form: thousands of realizations of uneven size in one
    persistent launch under a CUDA graph, tile shapes from the autotuner."""
    import numpy as np
    import torch

    from paper_1903_12227_gb300 import rve, workloads

    if int(os.environ.get("WORLD_SIZE", "1")) > 1:
        raise SystemExit("--workload uneven_4096 runs on one GPU")
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", "0")))
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream()
    ds = workloads.config_batch("uneven_4096", seed=0)
    B = len(ds)

    def timed_plan(path):
        """Autotune, capture, W untimed and K timed executions of a plan."""
        opts = rve.make_opts(precision=rve.MIXED, path=path, tol=1e-10)
        rve.tuner_clear()
        rve.autotune(ds[:256], opts, device=dev)
        plan = rve.Plan(ds, opts, device=dev)
        for _ in range(args.warmup):
            plan.execute()
        torch.cuda.synchronize()
        rve.launch_count()
        clocks = Clocks(dev.index)
        clocks.start()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        ev0.record(stream)
        for _ in range(args.steps):
            A, info = plan.execute()
        ev1.record(stream)
        torch.cuda.synchronize()
        ms = ev0.elapsed_time(ev1)
        clk = clocks.stop()
        launches = rve.launch_count()
        tiles = {str(n): rve.tuner_lookup(n, rve.MIXED, path == rve.PATH_PERSISTENT)
                 for n in (64, 128, 256, 512)}
        A, info_d = A.cpu().numpy(), rve.info_to_dicts(info, B)
        plan.close()
        return ms, clk, launches, A, info_d, tiles, opts

    # the persistent kernel (one cooperative launch per solve) for comparison
    ms_p, clk_p, _, A_p, info_p, tiles_p, _ = timed_plan(rve.PATH_PERSISTENT)
    # the headline: the fused kernels inside the graph's conditional loop
    elapsed_ms, clk, launches, A, info_d, tiles, opts = timed_plan(rve.PATH_FUSED)
    value = B * args.steps / (elapsed_ms / 1e3)
    # kernels that ran per execution: the captured ones once, the loop body
    # (4 steps x 5 kernels + the re-arming kernel) once per group of steps
    groups = -(-max(x["steps"] + x["refinements"] for x in info_d) // 4)
    launches += args.steps * (groups - 1) * 21
    # roofline: the algorithmic bytes of the solve (per realization n^2 x (CG
    # steps x 88.125 + refinements x 120.125)) over the time of one plan
    # execution (field and A_hom included: a lower bound on the solve's rate)
    iter_b = BYTES_PER_NODE["stencil"]["iter"] + BYTES_PER_NODE["update_row"]["iter"] + \
        BYTES_PER_NODE["column"]["iter"]
    ref_b = BYTES_PER_NODE["refine"]["refine"] + BYTES_PER_NODE["update_row"]["refine"] + \
        BYTES_PER_NODE["column"]["refine"]

    def alg_of(infos):
        return sum((d["L"] * d["m0"]) ** 2 * (x["steps"] * iter_b + x["refinements"] * ref_b)
                   for d, x in zip(ds, infos))
    alg = alg_of(info_d)
    per_exec_s = elapsed_ms / 1e3 / args.steps
    peaks, peak_src = measured_peaks()
    peak = float(peaks.get("hbm_gbs", 6800.0))
    achieved = alg / per_exec_s / 1e9
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": elapsed_ms / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f32 vectors + f64 dots/refinement/A_hom (mixed)", "data": "synthetic",
           "config": {"workload": f"uneven_4096: {UNEVEN_DESC}", "realizations_per_step": B,
                      "l2": "inputs larger than L2 (~5 GB working set per step)",
                      "precision": "mixed", "plan": "fused kernels in a conditional while node",
                      "tiles": tiles},
           "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                        "frac": achieved / peak, "traffic": None,
                        "kernel": "whole plan execution (fused pipeline kernels in the graph loop)",
                        "peak_source": f"hbm_gbs of {peak_src}", "bytes_per_launch": alg,
                        "avg_launch_us": per_exec_s * 1e6},
           "persistent_plan": {"value": B * args.steps / (ms_p / 1e3), "unit": UNIT,
                               "ms_per_step": ms_p / args.steps, "clocks": clk_p,
                               "tiles": tiles_p,
                               "roofline_frac": alg_of(info_p) / (ms_p / 1e3 / args.steps) / 1e9 / peak,
                               "a_hom_max_abs_diff_vs_loop_plan": float(np.abs(A_p - A).max()),
                               "note": "one cooperative persistent launch per solve"},
           "gpu_launches": launches, "clocks": clk,
           "solver": {"statuses": sorted({x["status"] for x in info_d}),
                      "mean_steps": float(np.mean([x["steps"] for x in info_d])),
                      "mean_refinements": float(np.mean([x["refinements"] for x in info_d])),
                      "max_relres": float(max(max(x["relres"]) for x in info_d))}}
    # end to end: host descriptors in, host A_hom out, same path and options
    ws_h = rve.workspace(rve.lib().rve_homogenize_workspace_size(
        rve.Batch(ds).ptr, B, rve.ctypes.byref(opts)), dev)
    rve.homogenize_host(ds, opts, ws=ws_h)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        rve.homogenize_host(ds, opts, ws=ws_h)
    dt = time.perf_counter() - t0
    out["e2e"] = {"value": args.steps * B / dt, "unit": UNIT, "h2d_bytes_per_step": B * 48,
                  "d2h_bytes_per_step": B * (32 + 40),
                  "api": "rve_homogenize_host on the fused path (host descriptors in, host "
                         "A_hom and solver report out; the host polls convergence)"}
    del ws_h
    if not args.no_cpu_baseline:
        # one realization per (L, contrast) pair against the FP64 oracle; the
        # same ones time the oracle on the host cores
        import oracle
        picks = {}
        for k, d in enumerate(ds):
            picks.setdefault((d["L"], d["a_incl"]), k)
        ks = [picks[key] for key in sorted(picks)]
        t0 = time.perf_counter()
        A_cpu, _, used = oracle.solve_batch([ds[k] for k in ks], tol=1e-12)
        dt = time.perf_counter() - t0
        out["cpu_baseline"] = {"value": len(ks) / dt, "unit": UNIT, "cores": used, "kind": "oracle",
                               "sample": f"{len(ks)} realizations, one per (L, contrast) pair, "
                                         f"one per host thread ({dt:.1f} s)"}
        err = per_entry_error(A[ks], A_cpu)
        err["sample"] = "one realization per (L, contrast) pair, mixed vs FP64 oracle (tol 1e-12)"
        out["a_hom_err_vs_oracle"] = err
    return out


def _single_gpu(name):
    import torch
    if int(os.environ.get("WORLD_SIZE", "1")) > 1:
        raise SystemExit(f"--workload {name} runs on one GPU")
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", "0")))
    torch.cuda.set_device(dev)
    return dev, torch.cuda.current_stream()


def _events_loop(torch, stream, fn, steps, warmup, index):
    """W untimed and K timed calls of fn(k) between CUDA events, with the
    clock record of the timed region."""
    for k in range(warmup):
        fn(k)
    torch.cuda.synchronize()
    clocks = Clocks(index)
    clocks.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record(stream)
    outs = [fn(warmup + k) for k in range(steps)]
    ev1.record(stream)
    torch.cuda.synchronize()
    return ev0.elapsed_time(ev1), clocks.stop(), outs


def run_large(args):
    """Large RVE statistics: L = 256, h = 1/8 (2048^2 nodes), contrast 100,
    density 0.7, mixed precision; one step = field + both correctors + A_hom
    for a batch of 16 realizations; the mixed results of the first batch
    against the FP64 GPU path, and the ensemble statistics (mean, variance,
    quartic tensor) of all timed realizations."""
    import numpy as np
    import torch

    from paper_1903_12227_gb300 import rve, workloads
    dev, stream = _single_gpu("large_L256")
    B = args.batch or 16
    opts = rve.make_opts(precision=rve.MIXED, tol=1e-10)
    probe = workloads.config_batch("large_L256", seed=0, count=B)
    ws = rve.workspace(rve.workspace_size(probe, opts), dev)
    rve.launch_count()

    def step(k):
        ds = workloads.config_batch("large_L256", seed=0, count=B, start=(k * B) % 256)
        mask = rve.gen_field(ds, device=dev)
        u, info = rve.solve(ds, mask=mask, opts=opts, ws=ws)
        return rve.a_hom(ds, u, mask=mask, precision=rve.MIXED), info

    ms, clk, outs = _events_loop(torch, stream, step, args.steps, args.warmup, dev.index)
    launches = rve.launch_count()
    A = torch.cat([o[0] for o in outs]).cpu().numpy()
    info_d = [d for o in outs for d in rve.info_to_dicts(o[1], B)]
    del ws
    # mixed against FP64 on two realizations of the first timed batch
    ds2 = workloads.config_batch("large_L256", seed=0, count=2, start=(args.warmup * B) % 256)
    m2 = rve.gen_field(ds2, device=dev)
    u64, i64 = rve.solve(ds2, mask=m2, opts=rve.make_opts(precision=rve.FP64, tol=1e-10))
    A64 = rve.a_hom(ds2, u64, mask=m2).cpu().numpy()
    err = per_entry_error(A[:2], A64)
    err["sample"] = "2 realizations of the first timed batch, mixed vs the FP64 GPU path"
    st = rve.statistics(A, 256.0)
    out = {"metric": METRIC, "value": B * args.steps / (ms / 1e3), "unit": UNIT, "n_gpus": 1,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f32 vectors + f64 dots/refinement/A_hom (mixed)", "data": "synthetic",
           "config": {"workload": "large_L256: L=256, h=1/8 (2048x2048 nodes, 4.2M unknowns per "
                                  "corrector), contrast 100, 45875 inclusions of side 1 (density "
                                  "0.7), PCG tol 1e-10 on the true residual",
                      "realizations_per_step": B, "precision": "mixed",
                      "l2": "inputs larger than L2 (~4 GB working set per step)"},
           "gpu_launches": launches, "clocks": clk,
           "solver": {"statuses": sorted({d["status"] for d in info_d}),
                      "mean_steps": float(np.mean([d["steps"] for d in info_d])),
                      "mean_refinements": float(np.mean([d["refinements"] for d in info_d])),
                      "max_relres": float(max(max(d["relres"]) for d in info_d))},
           "a_hom_err_vs_fp64": err,
           "statistics": {"count": int(len(A)), "mean": st["mean"].tolist(),
                          "var": st["var"].tolist(), "Q": st["Q"].tolist(),
                          "L2_var_a12": float(256.0 ** 2 * st["var"][0, 1])},
           "cpu_baseline": None,
           "cpu_baseline_note": "the oracle needs minutes per 2048^2 contrast-100 realization "
                                "on one host thread: no bounded sample"}
    print(json.dumps(out), flush=True)


def run_adjoint(args):
    """Adjoint: L = 64, h = 1/16 (1024^2 nodes), contrast 100, FP64 solve to
    1e-13; one step = AHom forward (field, both correctors, A_hom) and
    backward (dA/da per cell for a random 2x2 weight) for 16 realizations."""
    import numpy as np
    import torch

    from paper_1903_12227_gb300 import rve, workloads
    dev, stream = _single_gpu("adjoint_L64")
    B = args.batch or 16
    opts = rve.make_opts(precision=rve.FP64, tol=1e-13)
    G = torch.tensor(np.random.default_rng(4).standard_normal((B, 2, 2)), device=dev)
    rve.launch_count()

    def step(k):
        ds = workloads.config_batch("adjoint_L64", seed=0, count=B, start=(k * B) % 64)
        b = rve.Batch(ds)
        mask = rve.gen_field(b, device=dev)
        coef = rve.coef_from_mask(b, mask).requires_grad_(True)
        A = rve.AHom.apply(coef, b, opts)
        (A * G).sum().backward()
        return A.detach(), coef.grad

    ms, clk, outs = _events_loop(torch, stream, step, args.steps, args.warmup, dev.index)
    launches = rve.launch_count()
    A = torch.cat([o[0] for o in outs])
    out = {"metric": METRIC, "value": B * args.steps / (ms / 1e3), "unit": UNIT, "n_gpus": 1,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f64", "data": "synthetic",
           "config": {"workload": "adjoint_L64: L=64, h=1/16 (1024x1024 nodes), contrast 100, "
                                  "2867 inclusions, FP64 solve to 1e-13, A_hom and its gradient "
                                  "per cell (autograd Function, hand-written adjoint kernel)",
                      "realizations_per_step": B, "precision": "fp64",
                      "l2": "inputs larger than L2 (~2 GB working set per step)"},
           "gpu_launches": launches, "clocks": clk,
           "a_hom_mean_diag": float(A.diagonal(dim1=1, dim2=2).mean().item()),
           "cpu_baseline": None,
           "cpu_baseline_note": "the oracle needs minutes per 1024^2 contrast-100 realization at "
                                "tol 1e-13 on one host thread: no bounded sample"}
    print(json.dumps(out), flush=True)


def extras(args, rve, torch, np, dev, stream):
    """The FP64 comparison arms and the mixed-vs-FP64 agreement."""
    out = {}
    opts = rve.make_opts(precision=rve.MIXED, tol=WORKLOAD["tol"])
    # FP64 fused and plain FP64 paths on a small sample
    for name, o, cnt in (("fp64_fused", rve.make_opts(precision=rve.FP64, tol=WORKLOAD["tol"]), 16),
                         ("fp64_plain", rve.make_opts(precision=rve.FP64, path=rve.PATH_PLAIN,
                                                      tol=WORKLOAD["tol"]), 4)):
        ds = descs(0, cnt)
        mask = rve.gen_field(ds, device=dev)
        ws = rve.workspace(rve.workspace_size(ds, o), dev)
        rve.solve(ds, mask=mask, opts=o, ws=ws)   # warm
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        mask = rve.gen_field(ds, device=dev)
        u, info = rve.solve(ds, mask=mask, opts=o, ws=ws)
        A = rve.a_hom(ds, u, mask=mask, precision=rve.FP64)
        e1.record(stream)
        torch.cuda.synchronize()
        out[name] = {"value": cnt / (e0.elapsed_time(e1) / 1e3), "unit": UNIT,
                     "sample": f"{cnt} realizations",
                     "mean_iters": float(np.mean([max(d["iters"]) for d in rve.info_to_dicts(info, cnt)]))}
        if name == "fp64_fused":
            fp64_A = A.cpu().numpy()
        del ws
    # accuracy of mixed vs FP64 (GPU) on the same 16 realizations
    m16 = rve.gen_field(descs(0, 16), device=dev)
    u16, _ = rve.solve(descs(0, 16), mask=m16, opts=opts)
    A16 = rve.a_hom(descs(0, 16), u16, mask=m16, precision=rve.MIXED).cpu().numpy()
    out["a_hom_err_mixed_vs_fp64"] = per_entry_error(A16, fp64_A)
    out["a_hom_err_mixed_vs_fp64"]["sample"] = "16 realizations (indices 0..15), GPU FP64 path"

    return out


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    if args.workload == "cubes_L4":
        run_cubes(args)
        return
    if args.workload == "uneven_4096":
        run_uneven(args)
        return
    if args.workload == "large_L256":
        run_large(args)
        return
    if args.workload == "adjoint_L64":
        run_adjoint(args)
        return
    if args.batch is None:
        args.batch = WORKLOAD["realizations"]   # one step = the whole seeded set
    run_ours(args)


if __name__ == "__main__":
    main()
