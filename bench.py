"""Throughput benchmark of the biased neutron history loop on GB300.

Default (one GPU): the powder-diffractometer workload -- 1.5 A beam 1 x 2 cm on
a cylinder r = 0.5 cm, h = 2 cm of a synthetic fcc powder (18 Bragg lines) plus
incoherent scattering, 1 mm can, 3600-bin 2-theta cylinder detector -- with
1e8 histories per step in FP32 transport and FP64 tallies.  A step is one
persistent launch that runs every history through source, flights, boundary
crossings, collisions and scoring.  Beside it, the batched+adjoint workload
(256 powder instances with uneven history counts, score-function gradients
and the backward contraction) is timed, and both are compared at matched
tally error.

Prints one JSON line.  --impl reference times the CPU oracle instead (the
reference arm of this project) on a bounded sample of the same workload."""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time
from pathlib import Path

ROOT = Path(__file__).resolve().parent
sys.path.insert(0, str(ROOT))

METRIC = "histories/s on 1 GB300: plain vs batched+adjoint, at matched tally error"
UNIT = "histories/s"
POWDER_N = 100_000_000
# Thread instructions per history the kernel of the workload's benchmark line
# executes (ncu smsp__inst_executed.sum x active lanes / histories on a small
# case of the same launch): an implementation's count, reported beside the
# algorithmic one below.  Measured for the powder workload's warp-pool kernel.
EXECUTED_INST_PER_HISTORY = {"powder": 4455}
# Algorithmic lane operations of the method per step type, counted from its
# formulas (not from any kernel):
#   every event (biased flight, Eq. eStepLength2, and weight, Eq. eWeight):
#     one Philox4x32-10 block, 10 rounds x (2 mul-hi + 2 mul-lo + 4 xor + 2 key
#     adds) = 100; two uniforms 6; cross sections of the volume (1/v
#     absorption, incoherent, Bragg prefix-sum search over 18 lines, Sigma_t,
#     Sigma_g) 31; step -ln(xi)/Sigma_g 3; move 4; weight exp 3; distance to
#     the next boundary 40 (a tube's exit quadratic ~30, a box's three slabs
#     ~12, plus the world region's bounding-sphere tests) = 187
#   a collision: process choice and weight division 6, isotropic direction 13
#     (a Bragg line adds a second Philox block, two searches and a rotation,
#     ~150, in a minority of collisions) = 40 on average
#   a boundary crossing: nudge, relocation among neighbours and the scorer's
#     bin (angle, atomics) = 40
OPS_PER_EVENT, OPS_PER_COLLISION, OPS_PER_CROSSING = 187, 40, 40


def algorithmic_ops_per_history(counters: dict) -> float:
    h = max(1, counters["histories"])
    return (OPS_PER_EVENT * counters["events"] + OPS_PER_COLLISION * counters["collisions"]
            + OPS_PER_CROSSING * counters["crossings"]) / h


# DRAM bytes of one full-size step of the kernel variant the autotuner picks
# (ncu dram__bytes_read.sum + dram__bytes_write.sum), keyed by (workload,
# variant): powder, the warp-pool launch (measured on 1e7 histories: the
# tables' and tallies' cold misses, which do not grow with the histories);
# batched, the two passes of a queued-secondaries step (measured on 4e6
# histories of the same instance mix and scaled by histories: the queue grows
# with them).
TRAFFIC_PER_LAUNCH = {("powder", 3): 150016, ("batched", 2): 237655727793}
# The tally whose integrated total defines "matched tally error" per workload
# (each history scores it at most once).
FIGURE_TALLY = {"powder": 0, "guide": 0, "imaging": 0, "batched": 0, "slab": 1, "total_scattering": 1,
                "chopper": 2}
# Workloads whose configuration asks for the adjoint: their step is a run with
# the score-function accumulators plus the backward contraction.
GRAD_WORKLOADS = ("batched", "imaging")


def measured_peaks() -> dict:
    """The device's measured rates (tp_measure_peaks): FP32 FMA, integer,
    special-function and FP64 lane rates, FP64 atomics, L2 read bandwidth."""
    from paper_2304_06226_gb300 import native as NN
    return NN.tp_measure_peaks()


def workload_desc(name: str):
    import workloads as W
    if name == "powder":
        return W.powder(n_histories=POWDER_N), "powder diffractometer, 1e8 histories, FP32 transport"
    if name == "guide":
        return W.guide(n_histories=POWDER_N), "supermirror guide 20 m, 1e8 histories, FP32 transport"
    if name == "slab":
        return W.slab(g=3.0, n_histories=1_000_000), "slab, bias 3, 1e6 histories, FP64 transport"
    if name == "imaging":
        return W.imaging(n_histories=1_000_000_000), ("CSG imaging 1000 primitives, 512^2 PSD, 1e9 histories, FP32 "
                                                      "transport, adjoint w.r.t. the 3 material densities")
    if name == "total_scattering":
        return W.total_scattering(n_histories=100_000_000), ("total scattering: pencil on a 1.2 cm fcc-powder sphere, 4 pi "
                                                             "detector, Q per scattering order, 1e8 histories, FP32 transport")
    if name == "chopper":
        return W.chopper(n_histories=POWDER_N), ("disk chopper 4 x 20 deg at 100 Hz, 10 m from a 293 K MaxwellianGun, "
                                                 "TOF before/after, 1e8 histories, FP32 transport")
    if name == "batched":
        return W.batched(), ("256 powder instances, uneven history counts (5.9e8 total), gradients w.r.t. "
                             "radius, scale, density + backward, FP32 transport")
    raise SystemExit(f"unknown workload {name}")


def workload_config(name: str, label: str, extra: dict) -> dict:
    cfg = {"workload": label, "name": name, "l2": "flushed between timed steps (256 MiB write)"}
    cfg.update(extra)
    return cfg


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = Path(os.environ.get("TP_CLOCK_LOG", f"/tmp/tp_clocks_{os.getpid()}.csv"))

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.fh.close()

    def summary(self) -> dict:
        if not self.proc or not self.path.exists():
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.path.read_text().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def flush_l2(buf):
    buf.add_(1.0)


def run_ours(args, rank: int, world: int) -> dict | None:
    import numpy as np
    import torch
    from paper_2304_06226_gb300 import build
    build.build()
    from paper_2304_06226_gb300.engine import Scene
    from paper_2304_06226_gb300 import shard
    import workloads as W

    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", dev))
    desc, label = workload_desc(args.workload)
    grad = args.workload in GRAD_WORKLOADS
    if args.histories:
        if grad:   # keep the instance mix, scale the counts to the requested total
            c = desc["instances"]["counts"].astype(np.float64)
            desc["instances"]["counts"] = np.maximum(1, np.rint(c * args.histories / c.sum())).astype(np.int64)
            label += f" (scaled to {int(desc['instances']['counts'].sum()):.2e} histories)"
        else:
            desc["instances"]["counts"][0] = args.histories
            label = label.replace("1e8 histories", f"{args.histories:.0e} histories")
    n = int(desc["instances"]["counts"].sum())
    sc = Scene(desc)
    bgrad = torch.ones(sc.n_inst, sc.total_bins, dtype=torch.float64, device="cuda") if grad else None
    runs = (lambda st=None: sc.run(want_grad=True, stream=st, kernel=args.kernel, ctas_per_sm=args.ctas_per_sm,
                                   block_size=args.block_size, graph=True, first=first, seed=seed,
                                   secondaries=args.secondaries, stage=args.stage)) if grad else None
    stream = torch.cuda.current_stream()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")   # 256 MiB > L2
    first, seed = 0, None
    n_max = int(np.max(desc["instances"]["counts"]))   # ids per instance and rank

    def step(k, st=None):
        # every step and every rank runs its own histories (weak scaling): the
        # tallies then hold steps x ranks x n distinct histories
        nonlocal first, seed
        seed, first = shard.step_stream(k, rank, world, n_max, sc.seed)
        if grad:
            runs(st)
            sc.backward(bgrad, stream=st)
        else:
            sc.run(n, first=first, seed=seed, stream=st, kernel=args.kernel, ctas_per_sm=args.ctas_per_sm,
                   block_size=args.block_size, stage=args.stage)

    peaks = measured_peaks() if rank == 0 else None
    # ---- warm-up (the library is ahead-of-time compiled; the first run autotunes) ----
    for k in range(args.warmup):
        step(k)
    torch.cuda.synchronize()
    sc.reset()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    with ClockSampler(dev) as clk:
        t0 = time.perf_counter()
        for k in range(args.steps):
            flush_l2(flush)
            ev[k][0].record(stream)
            step(k, stream)
            ev[k][1].record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
    kernel_ms = [a.elapsed_time(b) for a, b in ev]
    dev_s = sum(kernel_ms) / 1e3
    if dist:
        t = torch.tensor([dev_s], device="cuda", dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dev_s = float(t.item())
    counters = sc.counters()
    tot = n * args.steps
    value = world * tot / dev_s
    if dist:
        # one FP64 sum all-reduce of every rank's partial tallies (after the
        # timed steps): rank 0 then holds the statistics of all histories
        sc.allreduce(sc.counts * args.steps if grad else [tot])
    # ---- tally error of the integrated detector total (per history) ----
    q = int(np.argsort(sc.counts)[len(sc.counts) // 2]) if grad else 0   # median-count instance
    raw = sc.raw(q)
    N = float(sc.counts[q] * args.steps * world) if grad else float(tot * world)
    ft = FIGURE_TALLY.get(args.workload, 0)
    lo, hi = sc.tally_off[ft], sc.tally_off[ft + 1]
    mean_tot = raw["sum"][lo:hi].sum() / N
    # rel. standard error of the integrated total: each history hits at most one bin
    var = raw["sumsq"][lo:hi].sum() / N - mean_tot ** 2
    rel_err = math.sqrt(max(var, 0.0) / (N - 1)) / mean_tot
    fom_plain = 1.0 / (rel_err ** 2 * (dev_s / world)) if rel_err > 0 else None

    # ---- end to end through the public API with host buffers ----
    import ctypes as C
    from paper_2304_06226_gb300 import native as NN
    host_mean = np.empty(sc.total_bins)
    host_err = np.empty(sc.total_bins)
    e2e_steps = max(1, min(args.steps, 3))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    host_grad = np.empty((sc.n_inst, max(1, sc.n_par)))
    for k in range(e2e_steps):
        sc.reset()
        seed, first = shard.step_stream(args.warmup + args.steps + k, rank, world, n_max, sc.seed)
        if grad:
            runs()
            g = sc.backward(bgrad)
            host_grad[:, : sc.n_par] = g.cpu().numpy()
        else:
            sc.run(n, first=first, seed=seed, kernel=args.kernel, ctas_per_sm=args.ctas_per_sm,
                   block_size=args.block_size, stage=args.stage)
        for t in range(len(sc.tally_bins)):
            o = sc.tally_off[t]
            NN.tp_read_tallies(sc.handle, t, q, host_mean[o:].ctypes.data, host_err[o:].ctypes.data, False)
    e2e_s = time.perf_counter() - t0
    e2e_value = world * n * e2e_steps / e2e_s
    h2d = 2 * 8 * sc.n_inst + 8          # history counts, first ids, prefix (per run)
    d2h = 2 * 8 * sc.total_bins + (8 * sc.n_inst * sc.n_par if grad else 0)   # means, errors, gradients

    # ---- batched + adjoint ----
    batched = None
    if args.batched and rank == 0 and not grad:
        batched = run_batched(args, W, Scene, torch, peaks)

    if rank != 0:
        return None
    exec_ph = EXECUTED_INST_PER_HISTORY.get(args.workload)
    traffic = TRAFFIC_PER_LAUNCH.get((args.workload, sc.launch()[0])) if not args.histories else None
    clocks = clk.summary()
    peak = peaks["fp32_fma"]
    alg_ph = algorithmic_ops_per_history(counters)
    t_s = sum(kernel_ms) / 1e3
    achieved = alg_ph * tot / t_s
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * dev_s / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32" if sc.precision == "f32" else "f64",
        "data": "synthetic",
        "config": workload_config(args.workload, label, {
            "histories_per_step_per_gpu": n, "tallies": "FP64 sum w, sum w^2 per bin",
            "launch": sc.launch_info(),
            "parallelism": f"history ids sharded over {world} GPU(s), one FP64 all-reduce of the tallies"}),
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "lane-ops/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "per_unit": alg_ph, "per_unit_basis": (
                         f"algorithmic lane operations per history: {OPS_PER_EVENT} per event + "
                         f"{OPS_PER_COLLISION} per collision + {OPS_PER_CROSSING} per crossing, "
                         "weighted by this run's counters"),
                     "peak_basis": (f"measured FP32 FMA lane rate of this GPU (tp_measure_peaks, "
                                    f"{peaks['sm_clock_mhz']:.0f} MHz during the measurement)"),
                     "executed": ({"per_unit": exec_ph, "frac": exec_ph * tot / t_s / peak,
                                   "basis": "thread instructions per history this workload's kernel executes (ncu, "
                                            "small case of the same launch)"}
                                  if exec_ph else None)},
        "peaks": peaks,
        "kernel_ms": kernel_ms,
        "tally": {"figure_tally": ft, "mean_total": mean_tot, "rel_stderr_total": rel_err, "fom": fom_plain,
                  "counters": counters},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        # transport launches of each timed step (+ the backward kernel of gradient runs)
        "gpu_launches": args.steps * (sc.launch_count() + (1 if grad else 0)),
        "clocks": clocks,
    }
    if batched:
        line["batched_adjoint"] = batched
        # matched error: time for each to reach the same relative error eps
        eps = 1e-3
        line["matched_error"] = {
            "eps": eps,
            "plain_s_to_eps": (rel_err / eps) ** 2 * tot / value,
            "batched_s_to_eps_per_instance": batched.get("s_to_eps_per_instance"),
        }
    if args.cpu_baseline and world == 1:
        line["cpu_baseline"] = cpu_baseline(args, desc, n, grad=grad)
    sc.close()
    return line


def run_batched(args, W, Scene, torch, peaks) -> dict:
    """Workload 4: 256 instances, one persistent launch, gradients + backward."""
    desc = W.batched()
    sc = Scene(desc)
    counts = sc.counts
    total = int(counts.sum())
    stream = torch.cuda.current_stream()
    grad = torch.ones(sc.n_inst, sc.total_bins, dtype=torch.float64, device="cuda")
    for _ in range(max(1, args.warmup // 2)):
        sc.run(want_grad=True, graph=True)
    torch.cuda.synchronize()
    sc.reset()
    steps = max(1, args.batched_steps)
    a, b, c = (torch.cuda.Event(enable_timing=True) for _ in range(3))
    fw_ms, bw_ms = [], []
    for k in range(steps):
        a.record(stream)
        # the step's CUDA graph, its own Philox key per step: each step runs distinct histories
        sc.run(want_grad=True, stream=stream, graph=True, seed=sc.seed + 1000 + k)
        b.record(stream)
        sc.backward(grad, stream=stream)
        c.record(stream)
        torch.cuda.synchronize()
        fw_ms.append(a.elapsed_time(b))
        bw_ms.append(b.elapsed_time(c))
    t = (sum(fw_ms) + sum(bw_ms)) / 1e3
    # matched error on the integrated total of a median-count instance
    import numpy as np
    q = int(np.argsort(counts)[len(counts) // 2])
    raw = sc.raw(q)
    N = float(counts[q]) * steps
    m = raw["sum"].sum() / N
    rel = math.sqrt(max(raw["sumsq"].sum() / N - m * m, 0.0) / (N - 1)) / m
    hist_s = total * steps / t
    launch = sc.launch_info()
    launches_per_step = sc.launch_count() + 1   # transport passes + backward
    fw_s = sum(fw_ms) / 1e3
    alg_ph = algorithmic_ops_per_history(sc.counters())
    achieved = alg_ph * total * steps / fw_s
    peak = peaks["fp32_fma"]
    sc.close()
    return {"value": hist_s, "unit": UNIT, "instances": int(len(counts)), "histories_per_step": total,
            "launch": launch,
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "lane-ops/s",
                         "frac": achieved / peak, "traffic": TRAFFIC_PER_LAUNCH.get(("batched", launch["kernel"])),
                         "per_unit": alg_ph, "per_unit_basis": "algorithmic lane operations per history "
                         "(secondaries included), weighted by the run's counters",
                         "kernel": "transport forward with score-function accumulators"},
            "forward_ms": fw_ms, "backward_ms": bw_ms, "gradients": "d tallies / d (radius, scale, density)",
            "gpu_launches_per_step": launches_per_step,
            "rel_stderr_total_median_instance": rel,
            "s_to_eps_per_instance": (rel / 1e-3) ** 2 * N / (hist_s / len(counts)),
            **({"cpu_baseline": cpu_baseline(args, desc, total, grad=True)} if args.cpu_baseline else {})}


def cpu_baseline(args, desc, n_full, grad: bool = False) -> dict:
    """The CPU oracle on the host cores, on a bounded sample of the workload:
    a pilot run sets the sample to about args.cpu_seconds of CPU work.  With
    grad, every instance runs a share of the sample in proportion to its
    history count, with the score-function accumulators."""
    import numpy as np
    from oracle.oracle import OracleScene
    cores = os.cpu_count() or 1
    sc = OracleScene(desc)
    counts = np.asarray(desc["instances"]["counts"], dtype=np.float64)

    def run(total, threads=cores):
        if not grad:
            sc.run(total, threads=threads)
            return total
        share = np.maximum(1, np.rint(total * counts / counts.sum())).astype(np.int64)
        for q, m in enumerate(share):
            sc.run(int(m), inst=q, threads=threads, want_grad=True)
        return int(share.sum())

    pilot = max(10_000, min(args.cpu_sample // 40, 1_000_000))
    run(min(100_000, pilot))                 # warm the library
    t0 = time.perf_counter()
    done = run(pilot)
    rate = done / (time.perf_counter() - t0)
    limit = min(args.cpu_sample, n_full)
    sample = int(min(max(rate * args.cpu_seconds, pilot), limit))
    for _ in range(3):   # the pilot's rate is rough: grow the sample until it takes about the target time
        t0 = time.perf_counter()
        sample = run(sample)
        dt = time.perf_counter() - t0
        if dt >= 0.5 * args.cpu_seconds or sample >= limit:
            break
        sample = int(min(sample * args.cpu_seconds / max(dt, 1e-3), limit))
    what = (f"{sample} histories of the {n_full}-history workload, a share of every instance in proportion "
            f"to its count, with gradients" if grad else f"the first {sample} histories of the {n_full}-history workload")
    # and on one thread, about a quarter of the target time
    one = max(1000, int(sample / dt / cores * args.cpu_seconds / 4))
    t0 = time.perf_counter()
    one = run(one, threads=1)
    dt1 = time.perf_counter() - t0
    return {"value": sample / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{what}; FP64, {cores} threads", "seconds": dt,
            "single_thread": {"value": one / dt1, "unit": UNIT, "histories": one, "seconds": dt1}}


def run_reference(args, rank: int) -> dict | None:
    if rank != 0:
        return None
    import numpy as np
    from oracle.oracle import OracleScene
    desc, label = workload_desc(args.workload)
    n = int(desc["instances"]["counts"][0])
    cores = os.cpu_count() or 1
    sc = OracleScene(desc)
    per_step = args.ref_sample
    counts = desc["instances"]["counts"]
    if args.workload == "batched":
        # a bounded sample of every instance, in proportion to its count, with gradients
        share = np.maximum(1, np.rint(per_step * counts / counts.sum())).astype(np.int64)
        per_step = int(share.sum())

        def one(k, scale=1.0):
            for q, m in enumerate(share):
                m = max(1, int(m * scale))
                sc.run(m, inst=q, first=k * m, threads=cores, want_grad=True)
    else:
        def one(k, scale=1.0):
            m = max(1, int(per_step * scale))
            sc.run(m, first=k * per_step, threads=cores)
    for k in range(args.warmup):
        one(k, 0.1)
    t0 = time.perf_counter()
    for k in range(args.steps):
        one(k)
    dt = time.perf_counter() - t0
    value = per_step * args.steps / dt
    return {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": int(os.environ.get("WORLD_SIZE", "1")),
            "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": workload_config(args.workload, label, {"histories_per_step": per_step}),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{per_step} histories per step of the {int(counts.sum())}-history workload"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main() -> None:
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="powder")
    ap.add_argument("--histories", type=int, default=0, help="override the histories per step")
    ap.add_argument("--kernel", type=int, default=0, help="0 autotuned, 1 history-based, 2 event-based, 3 warp pools")
    ap.add_argument("--secondaries", type=int, default=0,
                    help="gradient runs: 0 autotuned, 1 in place, 2 queued for a second pass")
    ap.add_argument("--block-size", type=int, default=0, help="threads per block with --kernel (0: 256)")
    ap.add_argument("--stage", type=int, default=0,
                    help="with --kernel: scene tables 0 staged when they fit, 1 staged, 2 read from device memory")
    ap.add_argument("--ctas-per-sm", type=int, default=0,
                    help="CTAs per SM with --kernel (4 x 256 threads selects the 64-register build)")
    ap.add_argument("--no-batched", dest="batched", action="store_false")
    ap.add_argument("--batched-steps", type=int, default=2)
    ap.add_argument("--no-cpu-baseline", dest="cpu_baseline", action="store_false")
    ap.add_argument("--cpu-sample", type=int, default=1_000_000_000, help="most histories of the CPU baseline")
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="CPU work the baseline sample is sized to")
    ap.add_argument("--ref-sample", type=int, default=10_000_000)
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.gpus != world:
        raise SystemExit(f"--gpus {args.gpus} but WORLD_SIZE={world}: launch N ranks with "
                         f"python -m torch.distributed.run --nproc-per-node N bench.py --gpus N")
    if args.impl == "reference":
        line = run_reference(args, rank)
    else:
        line = run_ours(args, rank, world)
    if line is not None:
        print(json.dumps(line))


if __name__ == "__main__":
    main()
