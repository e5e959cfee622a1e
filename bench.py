#!/usr/bin/env python
"""Throughput of one mODIL optimiser step on the GPU (and of the CPU oracle).

Default workload (the largest configuration on one GPU): 512 viscous Burgers
instances of uneven size (paper Section 3.2 discretisation; N_x, N_t drawn
from {64, 128, 256, 512}, nu log-uniform in [1e-3, 1e-1], 0.5 % of the cells
measured), all stepped together: one launch per phase of the step for all
instances (composition of the coarse levels, the warp-streaming fine kernel,
restriction + Adam of the coarse levels, per-instance tail), replayed as one
CUDA graph.  A step is one loss+gradient evaluation of
every instance followed by the Adam update of every level of every instance;
the metric is instance evaluations per second.  The ~1.3 GB working set is
larger than L2, so no flush is needed.

Timing: W untimed warm-up steps, then K steps between two CUDA events on the
problem's stream, bracketed by a barrier and a device synchronisation, the
maximum over ranks (replicas under torchrun); SM clocks sampled meanwhile.
One JSON line is printed by rank 0.  Other workloads: --workload heat | body |
cavity | burgers | poisson | unet | warmstart.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl modil|reference]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "mODIL loss+grad evals/s"
UNIT = "evals/s"
WORKLOAD = "heat conductivity inference, 512x512 space-time, 7 levels, FP32, Adam"
ALG_BYTES_PER_PARAM = 32     # p, m (FP32) and v (FP64), read and written
ALG_BYTES_PER_MEAS = 8       # cell index + value


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="modil", choices=["modil", "reference"])
    ap.add_argument("--tile", default=None,
                    help="fine tile 'ROWSxCOLS' (heat default 32x32; batched default 32x60, the "
                         "warp-streaming strip) or 'auto' (autotuner)")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--profile-steps", type=int, default=50)
    ap.add_argument("--workload", default="batched-burgers",
                    choices=["heat", "batched-burgers", "body", "warmstart", "unet", "burgers", "cavity",
                             "poisson", "burgers-paper"],
                    help="batched-burgers (default): 512 uneven Burgers instances in one "
                         "persistent graph-captured launch per phase, against sequential single "
                         "runs; heat: conductivity inference on 512x512; "
                         "body: 3-D body-shape inference, 128^3 cells, 8 levels, five fields; "
                         "warmstart: U-Net warm start of the body problem against zero init")
    ap.add_argument("--train", type=int, default=2048, help="warmstart: training ellipsoids")
    ap.add_argument("--epochs", type=int, default=10, help="warmstart: U-Net training epochs")
    ap.add_argument("--held-out", type=int, default=8, help="warmstart: held-out ellipsoids")
    ap.add_argument("--infer-steps", type=int, default=10000, help="heat: Adam steps of the inference run")
    ap.add_argument("--optimizer", choices=("lbfgs", "adam"), default="adam",
                    help="warmstart: optimiser of the 128^3 forward and inverse problems (Adam with a "
                         "decaying learning rate; L-BFGS stalls near 9e-3 on the 128^3 body problem)")
    ap.add_argument("--fwd-iters", type=int, default=5000,
                    help="warmstart, L-BFGS only: iterations of each 128^3 reference forward solve")
    ap.add_argument("--side", type=int, default=64, help="unet: grid side of the training step")
    ap.add_argument("--instances", type=int, default=512)
    return ap.parse_args()


def max_over_ranks(ms, world, device="cuda"):
    """Largest per-rank time (the job's time) of a replicated run; `ms` is this
    rank's value.  world == 1 returns it unchanged."""
    if world <= 1:
        return float(ms)
    import torch
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def job_throughput(steps_per_rank, world, job_ms):
    """Whole-job evaluations per second: every rank runs `steps_per_rank`
    steps of its own replica; the job takes the slowest rank's time."""
    return world * steps_per_rank / (job_ms * 1e-3)


def dist_env():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


def heat_config(args, w):
    """The `config` of the heat line, identical in both arms."""
    params, _ = workload_sizes(w)
    return {"workload": WORKLOAD, "grid": list(w["shape"]), "levels": w["n_levels"],
            "params": params, "measurements": len(w["meas_cell"]), "tile": args.tile,
            "data": "5 % of cells of the forward solution with k(u) = 0.02 exp(-20 (u - 1/2)^2) on 32 "
                    "nodes, N(0, 1e-3^2) noise",
            "adam_lr": w["lr"], "k_scale": w["k_scale"],
            "l2": "flushed before every timed step (256 MiB write)", "parallelism": "replicas"}


def workload_sizes(w):
    nt, nx = w["shape"]
    params = sum((nt >> l) * (nx >> l) for l in range(w["n_levels"])) + len(w["knodes"])
    fine = nt * nx
    return params, fine


# ---------------------------------------------------------------------------
# CPU oracle timing (baseline and the reference arm)
# ---------------------------------------------------------------------------
def blas_threads():
    try:
        from threadpoolctl import threadpool_info
        n = [i.get("num_threads", 1) for i in threadpool_info() if i.get("user_api") == "blas"]
        return max(n) if n else 1
    except Exception:
        return os.cpu_count() or 1


def oracle_setup(w):
    import oracle as o
    from paper_2303_04679_gb300 import inputs
    f32 = lambda a: np.asarray(a, np.float64).astype(np.float32).astype(np.float64)  # noqa: E731
    prob = o.Problem("heat", w["shape"], w["n_levels"], w_res=w["w_res"], w_data=w["w_data"],
                     w_reg=w["w_reg"], meas_cell=w["meas_cell"], meas_value=f32(w["meas_value"]),
                     aux=f32(w["aux"]), k_scale=w["k_scale"])
    levels = [np.zeros(s) for s in inputs.level_shapes(w["shape"], w["n_levels"])]
    st = o.OracleState.zeros_like_levels(levels, f32(w["knodes"]))
    return o, prob, st


def time_oracle(w, seconds, max_steps=None):
    o, prob, st = oracle_setup(w)
    o.oracle_step(prob, st, w["lr"])  # warm-up (imports, BLAS pools)
    n = 0
    t0 = time.perf_counter()
    while True:
        o.oracle_step(prob, st, w["lr"])
        n += 1
        el = time.perf_counter() - t0
        if el >= seconds or (max_steps and n >= max_steps):
            break
    return n, el


def cpu_model():
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu model")):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.machine()


def run_reference(args, w):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    # each timed step is one full oracle step on the whole workload; the run
    # stops early after ~150 s and reports the steps it timed
    _, _, _ = oracle_setup(w)
    o, prob, st = oracle_setup(w)
    for _ in range(max(args.warmup, 1) if args.warmup < 3 else 3):
        o.oracle_step(prob, st, w["lr"])
    t0 = time.perf_counter()
    n = 0
    for _ in range(args.steps):
        o.oracle_step(prob, st, w["lr"])
        n += 1
        if time.perf_counter() - t0 > 150.0:
            break
    el = time.perf_counter() - t0
    value = n / el
    cores = blas_threads()
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": n, "warmup": args.warmup, "ms_per_step": 1e3 * el / n, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": heat_config(args, w),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{n} full oracle Adam steps of the workload ({cpu_model()})"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# GPU clocks sampled during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx = float(parts[1])
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def make_desc(modil, w, tile):
    ty, tx = (int(v) for v in tile.split("x"))
    return modil.Desc("heat", w["shape"], w["n_levels"], "f32", w_res=w["w_res"],
                      w_data=w["w_data"], w_reg=w["w_reg"], meas_cell=w["meas_cell"],
                      meas_value=w["meas_value"], aux=w["aux"], knodes=w["knodes"], lr=w["lr"],
                      tile=(ty, tx), k_scale=w["k_scale"])


def heat_reference_workload():
    """The heat workload of the reference arm: the same record (the forward
    problem with the nodes of the reference conductivity) from the oracle's
    row-by-row implicit solve."""
    import oracle as o
    from paper_2303_04679_gb300 import inputs
    n = 512
    q = inputs.heat_k_true(np.arange(inputs.HEAT_KNODES) / (inputs.HEAT_KNODES - 1))
    rec = o.heat_implicit_solve(inputs.heat_ic(n), n, 1.0 / n, 1.0 / n, lambda uf: o.heat_conductivity(uf, q)[0])
    return inputs.heat_workload(field=rec)


def k_error(q):
    """RMS error of the nodes' piecewise-linear conductivity against the
    reference k over u in (0, 1), normalised by the reference's maximum 0.02
    (the measure of Section 3.4)."""
    from paper_2303_04679_gb300 import inputs
    uu = (np.arange(1000) + 0.5) / 1000
    uj = np.arange(len(q)) / (len(q) - 1)
    return float(np.sqrt(np.mean((np.interp(uu, uj, q) - inputs.heat_k_true(uu)) ** 2)) / 0.02)


def heat_inference(modil, w, args, chunk=250):
    """Conductivity inference to a tolerance: Adam from zero levels and
    constant nodes on the workload w, the conductivity error read every chunk
    of steps (wall time includes the reads)."""
    import torch
    tols = (0.5, 0.3, 0.2, 0.1, 0.06)
    hits = {t: None for t in tols}
    hist = []
    with modil.Problem(make_desc(modil, w, "0x0")) as p:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        done = 0
        while done < args.infer_steps:
            p.step(chunk, read_loss=False)
            done += chunk
            e = k_error(p.read_knodes())
            el = time.perf_counter() - t0
            hist.append((done, e))
            for t in tols:
                if hits[t] is None and e <= t:
                    hits[t] = {"steps": done, "seconds": el}
        q = p.read_knodes()
        loss = float(p.eval_loss()[0, 0])
    return {"metric": "conductivity error (RMS over u in (0,1) / max k, Section 3.4)",
            "grid": list(w["shape"]), "levels": w["n_levels"], "measurements": len(w["meas_cell"]),
            "adam_lr": w["lr"], "k_scale": w["k_scale"],
            "k_error_initial": k_error(w["knodes"]), "k_error_final": hist[-1][1], "steps": done,
            "to_tolerance": {str(t): hits[t] for t in tols}, "loss_final": loss,
            "k_error_every_1000": [round(e, 4) for s, e in hist if s % 1000 == 0],
            "k_over_0.02_every_3rd_node": [round(float(v) / 0.02, 3) for v in q[::3]],
            "k_max_over_min": float(np.max(q) / max(np.min(np.abs(q)), 1e-30))}


# Config 2's inference with the paper's optimiser (Section 3.4 runs mODIL with
# L-BFGS-B): the data weight and the node unit are readings (the paper states
# neither): the data term weighted 1e4 against the residual integral, the
# nodes in their own units (k_scale = 1).  With the data weight 1 the joint
# optimum at 512 x 512 lies far from the reference conductivity.
HEAT_LBFGS = dict(w_data=1e4, k_scale=1.0, history=50, chunk=100, iterations=2000)


def heat_inference_lbfgs(modil, w, args):
    """Conductivity inference to a tolerance by the device L-BFGS on the
    workload w (zero levels, constant nodes), the conductivity error read
    every chunk of iterations (wall time includes the reads)."""
    import torch
    c = HEAT_LBFGS
    tols = (0.5, 0.3, 0.2, 0.1, 0.05, 0.02, 0.01)
    hits = {t: None for t in tols}
    hist = []
    w2 = dict(w, w_data=c["w_data"], k_scale=c["k_scale"])
    with modil.Problem(make_desc(modil, w2, "0x0")) as p, modil.LBFGS(p, history=c["history"]) as opt:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        done = 0
        loss = None
        while done < c["iterations"]:
            h = opt.run(c["chunk"])
            done += len(h) - 1
            loss = float(h[-1])
            e = k_error(p.read_knodes())
            el = time.perf_counter() - t0
            hist.append((done, e))
            for t in tols:
                if hits[t] is None and e <= t:
                    hits[t] = {"iterations": done, "seconds": el}
            if len(h) - 1 < c["chunk"]:
                break
        q = p.read_knodes()
    return {"metric": "conductivity error (RMS over u in (0,1) / max k, Section 3.4)",
            "optimizer": f"device L-BFGS (history {c['history']}, Armijo backtracking)",
            "grid": list(w["shape"]), "levels": w["n_levels"], "measurements": len(w["meas_cell"]),
            "w_data": c["w_data"], "k_scale": c["k_scale"], "dtype": "f32",
            "k_error_initial": k_error(w["knodes"]), "k_error_final": hist[-1][1], "iterations": done,
            "to_tolerance": {str(t): hits[t] for t in tols}, "loss_final": loss,
            "k_error_every_500": [round(e, 4) for s, e in hist if s % 500 == 0],
            "k_over_0.02_every_3rd_node": [round(float(v) / 0.02, 3) for v in q[::3]]}


def measured_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


BATCH_METRIC_UNIT = "instance " + UNIT


def batched_config(args, tile, pers, fine, params, nmeas):
    """The `config` of the batched line, identical in both arms."""
    return {"workload": f"batched Burgers x{args.instances}: N_x, N_t uniform in {{64,128,256,512}}, "
                        "nu log-uniform in [1e-3, 1e-1], 0.5 % measured cells, "
                        "L = log2(min(N_x, N_t)/8) + 1, FP32, Adam, one launch per phase of the step "
                        "for all instances, the step captured in one CUDA graph",
            "instances": args.instances, "tile": list(tile), "persistent": pers,
            "fine_cells": fine, "params": params, "measurements": nmeas,
            "l2": "working set (about 1.3 GB) larger than L2 (no flush)",
            "parallelism": "replicas"}


def batch_sizes(batch):
    fine = sum(d["shape"][0] * d["shape"][1] for d in batch)
    params = sum(sum((d["shape"][0] >> l) * (d["shape"][1] >> l) for l in range(d["n_levels"]))
                 for d in batch)
    nmeas = sum(len(d["meas_cell"]) for d in batch)
    return fine, params, nmeas


def oracle_burgers(d):
    import oracle as o
    from paper_2303_04679_gb300 import inputs
    f32 = lambda a: np.asarray(a, np.float64).astype(np.float32).astype(np.float64)  # noqa: E731
    prob = o.Problem("burgers", d["shape"], d["n_levels"], coef={"nu": d["nu"]},
                     meas_cell=d["meas_cell"], meas_value=f32(d["meas_value"]))
    st = o.OracleState.zeros_like_levels([np.zeros(s) for s in inputs.level_shapes(d["shape"], d["n_levels"])])
    return o, prob, st


def time_batch_oracle(batch, seconds, per_step=None):
    """Oracle Adam steps on the batch's instances in order (cycling), each
    instance set up outside the clock; returns (instance steps, seconds)."""
    n, el, i = 0, 0.0, 0
    while el < seconds and (per_step is None or n < per_step):
        o, prob, st = oracle_burgers(batch[i % len(batch)])
        t0 = time.perf_counter()
        o.oracle_step(prob, st, 5e-3)
        el += time.perf_counter() - t0
        n += 1
        i += 1
    return n, el


def traffic_record(name, sources_ok=True):
    """A kernel's DRAM bytes from profiles/traffic.json, if its sources still
    hash to the recorded value (otherwise the counters are stale: None)."""
    tfile = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        from paper_2303_04679_gb300 import build as bld
        tj = json.load(open(tfile))[name]
        if tj.get("source_hash") == bld.source_hash(tj["sources"]):
            return tj
    except Exception:
        pass
    return None


def run_reference_batched(args):
    """The reference arm of the batched line: the FP64 CPU oracle as it
    stands, on the host cores; each step is a bounded sample of the same
    batch (16 consecutive instances, cycling through the 512), one oracle Adam
    step each; rank 0 only."""
    from paper_2303_04679_gb300 import inputs
    rank, world, _ = dist_env()
    if rank != 0:
        return
    batch = inputs.burgers_batch(args.instances)
    fine, params, nmeas = batch_sizes(batch)
    tile = tuple(int(v) for v in (args.tile or "32x60").split("x")) if args.tile != "auto" else (32, 60)
    per = 16
    for w in range(max(args.warmup, 0)):
        o, prob, st = oracle_burgers(batch[w % len(batch)])
        o.oracle_step(prob, st, 5e-3)
    n, el, i = 0, 0.0, 0
    for _ in range(args.steps):
        for _ in range(per):
            o, prob, st = oracle_burgers(batch[i % len(batch)])
            t0 = time.perf_counter()
            o.oracle_step(prob, st, 5e-3)
            el += time.perf_counter() - t0
            n += 1
            i += 1
    value = n / el
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": BATCH_METRIC_UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * el / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": batched_config(args, tile, tile != (32, 60), fine, params, nmeas),
        "cpu_baseline": {"value": value, "unit": BATCH_METRIC_UNIT, "cores": blas_threads(),
                         "kind": "oracle",
                         "sample": f"{per} instances of the batch per step (cycling, {n} in all), one "
                                   f"oracle Adam step each ({cpu_model()}, {os.cpu_count()} host cores)"},
        "e2e": {"value": value, "unit": BATCH_METRIC_UNIT, "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_batched(args):
    """512 uneven Burgers instances (the largest configuration): one batched,
    persistent, graph-captured launch per phase.  Device time of K steps with
    CUDA events; the same instances stepped one problem after another with
    the same kernels as the comparison; the fine kernel's roofline; the
    public-API end-to-end rate from pinned host buffers; the CPU oracle on a
    bounded sample."""
    import torch

    from paper_2303_04679_gb300 import autotune, inputs, modil
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    batch = inputs.burgers_batch(args.instances)

    def descs(tile):
        return [modil.Desc("burgers", d["shape"], d["n_levels"], "f32", coef=(d["nu"],),
                           meas_cell=d["meas_cell"], meas_value=d["meas_value"], lr=5e-3,
                           tile=tile) for d in batch]

    if args.tile == "auto":
        tile, pers, _ = autotune.autotune(
            descs((16, 32)), measure=lambda d, t, q: autotune.time_steps(d, t, q, steps=10, warmup=3))
    else:
        tile = tuple(int(v) for v in (args.tile or "32x60").split("x"))
        pers = tile != autotune.STREAM_TILE
    ds = descs(tile)
    fine, params, nmeas = batch_sizes(batch)
    K = args.steps
    with modil.Problem(ds) as p:
        if pers:
            p.set_persistent(True)
        p.step(max(3, args.warmup), read_loss=False)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        sampler = ClockSampler(local)
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        sampler.start()
        time.sleep(0.25)
        a.record(p.stream)
        p.step(K, read_loss=False)
        b.record(p.stream)
        b.synchronize()
        clocks = sampler.stop()
        if world > 1:
            torch.distributed.barrier()
        job_ms = max_over_ranks(a.elapsed_time(b), world)
        t_batch = job_ms / K
        final_batch = p.eval_loss()[:, 0].copy()
        prof = np.array([p.profile_step() for _ in range(5)]).mean(axis=0)
        labels = p.profile_labels()
        launches = p.launches_per_step()
    # the same instances as separate problems, stepped one after another
    t_seq, same, maxrel = None, None, None
    if rank == 0 and world == 1:
        probs = [modil.Problem(d, stream=torch.cuda.Stream()) for d in ds]
        s0 = torch.cuda.current_stream()
        for q in probs:
            q.step(max(3, args.warmup), read_loss=False)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(s0)
        prev = a
        for q in probs:  # each problem starts when the previous one has finished
            q.stream.wait_event(prev)
            q.step(K, read_loss=False)
            prev = torch.cuda.Event()
            prev.record(q.stream)
        s0.wait_event(prev)
        b.record(s0)
        b.synchronize()
        t_seq = a.elapsed_time(b) / K
        final_seq = np.array([q.eval_loss()[0, 0] for q in probs])
        for q in probs:
            q.close()
        same = bool(np.array_equal(final_batch, final_seq))
        maxrel = float(np.max(np.abs(final_batch - final_seq) / np.abs(final_seq)))

    # end to end through the public C ABI: create from host descriptors, write
    # every level from pinned host memory, K steps each reading the loss terms
    # back, read the composed fields; copies inside the timed region
    lv_host = [[torch.zeros(s, dtype=torch.float32).pin_memory()
                for s in inputs.level_shapes(d["shape"], d["n_levels"])] for d in batch]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    with modil.Problem(ds) as pe:
        if pers:
            pe.set_persistent(True)
        for i, lv in enumerate(lv_host):
            for lvl, t in enumerate(lv):
                modil._check(modil.LIB.modil_write_level(pe._h, i, 0, lvl, t.data_ptr(), t.numel() * 4, 0))
        for _ in range(K):
            pe.step(1, read_loss=True)
        fields = [pe.read_field(instance=i) for i in range(len(batch))]
    e2e_s = time.perf_counter() - t0
    h2d = (sum(t.numel() * 4 for lv in lv_host for t in lv) + nmeas * 8)
    d2h = K * len(batch) * 4 * 8 + sum(f.nbytes for f in fields)
    e2e_ms = max_over_ranks(1e3 * e2e_s, world)

    peak, peak_kind = measured_peak()
    fine_bytes = fine * ALG_BYTES_PER_PARAM + nmeas * ALG_BYTES_PER_MEAS
    kms = {lab: float(v) for lab, v in zip(labels, prof)}
    ach = fine_bytes / (kms["fine"] * 1e-3) / 1e9
    tr = traffic_record("batched_fine")
    traffic = None
    if tr is not None and tr.get("tile") == list(tile):
        traffic = tr["bytes_per_fine_cell"] * fine
    out = {
        "metric": METRIC, "value": job_throughput(args.instances * K, world, job_ms),
        "unit": BATCH_METRIC_UNIT, "n_gpus": world, "steps": K, "warmup": args.warmup,
        "ms_per_step": t_batch, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": batched_config(args, tile, pers, fine, params, nmeas),
        "fine_cells_per_s": world * fine / (t_batch * 1e-3),
        "effective_step_GBps": (params * ALG_BYTES_PER_PARAM + nmeas * 8) / (t_batch * 1e-3) / 1e9,
        "hbm_frac_step": (params * ALG_BYTES_PER_PARAM + nmeas * 8) / (t_batch * 1e-3) / 1e9 / peak,
        "sequential_ms_per_step": t_seq, "batched_speedup": (t_seq / t_batch) if t_seq else None,
        "same_final_loss": same, "final_loss_max_rel_diff": maxrel,
        "kernel_ms": kms,
        "roofline": {"kernel": "fine" + (" (warp-streaming)" if tile == autotune.STREAM_TILE else " (tile)"),
                     "bound": "hbm", "achieved": ach, "peak": peak,
                     "peak_kind": peak_kind, "unit": "GB/s", "frac": ach / peak, "traffic": traffic,
                     "alg_bytes_per_launch": fine_bytes,
                     "note": "algorithmic bytes: 32 B per fine cell (p, m FP32 and v FP64 read and "
                             "written) + 8 B per measurement; fine kernel's CUDA-event time on the "
                             "problem's stream; peak = measured burst copy"},
        "clocks": clocks,
        "gpu_launches": launches * K,
        "e2e": {"value": world * args.instances * K / (e2e_ms * 1e-3), "unit": BATCH_METRIC_UNIT,
                "h2d_bytes_per_step": h2d / K, "d2h_bytes_per_step": d2h / K, "steps": K,
                "note": "create + level upload from pinned host memory + K steps with the loss "
                        "terms read back every step + composed fields read"},
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        n, el = time_batch_oracle(batch, args.cpu_seconds)
        out["cpu_baseline"] = {"value": n / el, "unit": BATCH_METRIC_UNIT, "cores": blas_threads(),
                               "kind": "oracle",
                               "sample": f"{n} oracle Adam steps of single instances, cycling through the "
                                         f"batch in order, {el:.1f} s ({cpu_model()}, {os.cpu_count()} host cores)"}
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def body_levels(w):
    """Initial guess of the body problem: uniform inflow u = 1 on the fine
    level, every other level and field zero (chihat = 0)."""
    from paper_2303_04679_gb300 import inputs
    shapes = inputs.level_shapes(w["shape"], w["n_levels"])
    lv = [[np.zeros(s, np.float32) for s in shapes] for _ in range(5)]
    lv[0][0][:] = 1.0
    return lv


def time_body_oracle(w, seconds):
    """Oracle loss+gradient evaluations of the body problem on a 16 x 16 x 32
    sample grid (the full 128^3 gradient takes the oracle tens of minutes);
    returns (evaluations, seconds, sample cells)."""
    import oracle as o
    from paper_2303_04679_gb300 import inputs
    sh, L = (16, 16, 32), 5
    centre, axes = w["centre"], w["axes"]
    cells, fields, vals = inputs.ns3d_slab(sh, 5, centre, axes)
    prob = o.Problem("ns3d", sh, L, coef=dict(w["coef"]), meas_cell=cells, meas_field=fields,
                     meas_value=vals)
    lv = inputs.random_levels(sh, L, 5, 1, -0.5, 0.5, 0.2)
    o.loss_grad_levels(prob, lv)
    n, t0 = 0, time.perf_counter()
    while True:
        o.loss_grad_levels(prob, lv)
        n += 1
        el = time.perf_counter() - t0
        if el >= seconds:
            return n, el, int(np.prod(sh))


def run_body(args):
    """3-D body-shape inference (penalised steady Navier-Stokes, five fields)
    on 128^3 cells with 8 levels, FP32; the 384 MB working set is larger than
    L2, so the steps run back to back without a flush."""
    import torch

    from paper_2303_04679_gb300 import inputs, modil
    torch.cuda.set_device(0)
    w = inputs.ns3d_workload()
    cf = w["coef"]
    shape, L = w["shape"], w["n_levels"]
    desc = modil.Desc("ns3d", shape, L, "f32", coef=(cf["Re"], cf["D"], cf["lam"], cf["tau"]),
                      w_res=w["w_res"], w_data=w["w_data"], meas_cell=w["meas_cell"],
                      meas_field=w["meas_field"], meas_value=w["meas_value"], lr=w["lr"])
    fine = int(np.prod(shape))
    params = 5 * sum(int(np.prod(s)) for s in inputs.level_shapes(shape, L))
    n_meas = len(w["meas_cell"])
    step_bytes = params * ALG_BYTES_PER_PARAM + n_meas * ALG_BYTES_PER_MEAS
    lev0_bytes = 5 * fine * ALG_BYTES_PER_PARAM + n_meas * ALG_BYTES_PER_MEAS
    K = args.steps
    with modil.Problem(desc) as p:
        p.write_fields(body_levels(w))
        launches = p.launches_per_step()
        p.step(max(3, args.warmup), read_loss=False)
        torch.cuda.synchronize()
        sampler = ClockSampler(0)
        sampler.start()
        time.sleep(0.25)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(p.stream)
        p.step(K, read_loss=False)
        b.record(p.stream)
        b.synchronize()
        clocks = sampler.stop()
        ms = a.elapsed_time(b) / K
        loss = float(p.eval_loss()[0, 0])
        prof = np.array([p.profile_step() for _ in range(max(1, min(args.profile_steps, 20)))])
    kern_ms = prof.mean(axis=0)
    names = ([f"prolong3_L{l + 1}" for l in range(L - 2, -1, -1)] + ["residual_adjoint_adam3"] +
             [f"restrict_adam3_L{l + 1}" for l in range(1, L)] + ["finalize"])
    dom = int(np.argmax(kern_ms))
    peak, peak_kind = measured_peak()
    dom_bytes = lev0_bytes if names[dom] == "residual_adjoint_adam3" else None
    achieved = dom_bytes / (kern_ms[dom] * 1e-3) / 1e9 if dom_bytes else None
    # end to end: create, upload the initial guess from pinned host memory,
    # steps with the loss read back, read the composed fields
    e2e_steps = min(K, 200)
    host = [[torch.from_numpy(a).pin_memory() for a in lv] for lv in body_levels(w)]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    with modil.Problem(desc) as p2:
        for f, lv in enumerate(host):
            for lvl, a in enumerate(lv):
                modil._check(modil.LIB.modil_write_level(p2._h, 0, f, lvl, a.data_ptr(),
                                                         a.numel() * 4, 0))
        for _ in range(e2e_steps):
            p2.step(1, read_loss=True)
        fields = [p2.read_field(f) for f in range(5)]
    e2e_s = time.perf_counter() - t0
    h2d = sum(a.numel() * 4 for lv in host for a in lv) + n_meas * 12
    d2h = 32 * e2e_steps + sum(x.nbytes for x in fields)
    value = 1.0 / (ms * 1e-3)
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": K,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "3-D body-shape inference, 128^3 cells, 8 levels, u,v,w,p,chihat, "
                               "FP32, Adam", "params": params, "measurements": n_meas,
                   "l2": "working set (384 MB) larger than L2 (no flush)"},
        "fine_cells_per_s": value * fine,
        "effective_step_GBps": step_bytes * value / 1e9,
        "hbm_frac_step": step_bytes * value / 1e9 / peak,
        "loss_final": loss,
        "kernel_ms": {n: float(v) for n, v in zip(names, kern_ms)},
        "roofline": {"kernel": names[dom], "bound": "hbm", "achieved": achieved, "peak": peak,
                     "peak_kind": peak_kind, "unit": "GB/s",
                     "frac": (achieved / peak) if achieved else None, "traffic": None,
                     "alg_bytes_per_launch": dom_bytes},
        "clocks": clocks,
        "gpu_launches": launches * K,
        "e2e": {"value": e2e_steps / e2e_s, "unit": UNIT, "h2d_bytes_per_step": h2d / e2e_steps,
                "d2h_bytes_per_step": d2h / e2e_steps, "steps": e2e_steps,
                "note": "create + upload + steps with loss read back + field read"},
    }
    if not args.no_cpu_baseline:
        n, el, cells = time_body_oracle(w, args.cpu_seconds)
        out["cpu_baseline"] = {
            "value": n * cells / el / fine, "unit": UNIT, "cores": blas_threads(), "kind": "oracle",
            "sample": f"{n} oracle loss+gradient evaluations of a 16x16x32, 5-level body problem "
                      f"in {el:.1f} s, scaled by cells to the 128^3 grid ({cpu_model()})"}
    print(json.dumps(out), flush=True)


def flushed_steps(step, stream, flush, K, W):
    """Per-step CUDA-event times (ms) of K calls of step(), each after an L2
    flush (a write of a buffer larger than L2) on the same stream."""
    import torch
    for _ in range(max(3, W)):
        with torch.cuda.stream(stream):
            flush.zero_()
        step()
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    for a, b in evs:
        with torch.cuda.stream(stream):
            flush.zero_()
        a.record(stream)
        step()
        b.record(stream)
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in evs]


def run_poisson(args):
    """The paper's Poisson level sweep (Section 3.1): d = 1, 2, 3, node and cell
    layouts, N = 32 cells per axis, zero initial guess, L = 1..5 levels; 400
    Adam iterations (lr 0.005) and 400 L-BFGS iterations (history 50); the
    RMS error relative to the exact solution of the discrete problem, which
    the library itself computes first (L-BFGS with five levels until the loss
    stops falling).  The right-hand side is the closed-form Laplacian of the
    reference u_ref of the recipe."""
    import torch

    from paper_2303_04679_gb300 import inputs, modil
    torch.cuda.set_device(0)
    n = 32
    sweeps = []
    for d in (1, 2, 3):
        for layout in ("node", "cell"):
            w = inputs.poisson_workload(n, d, layout)

            def desc(L):
                return modil.Desc("poisson", w["shape"], L, "f64", aux=w["f"].ravel(), layout=layout, lr=5e-3)

            def solution(u):
                # node layout: the boundary nodes hold the imposed Dirichlet value
                if layout == "node":
                    u = u.copy()
                    for ax in range(d):
                        idx = [slice(None)] * d
                        idx[ax] = 0
                        u[tuple(idx)] = 0.0
                        idx[ax] = -1
                        u[tuple(idx)] = 0.0
                return u
            with modil.Problem(desc(5)) as p, modil.LBFGS(p, history=50) as opt:
                hist = opt.run(3000)
                exact = solution(p.read_field())
            scale = float(np.sqrt(np.mean(exact ** 2)))
            err = lambda u: float(np.sqrt(np.mean((solution(u) - exact) ** 2)) / scale)  # noqa: E731
            rows = []
            for L in range(1, 6):
                with modil.Problem(desc(L)) as p:
                    torch.cuda.synchronize()
                    t0 = time.perf_counter()
                    p.step(400, read_loss=False)
                    torch.cuda.synchronize()
                    t_adam = time.perf_counter() - t0
                    e_adam = err(p.read_field())
                errs = []
                t_lb = 0.0
                with modil.Problem(desc(L)) as p, modil.LBFGS(p, history=50) as opt:
                    for _ in range(20):  # 20 x 20 iterations; the pair history carries over
                        torch.cuda.synchronize()
                        t0 = time.perf_counter()
                        h = opt.run(20)
                        t_lb += time.perf_counter() - t0
                        errs.append(err(p.read_field()))
                        if len(h) < 21:
                            break
                reach = next((20 * (k + 1) for k, e in enumerate(errs) if e < 1e-10), None)
                rows.append({"levels": L, "adam_error": e_adam, "adam_seconds": t_adam,
                             "lbfgs_error": errs[-1], "lbfgs_seconds": t_lb,
                             "lbfgs_iterations_to_1e-10": reach})
            sweeps.append({"d": d, "layout": layout, "exact_solve_loss": float(hist[-1]),
                           "exact_vs_u_ref": float(np.sqrt(np.mean((exact - w["u_ref"]) ** 2)) / scale),
                           "levels": rows})
    out = {
        "metric": "relative RMS error after 400 iterations (Adam, L-BFGS) against the discrete solution",
        "unit": "relative RMS error", "n_gpus": 1, "steps": 400, "warmup": 0, "higher_is_better": False,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": "Poisson, d = 1, 2, 3, node and cell layouts, 32 cells per axis, "
                               "levels 1..5, zero initial guess"},
        "sweep": sweeps,
    }
    print(json.dumps(out), flush=True)


def bilinear_at(u, pts, lengths=(1.0, 1.0), origin=(0.0, 0.0)):
    """Values of a cell-centred 2-D field at (y, x) points, linear between the
    two nearest centres along each axis (clamped at the outermost centres);
    used to impose a reference field at off-grid points."""
    out = np.zeros(len(pts))
    coords = []
    for a in range(2):
        n = u.shape[a]
        s = np.clip((pts[:, a] - origin[a]) / (lengths[a] / n) - 0.5, 0.0, n - 1.0)
        i0 = np.minimum(np.floor(s).astype(int), max(n - 2, 0))
        coords.append((i0, s - i0, np.minimum(i0 + 1, n - 1)))
    (y0, ty, y1), (x0, tx, x1) = coords
    out = ((1 - ty) * ((1 - tx) * u[y0, x0] + tx * u[y0, x1]) + ty * ((1 - tx) * u[y1, x0] + tx * u[y1, x1]))
    return out


def run_burgers_paper(args):
    """The paper's Burgers reconstruction (Section 3.2): inviscid, [0, 1]^2,
    64 x 64, the reference solution imposed at 84 points on the edges of a
    rectangle; L-BFGS (history 50) with six levels (mODIL) against one level
    (plain ODIL), with and without U[0, 0.05] noise.  The reference is the
    discrete problem solved by the library itself: the initial row imposed at
    every cell, the loss minimised by L-BFGS until it vanishes."""
    import torch

    from paper_2303_04679_gb300 import inputs, modil
    torch.cuda.set_device(0)
    P = inputs.BURGERS_PAPER
    nt, nx = P["shape"]
    x = (np.arange(nx) + 0.5) / nx
    ic = inputs.burgers_paper_ic(x)
    fwd = modil.Desc("burgers", P["shape"], P["n_levels"], "f64", coef=(0.0,), domain=P["domain"],
                     meas_cell=np.arange(nx, dtype=np.int32), meas_value=ic)
    with modil.Problem(fwd) as p, modil.LBFGS(p, history=50) as opt:
        fh = opt.run(3000)
        u_ref = p.read_field()
    pts = inputs.rectangle_points()
    vals = bilinear_at(u_ref, pts)
    T, X = np.meshgrid((np.arange(nt) + 0.5) / nt, x, indexing="ij")
    (t0, t1), (x0, x1) = P["rect"]
    inside = (T >= t0) & (T <= t1) & (X >= x0) & (X <= x1)
    out = {"metric": "Burgers reconstruction: L-BFGS iterations and wall time to loss 1e-4, RMS error",
           "workload": "Section 3.2: inviscid Burgers, [0,1]^2, 64x64, 84 points on the edges of the "
                       "square [1/4,3/4]^2, FP64, L-BFGS history 50",
           "reference": {"loss": float(fh[-1]), "iterations": len(fh) - 1,
                         "max": float(u_ref.max()), "min": float(u_ref.min())},
           "runs": []}
    for noise in (0.0, 0.05):
        v = vals if noise == 0 else inputs.uniform_noise(vals, noise, seed=1)
        for L in (P["n_levels"], 1):
            d = modil.Desc("burgers", P["shape"], L, "f64", coef=(0.0,), domain=P["domain"], points=pts,
                           point_value=v)
            iters = min(args.steps, 2000)
            with modil.Problem(d) as p, modil.LBFGS(p, history=50) as opt:
                torch.cuda.synchronize()
                t0_ = time.perf_counter()
                hist = opt.run(iters)
                el = time.perf_counter() - t0_
                u = p.read_field()
            reach = next((k for k, val in enumerate(hist) if val <= 1e-4), None)
            dd = u - u_ref
            out["runs"].append({
                "levels": L, "noise": noise, "iterations": len(hist) - 1, "seconds": el,
                "ms_per_iteration": 1e3 * el / max(len(hist) - 1, 1), "final_loss": float(hist[-1]),
                "iterations_to_1e-4": reach,
                "rms_error": float(np.sqrt(np.mean(dd ** 2))),
                "rms_error_inside_rectangle": float(np.sqrt(np.mean(dd[inside] ** 2))),
                "loss_at": {str(k): float(hist[k]) for k in (10, 40, 100, 400, 1000, 2000) if k < len(hist)}})
    print(json.dumps(out), flush=True)


def run_small(args):
    """The two small configurations: Burgers reconstruction on 64 x 64 in FP64
    (4 levels, 200 measured cells) and the lid-driven cavity on 256^2 in FP32
    (8 levels, 1000 velocity samples), the latter also through the
    torch.autograd.Function over the hand-written adjoint with a torch Adam.
    L2 flushed before every timed step."""
    import torch

    from paper_2303_04679_gb300 import inputs, modil
    torch.cuda.set_device(0)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    K = min(args.steps, 2000)
    out_extra = {}
    from paper_2303_04679_gb300 import records
    if args.workload == "burgers":
        w = inputs.burgers_workload()
        nt, nx = w["shape"]
        # the reference field: the library's forward solve from the initial condition
        rec, rec_hist = records.burgers_record(nt, nx, w["n_levels"], w["nu"], w["amps"])
        out_extra["record"] = {"kind": "library forward solve (L-BFGS)", "iterations": len(rec_hist) - 1,
                               "loss": float(rec_hist[-1])}
        vals = rec.reshape(-1)[w["meas_cell"]]
        desc = modil.Desc("burgers", w["shape"], w["n_levels"], "f64", coef=(w["nu"],), meas_cell=w["meas_cell"],
                          meas_value=vals, lr=w["lr"])
        name = "Burgers reconstruction 64x64 space-time, 4 levels, FP64, Adam"
        dtype = "f64"
    else:
        # velocity samples of the library's converged forward solution
        (cu, cv, _), rec_hist = records.cavity_record(256, 8, 100.0)
        out_extra["record"] = {"kind": "library forward solve (L-BFGS, nested from 64^2)",
                               "iterations": len(rec_hist) - 1, "loss": float(rec_hist[-1])}
        w = inputs.cavity_workload(field=(cu, cv))
        desc = modil.Desc("ns2d", w["shape"], w["n_levels"], "f32", coef=w["coef"], meas_cell=w["meas_cell"],
                          meas_field=w["meas_field"], meas_value=w["meas_value"], lr=w["lr"])
        name = "lid-driven cavity 256^2, Re 100, 8 levels, FP32, Adam"
        dtype = "f32"
    with modil.Problem(desc) as p:
        ms = flushed_steps(lambda: p.step(1, read_loss=False), p.stream, flush, K, args.warmup)
        prof = np.array([p.profile_step() for _ in range(10)]).mean(axis=0)
        loss = float(p.eval_loss()[0, 0])
        launches = p.launches_per_step()
        if args.workload == "cavity":
            from paper_2303_04679_gb300.autograd import ModilParameters
            params = ModilParameters(p)
            opt = torch.optim.Adam(params.parameters(), lr=w["lr"])

            def ag_step():
                opt.zero_grad()
                params().backward()
                opt.step()
            ms_ag = flushed_steps(ag_step, torch.cuda.current_stream(), flush, min(K, 300), args.warmup)
            out_extra["autograd"] = {"ms_per_step": float(np.median(ms_ag)), "evals_per_s": 1e3 / float(np.median(ms_ag)),
                                     "note": "ModilLoss forward + backward (hand-written adjoint) + torch.optim.Adam, "
                                             "launched op by op from Python"}
            # the same autograd step captured once in a CUDA graph (the library's
            # launches join torch's capture through the stream waits) and replayed
            try:
                p2 = ModilParameters(p)
                opt2 = torch.optim.Adam(p2.parameters(), lr=w["lr"], capturable=True)
                side = torch.cuda.Stream()
                side.wait_stream(torch.cuda.current_stream())
                with torch.cuda.stream(side):
                    for _ in range(3):
                        opt2.zero_grad(set_to_none=True)
                        p2().backward()
                        opt2.step()
                torch.cuda.current_stream().wait_stream(side)
                graph = torch.cuda.CUDAGraph()
                opt2.zero_grad(set_to_none=True)
                with torch.cuda.graph(graph):
                    static_loss = p2()
                    static_loss.backward()
                    opt2.step()
                ms_g = flushed_steps(graph.replay, torch.cuda.current_stream(), flush, min(K, 300), args.warmup)
                out_extra["autograd_graph"] = {"ms_per_step": float(np.median(ms_g)),
                                               "evals_per_s": 1e3 / float(np.median(ms_g)),
                                               "loss_after": float(static_loss.item())}
            except Exception as e:  # report, keep the line
                out_extra["autograd_graph"] = {"error": str(e)[:300]}
    if args.workload == "burgers":
        # the configuration's plain Adam run (2000 steps) against L-BFGS with
        # a history of 50 (the paper's optimiser), both from zero levels
        with modil.Problem(desc) as pa:
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            pa.step(2000, read_loss=False)
            torch.cuda.synchronize()
            t_adam = time.perf_counter() - t0
            loss_adam = float(pa.eval_loss()[0, 0])

        def lbfgs_run(iters):
            with modil.Problem(desc) as pl, modil.LBFGS(pl, history=50) as opt:
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                h = opt.run(iters)
                return h, time.perf_counter() - t0
        hist, t_lb = lbfgs_run(400)
        reach = next((k for k, v in enumerate(hist) if v <= loss_adam), None)
        t_reach = lbfgs_run(reach)[1] if reach else None
        out_extra["lbfgs"] = {
            "history": 50, "iterations": len(hist) - 1, "seconds": t_lb,
            "ms_per_iteration": 1e3 * t_lb / max(len(hist) - 1, 1), "final_loss": float(hist[-1]),
            "adam_2000_steps": {"seconds": t_adam, "final_loss": loss_adam},
            "iterations_to_adam_final_loss": reach, "seconds_to_adam_final_loss": t_reach,
            "note": "host wall time, no L2 flush; L-BFGS line search reads the loss on the host"}
    step_ms = float(np.sum(ms) / K)
    peak, kind = measured_peak()
    nf = 3 if args.workload == "cavity" else 1
    fine = int(np.prod(w["shape"]))
    fine_bytes = nf * fine * ALG_BYTES_PER_PARAM + len(w["meas_cell"]) * ALG_BYTES_PER_MEAS
    ach = fine_bytes / (prof[0] * 1e-3) / 1e9
    out = {
        "metric": METRIC, "value": 1e3 / step_ms, "unit": UNIT, "n_gpus": 1, "steps": K, "warmup": args.warmup,
        "ms_per_step": step_ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": dtype,
        "data": "synthetic", "config": {"workload": name, "l2": "flushed before every timed step (256 MiB write)"},
        "fine_cells_per_s": fine * 1e3 / step_ms, "loss_final": loss,
        "kernel_ms": [float(v) for v in prof],
        "roofline": {"kernel": "fine_tile_fused", "bound": "hbm", "achieved": ach, "peak": peak, "peak_kind": kind,
                     "unit": "GB/s", "frac": ach / peak, "traffic": None, "alg_bytes_per_launch": fine_bytes},
        "gpu_launches": launches * K,
    }
    out.update(out_extra)
    print(json.dumps(out), flush=True)


def unet_train_flops(side, batch, base, levels, in_pad=8, out_ch=5):
    """FLOPs of one training step (forward, input and weight gradients) of the
    U-Net's contractions: 2 M K N per GEMM, three GEMMs per convolution (the
    first convolution has no input gradient)."""
    tot = 0
    first = True

    def conv(S, cin, cout, taps=27):
        nonlocal tot, first
        m = batch * S ** 3
        f = 2 * m * taps * cin * cout
        tot += f * (2 if first else 3)
        first = False
    for l in range(levels):
        conv(side >> l, in_pad if l == 0 else base << (l - 1), base << l)
        conv(side >> l, base << l, base << l)
    for l in range(levels - 2, -1, -1):
        conv(side >> l, (base << (l + 1)) + (base << l), base << l)
        conv(side >> l, base << l, base << l)
    conv(side, base, 16, taps=1)
    return tot


def run_unet(args):
    """U-Net training throughput on 64^3 (batch 2, 4 levels x 32 channels) and
    the tensor-core GEMM against the measured BF16 peak."""
    import torch

    from paper_2303_04679_gb300 import inputs, unet
    from paper_2303_04679_gb300 import warmstart as W
    torch.cuda.set_device(0)
    side, batch, base, levels = args.side, 2, 32, 4
    net = unet.UNet(side, batch=batch, in_ch=4, out_ch=5, base_ch=base, levels=levels, lr=1e-4)
    net.write_params(inputs.unet_params(W.param_shapes(levels, base), 0))
    rng = inputs.make_rng(1)
    x = torch.from_numpy(rng.normal(size=(batch, side, side, side, 4)).astype(np.float32)).cuda()
    y = torch.from_numpy(rng.normal(size=(batch, side, side, side, 5)).astype(np.float32)).cuda()
    for _ in range(max(3, args.warmup)):
        net.train_step(x, y, read_loss=False)
    torch.cuda.synchronize()
    K = max(1, min(args.steps, 200))
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    sampler = ClockSampler(0)
    sampler.start()
    time.sleep(0.25)
    a.record(net.stream)
    for _ in range(K):
        net.train_step(x, y, read_loss=False)
    b.record(net.stream)
    b.synchronize()
    clocks = sampler.stop()
    ms = a.elapsed_time(b) / K
    prof = net.profile_step(x, y)
    flops = unet_train_flops(side, batch, base, levels)
    # the GEMMs alone: the largest convolution of the network (decoder level 0,
    # 96 -> 32 channels: M = 2 side^3, K = 27 x 96, N = 32) and a square 8192^3
    gem = {}
    for name, (M, N, Kd) in {"conv_dec0": (batch * side ** 3, 32, 27 * 96), "square_8192": (8192, 8192, 8192)}.items():
        A = torch.randn(M, Kd, device="cuda").to(torch.bfloat16)
        B = torch.randn(N, Kd, device="cuda").to(torch.bfloat16)
        D = torch.empty(M, N, device="cuda", dtype=torch.float32)
        for _ in range(3):
            unet.gemm_bf16(A, B, D, mode=1)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(10):
            unet.gemm_bf16(A, B, D, mode=1)
        e1.record()
        e1.synchronize()
        t = e0.elapsed_time(e1) / 10
        gem[name] = {"M": M, "N": N, "K": Kd, "ms": t, "tflops": 2.0 * M * N * Kd / (t * 1e-3) / 1e12,
                     "operand_GBps": 2.0 * (M + N) * Kd / (t * 1e-3) / 1e9}
        del A, B, D
    net.close()
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        peak, kind = float(peaks["bf16_tflops"]), "measured"
    except (OSError, KeyError, ValueError):
        peak, kind = 1900.0, "fallback"
    sq = gem["square_8192"]
    out = {
        "metric": "U-Net training samples/s", "value": batch / (ms * 1e-3), "unit": "samples/s", "n_gpus": 1,
        "steps": K, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "bf16 (f32 accumulate)", "data": "synthetic",
        "config": {"workload": f"3-D U-Net training step, {side}^3, batch 2, 4 levels x 32 channels, Adam",
                   "flops_per_step": flops},
        "effective_tflops": flops / (ms * 1e-3) / 1e12,
        "launches_per_step": int(len(prof)),
        "gemm": gem,
        "roofline": {"kernel": "tc_gemm (square 8192^3)", "bound": "tensor", "achieved": sq["tflops"],
                     "peak": peak, "peak_kind": kind + " (bf16 burst)", "unit": "TFLOP/s",
                     "frac": sq["tflops"] / peak, "traffic": None},
        "clocks": clocks,
        "gpu_launches": int(len(prof)) * K,
    }
    print(json.dumps(out), flush=True)


def _fractions(args):
    from paper_2303_04679_gb300 import inputs
    shape, case = args
    return inputs.ns3d_body_fraction(shape, *case)


# Adam's learning rate by phases, [(steps, lr), ...]: at a constant 1e-3 the
# 128^3 body losses stall near 7e-3 (Adam's step size, not the problem); the
# decaying rate takes the references to ~1e-6 and the inverse problems below
# 1e-4
TRAIN_SCHEDULE = [(2000, 1e-3), (1000, 3e-4)]
REF_SCHEDULE = [(2000, 1e-3), (3000, 3e-4), (3000, 1e-4), (2000, 3e-5)]
INVERSE_SCHEDULE = [(2000, 1e-3), (2000, 3e-4), (3000, 1e-4), (3000, 3e-5)]


def run_warmstart(args):
    """Learned warm start of the 3-D body problem (the configured scale):
    plain-mODIL forward solutions around seeded ellipsoids on 64^3 (training
    data, R17), the U-Net (4 levels x 32 channels) trained on them by the
    library's kernels, then the 128^3 inverse problem (8 levels) from the
    wake slab of held-out ellipsoids, zero init against the network's
    prediction on level 2 (64^3) of the decomposition: steps and wall time to
    each loss threshold (inference included for the warm start) and the mean
    body-fraction error along the way."""
    import multiprocessing as mp

    from paper_2303_04679_gb300 import inputs
    side, Lf, big, Lb = 64, 7, 128, 8
    cases = [inputs.ns3d_ellipsoid(10000 + i) for i in range(args.train)]
    held = list(range(5, 5 + args.held_out))
    t0 = time.perf_counter()
    # body fractions on the host cores (a spawned pool, before any GPU work)
    with mp.get_context("spawn").Pool(min(16, os.cpu_count() or 1)) as pool:
        fracs = pool.map(_fractions, [((side,) * 3, c) for c in cases], chunksize=8)
        held_cases = [inputs.ns3d_ellipsoid(s) for s in held]
        held_fracs = pool.map(_fractions, [((big,) * 3, c) for c in held_cases])
    t_frac = time.perf_counter() - t0

    import torch

    from paper_2303_04679_gb300 import unet
    from paper_2303_04679_gb300 import warmstart as W
    torch.cuda.set_device(0)
    t0 = time.perf_counter()
    fields, fterms = W.forward_solves(cases, side, Lf, 0, fractions=fracs, schedule=TRAIN_SCHEDULE)
    t_data = time.perf_counter() - t0
    xs = np.stack([W.unet_input((side,) * 3, *W.slab((side,) * 3, 10000 + i, c, a, fields[i]), side)
                   for i, (c, a) in enumerate(cases)])
    norm = W.Normaliser(fields)
    ys = norm.to_net(fields)
    del fields
    net, hist, t_train = W.train(xs, ys, args.epochs, batch=2, lr=1e-3, base_ch=32, levels=4)
    prof = net.profile_step(torch.from_numpy(xs[:2]).cuda(), torch.from_numpy(ys[:2]).cuda())
    inf = unet.UNet(side, batch=1, in_ch=4, out_ch=5, base_ch=32, levels=4)
    inf.write_params(net.read_params())
    net.close()
    del xs, ys
    thresholds = [1e-2, 3e-3, 1e-3, 3e-4, 1e-4]
    results = []
    for seed, (c, a), chi_ref in zip(held, held_cases, held_fracs):
        lb = args.optimizer == "lbfgs"
        fb, tb = W.forward_solves([(c, a)], big, Lb, 0, fractions=[chi_ref], lbfgs_iters=args.fwd_iters if lb else 0,
                                  schedule=None if lb else REF_SCHEDULE)
        cells, fidx, vals = W.slab((big,) * 3, seed, c, a, fb[0])
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        pred = W.predict(inf, norm, W.unet_input((big,) * 3, cells, fidx, vals, side))
        torch.cuda.synchronize()
        t_inf = time.perf_counter() - t1
        desc = W.inverse_problem((big,) * 3, Lb, cells, fidx, vals)
        sched = None if lb else INVERSE_SCHEDULE
        hz, lz, cz = W.steps_to_losses(desc, W.zero_levels((big,) * 3, Lb), thresholds, args.steps,
                                       chi_ref=chi_ref, run_all=True, optimizer=args.optimizer, schedule=sched)
        hw, lw, cw = W.steps_to_losses(desc, W.warm_levels((big,) * 3, Lb, 1, pred), thresholds, args.steps,
                                       chi_ref=chi_ref, run_all=True, optimizer=args.optimizer, schedule=sched)
        at = lambda h, k: h[min(k, len(h) - 1)]  # noqa: E731
        results.append({
            "seed": seed, "forward_loss": float(tb[0][0]), "inference_s": t_inf,
            "zero": {str(t): hz[t] for t in thresholds},
            "warm": {str(t): (hw[t][0], hw[t][1] + t_inf) if hw[t] else None for t in thresholds},
            "loss_at_1000_3000_end": {"zero": [at(lz, 9), at(lz, 29), lz[-1]], "warm": [at(lw, 9), at(lw, 29), lw[-1]]},
            "chi_err_at_100_1000_3000_end": {"zero": [cz[0], at(cz, 9), at(cz, 29), cz[-1]],
                                             "warm": [cw[0], at(cw, 9), at(cw, 29), cw[-1]]}})
    summary = {}
    for t in thresholds:
        zs = [r["zero"][str(t)] for r in results]
        ws = [r["warm"][str(t)] for r in results]
        summary[str(t)] = {"zero_reached": sum(v is not None for v in zs), "warm_reached": sum(v is not None for v in ws),
                           "zero_median_s": float(np.median([v[1] for v in zs if v])) if any(zs) else None,
                           "warm_median_s": float(np.median([v[1] for v in ws if v])) if any(ws) else None,
                           "zero_median_steps": float(np.median([v[0] for v in zs if v])) if any(zs) else None,
                           "warm_median_steps": float(np.median([v[0] for v in ws if v])) if any(ws) else None}
    out = {
        "metric": "steps and wall time to loss 1e-4, warm-started (inference included) vs zero-init mODIL; "
                  "body-fraction error", "unit": "s", "n_gpus": 1,
        "steps": args.steps if args.optimizer == "lbfgs" else sum(s for s, _ in INVERSE_SCHEDULE), "warmup": 0,
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32 (mODIL), bf16/f32 (U-Net)", "data": "synthetic",
        "config": {"workload": "body-shape inverse problem 128^3, 8 levels; U-Net 4 levels x 32 ch on 64^3",
                   "training_ellipsoids": args.train, "epochs": args.epochs, "held_out_seeds": held,
                   "optimizer": args.optimizer,
                   "adam_schedules": {"training_64": TRAIN_SCHEDULE, "reference_128": REF_SCHEDULE,
                                      "inverse_128": INVERSE_SCHEDULE}},
        "summary": summary,
        "mean_chi_err_end": {"zero": float(np.mean([r["chi_err_at_100_1000_3000_end"]["zero"][-1] for r in results])),
                             "warm": float(np.mean([r["chi_err_at_100_1000_3000_end"]["warm"][-1] for r in results]))},
        "training": {"fractions_s": t_frac, "forward_solves_s": t_data, "unet_train_s": t_train,
                     "unet_loss_first_last": [hist[0], hist[-1]],
                     "forward_loss_median": float(np.median(fterms[:, 0])),
                     "unet_step_ms": float(np.sum(prof)), "unet_launches_per_step": int(len(prof))},
        "cases": results,
    }
    print(json.dumps(out), flush=True)


def main():
    args = parse()
    from paper_2303_04679_gb300 import inputs
    if args.workload == "batched-burgers":
        if args.impl == "reference":
            run_reference_batched(args)
        else:
            run_batched(args)
        return
    if args.workload == "body":
        run_body(args)
        return
    if args.workload == "warmstart":
        run_warmstart(args)
        return
    if args.workload == "unet":
        run_unet(args)
        return
    if args.workload in ("burgers", "cavity"):
        run_small(args)
        return
    if args.workload == "poisson":
        run_poisson(args)
        return
    if args.workload == "burgers-paper":
        run_burgers_paper(args)
        return
    args.tile = args.tile or "32x32"
    if args.impl == "reference":
        run_reference(args, heat_reference_workload())
        return

    import torch
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    from paper_2303_04679_gb300 import modil, records

    # the temperature record: the library's forward solve with the nodes of
    # the reference conductivity held fixed (outside every timed region)
    t0 = time.perf_counter()
    rec, rec_hist = records.heat_record()
    t_rec = time.perf_counter() - t0
    w = inputs.heat_workload(field=rec)
    params, fine = workload_sizes(w)
    n_meas = len(w["meas_cell"])
    step_alg_bytes = params * ALG_BYTES_PER_PARAM + n_meas * ALG_BYTES_PER_MEAS
    fine_alg_bytes = fine * ALG_BYTES_PER_PARAM + n_meas * ALG_BYTES_PER_MEAS

    prob = modil.Problem(make_desc(modil, w, args.tile))
    stream = prob.stream
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    launches = prob.launches_per_step()

    def flush_l2():
        with torch.cuda.stream(stream):
            flush.zero_()

    for _ in range(args.warmup):
        flush_l2()
        prob.step(1, read_loss=False)
    torch.cuda.synchronize()

    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    sampler = ClockSampler(local)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    sampler.start()
    time.sleep(0.25)
    wall0 = time.perf_counter()
    for a, b in evs:
        flush_l2()
        a.record(stream)
        prob.step(1, read_loss=False)
        b.record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    clocks = sampler.stop()
    if world > 1:
        torch.distributed.barrier()
    step_ms = [a.elapsed_time(b) for a, b in evs]
    tot_ms = sum(step_ms)
    tot_ms = max_over_ranks(tot_ms, world)
    terms = prob.eval_loss()[0]

    # per-kernel device times of a step launched kernel by kernel (cold L2)
    prof = []
    for _ in range(max(1, args.profile_steps)):
        flush_l2()
        torch.cuda.synchronize()
        prof.append(prob.profile_step())
    prof = np.array(prof)
    kern_ms = prof.mean(axis=0)
    names = (["fine_tile_fused"] + [f"restrict_adam_L{l + 1}" for l in range(1, len(kern_ms) - 1)]
             + ["coarse_tail"])
    dom = int(np.argmax(kern_ms))
    peak, peak_kind = measured_peak()
    dom_bytes = fine_alg_bytes if dom == 0 else None
    achieved = dom_bytes / (kern_ms[dom] * 1e-3) / 1e9 if dom_bytes else None
    traffic = None
    tfile = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(tfile):
        try:
            from paper_2303_04679_gb300 import build as bld
            tj = json.load(open(tfile))["fine_tile_fused"]
            if tj.get("source_hash") == bld.source_hash(tj["sources"]):
                traffic = tj.get("bytes_per_launch")
        except Exception:
            traffic = None
    prob.close()

    # end to end through the public API, host buffers, copies inside the timed region
    e2e_steps = min(args.steps, 2000)
    levels0 = [torch.zeros(s, dtype=torch.float32).pin_memory()
               for s in inputs.level_shapes(w["shape"], w["n_levels"])]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    p2 = modil.Problem(make_desc(modil, w, args.tile))
    for lvl, a in enumerate(levels0):
        modil._check(modil.LIB.modil_write_level(p2._h, 0, 0, lvl, a.data_ptr(),
                                                 a.numel() * 4, 0))
    for _ in range(e2e_steps):
        p2.step(1, read_loss=True)
    field = p2.read_field()
    e2e_s = time.perf_counter() - t0
    p2.close()
    h2d = (sum(a.numel() * 4 for a in levels0) + n_meas * 8 + w["shape"][1] * 4 +
           len(w["knodes"]) * 4)
    d2h = 32 * e2e_steps + field.nbytes

    value = job_throughput(args.steps, world, tot_ms)
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": tot_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": heat_config(args, w),
        "fine_cells_per_s": value * fine,
        "effective_step_GBps": step_alg_bytes * value / world / 1e9,
        "hbm_frac_step": step_alg_bytes * value / world / 1e9 / peak,
        "step_ms_median": statistics.median(step_ms),
        "wall_s": wall,
        "loss_final": float(terms[0]),
        "kernel_ms": {n: float(v) for n, v in zip(names, kern_ms)},
        "roofline": {"kernel": names[dom], "bound": "hbm", "achieved": achieved, "peak": peak,
                     "peak_kind": peak_kind, "unit": "GB/s",
                     "frac": (achieved / peak) if achieved else None, "traffic": traffic,
                     "alg_bytes_per_launch": dom_bytes},
        "clocks": clocks,
        "gpu_launches": launches * args.steps,
        "e2e": {"value": e2e_steps / e2e_s, "unit": UNIT,
                "h2d_bytes_per_step": h2d / e2e_steps, "d2h_bytes_per_step": d2h / e2e_steps,
                "steps": e2e_steps, "note": "create + upload + steps with loss read back + field read"},
    }
    out["record"] = {"kind": "library forward solve (k_fixed, L-BFGS nested from 64^2)",
                     "finest_iterations": len(rec_hist) - 1, "loss": float(rec_hist[-1]), "seconds": t_rec}
    # conductivity inference to a tolerance in the setting of Section 3.4: the
    # inverse problem on 64 x 64 cells, 500 measured cells without noise, by
    # Adam; on the 512 x 512 configuration with seven levels and noisy data
    # Adam does not identify k within 10 000 steps (reported beside it), the
    # device L-BFGS does (HEAT_LBFGS)
    rec64, _ = records.heat_record(64, 64, 4, depth=1)
    w64 = inputs.heat_workload(64, 64, 4, field=rec64, frac=500 / 4096, sigma=0.0)
    w64["lr"] = 3e-3
    out["inference"] = heat_inference(modil, w64, args)
    out["inference_512"] = heat_inference(modil, w, args)
    out["inference_512_lbfgs"] = heat_inference_lbfgs(modil, w, args)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        n, el = time_oracle(w, args.cpu_seconds)
        out["cpu_baseline"] = {"value": n / el, "unit": UNIT, "cores": blas_threads(),
                               "kind": "oracle",
                               "sample": f"{n} full oracle Adam steps of the workload in {el:.1f} s "
                                         f"({cpu_model()}, {os.cpu_count()} host cores)"}
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
