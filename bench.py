#!/usr/bin/env python
"""Benchmark of one coupling step of the actuator-line transfer operators.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload flume|canopy|plain|batched|serve]
                    [--eps 2.0] [--impl ours|reference]

A step is one call of al_sample_drag_spread (sampling, Morison line force,
relaxation, normalised Gaussian projection of every line) on one instance
whose fields and points are resident in HBM.  Under torchrun every rank runs
its own independent instance (seed = rank) with no collective on the data
path (weak scaling); timing is the max over ranks.

Prints ONE JSON line (rank 0).  Throughput `value` is coupling steps/s over
all ranks, device-timed with CUDA events; L2 is flushed (256 MiB write)
between timed steps, outside the events.  `e2e` is the same metric through
the public API with pinned host buffers (al_step_host: every step's inputs
copied in and S and F copied out inside the timed region; consecutive steps
on two alternating streams).  `roofline` reports the projection kernel k_spread against
the measured HBM copy bandwidth (its algorithmic bytes: the dense S write
plus the per-node data, over its event-timed duration); it also carries the
whole step's fraction (the step's algorithmic bytes over the step time) and
the weights pass against the FP32 FMA peak of the SMs (its algorithmic
operations per (cell, line) pair times the pairs).  The default workload is
the wave flume (1024 x 256 x 128 cells, 4000 stems of 80 CVs), the largest
single-GPU configuration.
"""
import argparse
import hashlib
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



def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--workload", default="flume", choices=["flume", "canopy", "plain", "batched", "serve"])
    ap.add_argument("--instances", type=int, default=64, help="batched: number of instances")
    ap.add_argument("--sims", type=int, default=256, help="serve: number of simulations")
    ap.add_argument("--sim-steps", type=int, default=100, help="serve: steps per simulation")
    ap.add_argument("--rates", default="100,200,500,1000,2000,5000,10000,20000,50000",
                    help="serve: arrival rates (1/s)")
    ap.add_argument("--plain-rates", default="100,50000", help="serve: rates that also run the plain path")
    ap.add_argument("--window", type=float, default=8.0, help="serve: seconds of each rate's request stream")
    ap.add_argument("--slots", type=int, default=256, help="serve: simulations resident at a time")
    ap.add_argument("--budget-gb", type=float, default=40.0, help="serve: HBM budget for resident simulations")
    ap.add_argument("--eps", type=float, default=2.0, help="canopy kernel width in cells")
    ap.add_argument("--reduced", action="store_true",
                    help="a reduced grid of the same workload (flume 256x64x128 with 20x8 stems, canopy "
                         "128x64x128 with 10x10 stems): for profiler captures, not a bench line")
    ap.add_argument("--inertia", action="store_true",
                    help="add the Morison inertia term (accelerating fluid and beams, C_Mn = 1, C_Mt = 0.1)")
    ap.add_argument("--sample", default="trilinear", choices=["trilinear", "cell", "gauss"],
                    help="sampling operator of both velocity samples (cell: the containing cell; gauss: Gaussian volume average)")
    ap.add_argument("--projection", default="nearest", choices=["nearest", "integrated"],
                    help="projection: nearest segment (the paper's) or segment-integrated 3-D Gaussian")
    ap.add_argument("--reflect", type=int, default=0,
                    help="faces that reflect the kernel (bit mask: 1 x-, 2 x+, 4 y-, 8 y+, 16 z-, 32 z+)")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--split", default="none", choices=["none", "slab"],
                    help="slab: one instance split along x over the ranks (strong scaling); "
                         "none: one instance per rank (weak scaling)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-tune", action="store_true", help="skip the autotuner (default options)")
    ap.add_argument("--no-variants", action="store_true", help="skip timing the scatter projection")
    ap.add_argument("--weights", choices=["brick", "segment"], default=None, help="fix the weights pass (no tuning)")
    ap.add_argument("--brick-z", type=int, choices=[4, 8, 16], default=None, help="fix the brick height (no tuning)")
    ap.add_argument("--column", choices=["on", "off"], default=None,
                    help="fix the column march on or off (no tuning)")
    ap.add_argument("--records", choices=["on", "off"], default=None,
                    help="fix whether the segment pass records pairs for the spread to replay (no tuning)")
    return ap.parse_args()


def _workload(name, seed, eps, reduced=False):
    from paper_2609_39443_b300 import workloads as W
    if name == "canopy":
        return W.make_canopy(seed, eps, nx=128, ny=64, n_sx=10, n_sy=10) if reduced else W.make_canopy(seed, eps)
    if name == "flume":
        return W.make_flume(seed, nx=256, ny=64, nz=128, n_sx=20, n_sy=8) if reduced else W.make_flume(seed)
    return W.make_plain(seed)


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6400.0, "fallback"


def _kernel_hash():
    h = hashlib.sha256()
    for f in ("paper_2609_39443_b300/csrc/al_kernels.cuh", "paper_2609_39443_b300/csrc/al_cm.cuh",
              "paper_2609_39443_b300/csrc/al_api.cu"):
        h.update(open(os.path.join(ROOT, f), "rb").read())
    return h.hexdigest()[:16]


def _traffic(workload_name, kernel="k_spread", options=None):
    """dram bytes per launch of a kernel from a committed ncu summary, if it
    was taken on the current kernel source with the same options (weights
    pass, brick height, records)."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p))
    e = d.get(f"{workload_name}/{kernel}")
    if not e or e.get("kernel_hash") != _kernel_hash():
        return None
    if options is not None and "options" in e:
        if any(e["options"].get(k) != options.get(k) for k in ("weights", "brick_z", "records", "column_march")):
            return None
    return e.get("dram_bytes_per_launch")


class Clocks:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=2)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                sm.append(float(r[0]))
                mx.append(float(r[1]))
                for n, v in zip(names, r[4:8]):
                    if v.lower().startswith("active"):
                        reasons.add(n)
            except (ValueError, IndexError):
                pass
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# FP32 ALU peak: 148 SMs x 128 FP32 lanes x 2 flop (FMA) x 2.032 GHz
ALU_PEAK_TFLOPS = 148 * 128 * 2 * 2.032e9 / 1e12
# operations of one (cell, segment) pair of the weights pass by definition:
# offset to the segment start (3), foot parameter x.D / |D|^2 (6), foot
# offset and squared distance (6 + 5), Gaussian exp(-(r/eps)^2) eta0 (3),
# the two node weights (1 - s) eta, s eta (3)
FLOP_PER_PAIR = 26


def _algorithmic_bytes(wl):
    """Bytes the projection kernel must move per launch: the dense S write
    (3 components of every cell) plus, per actuator point, its position and
    normalised force (staged once per brick that needs it; counted once)."""
    es = 8 if wl.grid.precision == "fp64" else 4
    return 3 * es * wl.grid.n_cells + wl.beams.n_points * (3 * es + 3 * es)


def _step_algorithmic_bytes(wl):
    """Bytes one whole coupling step must move: the spread's (dense S write,
    per-node position and normalised force), the field stencils of the two
    samples of every point (8 cells x (3 velocity components + alpha) each,
    an upper bound that ignores sharing between points), and per point its
    velocity and CV length in, its load out, the relaxation state read and
    written and the FP64 nodal weight."""
    es = 8 if wl.grid.precision == "fp64" else 4
    ncomp = 4 if wl.grid.has_alpha else 3
    npt = wl.beams.n_points
    stencils = 2 * 8 * ncomp * es * npt
    points = npt * (3 * es + 8 + 3 * es + 2 * 3 * es + 8)
    return _algorithmic_bytes(wl) + stencils + points


def _cpu_baseline(wl, budget_s=12.0):
    """The FP64 oracle as it stands, on this host's cores, on a bounded
    sample of the same workload.  Returns (steps/s, cores, sample text)."""
    import oracle
    nl = wl.beams.n_lines
    # sample: every m-th line's projection plus all points' sampling; the
    # step rate is scaled by the fraction of lines projected
    t0 = time.perf_counter()
    oracle.point_step(wl.grid, wl.beams, wl.step)
    t_point = time.perf_counter() - t0
    m = 1
    mask = np.ones(nl, np.uint8)
    est = None
    while True:
        t0 = time.perf_counter()
        ps = oracle.point_step(wl.grid, wl.beams, wl.step)
        Psp = wl.step.P if wl.step.P_spread is None else wl.step.P_spread
        oracle.project(wl.grid, wl.beams, Psp, ps["F"], line_mask=mask)
        dt = time.perf_counter() - t0
        frac = mask.sum() / max(nl, 1)
        est = dt - t_point
        if dt > 2.0 and m == 1 and nl > 1:
            m = int(np.ceil(dt / 2.0))
            mask = np.zeros(nl, np.uint8)
            mask[::m] = 1
            continue
        break
    reps, tot = 0, 0.0
    while tot < budget_s and reps < 50:
        t0 = time.perf_counter()
        ps = oracle.point_step(wl.grid, wl.beams, wl.step)
        oracle.project(wl.grid, wl.beams, Psp, ps["F"], line_mask=mask)
        tot += time.perf_counter() - t0
        reps += 1
    per = tot / reps
    t_full = t_point + (per - t_point) / frac if frac < 1 else per
    cores = os.cpu_count()
    sample = (f"{reps} oracle steps of {wl.name}" if frac >= 1 else
              f"{reps} oracle steps of {wl.name} projecting every {m}-th line ({int(mask.sum())}/{nl}); "
              f"step time scaled by the projected-line fraction")
    del est
    return 1.0 / t_full, cores, sample


def run_reference(a):
    """Reference arm: the FP64 oracle on the host cores (rank 0 only)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    wl = _workload(a.workload, 0, a.eps, a.reduced)
    v, cores, sample = _cpu_baseline(wl, budget_s=max(5.0, min(60.0, 2.0 * (a.steps + a.warmup))))
    line = {"impl": "reference", "metric": "coupling steps/s", "value": v, "unit": "steps/s",
            "n_gpus": a.gpus, "steps": a.steps, "warmup": a.warmup, "ms_per_step": 1e3 / v,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": wl.name},
            "cpu_baseline": {"value": v, "unit": "steps/s", "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": "steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(a):
    import torch
    from paper_2609_39443_b300.ranks import instance_seed, max_over_ranks, rank_env
    world, rank, local = rank_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    from paper_2609_39443_b300 import build as B
    if B.stale():
        if rank == 0:
            B.build()
        if dist:
            dist.barrier()
    from paper_2609_39443_b300.al import Instance, PHASES, ST_COLUMN, ST_SUPPORT

    wl = _workload(a.workload, instance_seed(rank), a.eps, a.reduced)
    if a.inertia:
        from paper_2609_39443_b300 import workloads as W
        wl = W.with_inertia(wl, 1000 + instance_seed(rank))
    if a.sample != "trilinear":
        from paper_2609_39443_b300 import workloads as W
        wl = W.with_sample_mode(wl, a.sample)
    if a.projection != "nearest":
        from paper_2609_39443_b300 import workloads as W
        wl = W.with_projection(wl, a.projection)
    if a.reflect:
        from paper_2609_39443_b300 import workloads as W
        wl = W.with_reflect(wl, a.reflect)
    inst = Instance(wl, device=f"cuda:{local}")
    tuned = {"weights": "brick", "brick_z": 8, "autotuned": False}
    if a.weights or a.brick_z or a.records or a.column:
        from paper_2609_39443_b300.al import OPT_BRICK_Z, OPT_COLUMN, OPT_RECORD, OPT_WEIGHTS
        tuned = {"weights": a.weights or "brick", "brick_z": a.brick_z or 8, "records": a.records != "off",
                 "column_march": a.column != "off", "autotuned": False}
        inst.grid.set_option(OPT_WEIGHTS, 1 if tuned["weights"] == "segment" else 0)
        inst.grid.set_option(OPT_BRICK_Z, tuned["brick_z"])
        inst.grid.set_option(OPT_RECORD, 1 if tuned["records"] else 0)
        inst.grid.set_option(OPT_COLUMN, 1 if tuned["column_march"] else 0)
    elif not a.no_tune:
        wmode, bz, rec, col = inst.autotune(trials=4)
        tuned = {"weights": "segment" if wmode else "brick", "brick_z": bz, "records": bool(rec),
                 "column_march": bool(col), "autotuned": True}
    if a.reflect:                                    # the library takes the brick passes for it
        tuned.update(weights="brick", records=False, column_march=False)
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=f"cuda:{local}")

    for _ in range(a.warmup):
        inst.status.zero_()
        inst.step()
    torch.cuda.synchronize()
    supp = int(inst.status[ST_SUPPORT].item())
    tuned["column_march"] = int(inst.status[ST_COLUMN].item()) > 0       # bricks that took it in the last step

    ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(a.steps)]
    ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(a.steps)]
    phases = np.zeros(len(PHASES))
    clocks = Clocks(local)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    launches0 = inst.grid.launches()
    for k in range(a.steps):
        flush.zero_()
        ev0[k].record(stream)
        inst.step()
        ev1[k].record(stream)
    torch.cuda.synchronize()
    launches = inst.grid.launches() - launches0      # the library's own kernels, counted as enqueued
    if dist:
        dist.barrier()
    clk = clocks.stop()
    step_ms = [e0.elapsed_time(e1) for e0, e1 in zip(ev0, ev1)]
    # the phases from as many steps again with the library's per-phase events
    # (events between the phases, so these steps run a little longer than the
    # timed ones)
    inst.grid.trace(True)
    for k in range(a.steps):
        flush.zero_()
        inst.step()
        phases += np.array(inst.grid.trace_last())
    torch.cuda.synchronize()
    total_s = sum(step_ms) / 1e3
    total_s = max_over_ranks([total_s], dist, f"cuda:{local}")[0]
    value = world * a.steps / total_s
    ph = phases / a.steps
    spread_s = ph[PHASES.index("spread")] / 1e3

    # ---- the quasi-static beam reconstruction on this step's forces: time per
    # call through the Python binding (launch overhead included; the kernel's
    # own device time is in the committed launch list) ----------------------
    beam_ms = None
    if a.workload in ("canopy", "flume"):
        P_out = torch.empty_like(inst.P)
        EI = np.full(wl.beams.n_lines, 5e-3)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        inst.grid.beam_quasistatic(EI, (0.0, 0.0, 1.0), inst.P, inst.F, P_out)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(10):
            inst.grid.beam_quasistatic(EI, (0.0, 0.0, 1.0), inst.P, inst.F, P_out)
        e1.record(stream)
        torch.cuda.synchronize()
        beam_ms = e0.elapsed_time(e1) / 10

    # ---- end to end through the public API with host buffers -----------------
    # al_step_host per step: the step's inputs copied in from pinned host
    # memory, the step, S and F copied back, on one stream; consecutive steps
    # alternate two streams and two device buffer sets, so one step's copies
    # overlap the other's (the library keeps the steps in call order)
    e2e = None
    if not a.no_e2e:
        def pin(x):
            return None if x is None else torch.as_tensor(np.ascontiguousarray(x)).pin_memory()
        host_in = {"U": pin(wl.step.U), "P": pin(wl.step.P), "Pdot": pin(wl.step.Pdot), "alpha": pin(wl.step.alpha),
                   "U_prev": pin(getattr(wl.step, "U_prev", None)), "Pddot": pin(getattr(wl.step, "Pddot", None)),
                   "P_spread": pin(wl.step.P_spread),
                   "tangent": pin(wl.step.tangent) if wl.beams.tangents_given else None}
        host_out = [{"S": torch.empty(inst.S.shape, dtype=inst.S.dtype).pin_memory(),
                     "F": torch.empty(inst.F.shape, dtype=inst.F.dtype).pin_memory()} for _ in range(2)]
        dsets = [inst.own_buffers(), inst.buffers()]
        streams = [torch.cuda.Stream(device=f"cuda:{local}") for _ in range(2)]
        h2d = sum(int(t.numel() * t.element_size()) for t in host_in.values() if t is not None)
        d2h = int(host_out[0]["S"].numel() * host_out[0]["S"].element_size() +
                  host_out[0]["F"].numel() * host_out[0]["F"].element_size())
        n_e2e = max(4, min(a.steps, 10))

        def e2e_step(k):
            inst.step_host({**host_in, **host_out[k % 2]}, dsets[k % 2], stream=streams[k % 2])

        inst.grid.trace(False)                       # as a caller runs it: no per-phase events
        for k in range(2):
            e2e_step(k)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        t0 = time.perf_counter()
        for k in range(n_e2e):
            e2e_step(k)
        torch.cuda.synchronize()
        te = time.perf_counter() - t0
        inst.grid.trace(True)
        te = max_over_ranks([te], dist, f"cuda:{local}")[0]
        e2e = {"value": world * n_e2e / te, "unit": "steps/s", "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "call": "al_step_host, two streams and two device buffer sets alternating"}
        del dsets

    # ---- the scatter-with-atomics projection on the same instance (comparison) ----
    variants = None
    if not a.no_variants and not a.reflect:          # the reflected kernel always gathers
        from paper_2609_39443_b300.al import OPT_SPREAD, SPREAD_GATHER, SPREAD_SCATTER
        variants = {}
        for name, mode in (("gather", SPREAD_GATHER), ("scatter_atomics", SPREAD_SCATTER)):
            inst.grid.set_option(OPT_SPREAD, mode)
            acc = np.zeros(len(PHASES))
            for k in range(3 + 5):
                flush.zero_()
                inst.step()
                if k >= 3:
                    acc += np.array(inst.grid.trace_last())
            variants[name] = {"projection_ms": float(acc[PHASES.index("spread")] / 5),
                              "step_ms": float(acc.sum() / 5)}
        inst.grid.set_option(OPT_SPREAD, SPREAD_GATHER)

    peak, peak_kind = _peaks()
    alg = _algorithmic_bytes(wl)
    achieved = alg / spread_s / 1e9
    cmk = bool(tuned.get("column_march"))
    spread_kernel = "k_cm_spread" if cmk else "k_spread"
    weights_kernel = "k_cm_weights" if cmk else ("k_weights" if tuned["weights"] == "segment" else "k_bweights")
    traffic = _traffic(wl.name, spread_kernel, options=tuned)
    weights_s = ph[PHASES.index("weights")] / 1e3
    step_alg = _step_algorithmic_bytes(wl)
    step_gbs = step_alg / (total_s / a.steps) / 1e9 * world
    flop = supp * FLOP_PER_PAIR
    w_tf = flop / weights_s / 1e12 if weights_s > 0 else 0.0
    roofline = {"bound": "hbm", "kernel": spread_kernel, "achieved": achieved, "peak": peak,
                "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / peak,
                "algorithmic_bytes": alg, "traffic": traffic,
                "step": {"bound": "hbm", "achieved": step_gbs, "peak": peak, "unit": "GB/s",
                         "frac": step_gbs / peak, "algorithmic_bytes": step_alg,
                         "ms": 1e3 * total_s / a.steps},
                "weights_pass": {"bound": "alu", "kernel": weights_kernel,
                                 "achieved": w_tf, "peak": ALU_PEAK_TFLOPS,
                                 "peak_kind": "derived (148 SMs x 128 FP32 lanes x FMA x 2.032 GHz)",
                                 "unit": "TFLOP/s", "frac": w_tf / ALU_PEAK_TFLOPS, "algorithmic_flop": flop,
                                 "ms": 1e3 * weights_s,
                                 "traffic": _traffic(wl.name, weights_kernel, tuned)}}
    cpu = None
    if rank == 0 and world == 1 and not a.no_cpu:
        v, cores, sample = _cpu_baseline(wl)
        cpu = {"value": v, "unit": "steps/s", "cores": cores, "kind": "oracle", "sample": sample}
    if rank == 0:
        line = {"metric": "coupling steps/s", "value": value, "unit": "steps/s", "n_gpus": world,
                "steps": a.steps, "warmup": a.warmup, "ms_per_step": 1e3 * total_s / a.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f64" if wl.grid.precision == "fp64" else "f32", "data": "synthetic",
                "config": {"workload": wl.name, "cells": wl.grid.n_cells, "points": wl.beams.n_points,
                           "inertia": bool(a.inertia), "sample": a.sample, "projection": a.projection, "reflect": a.reflect,
                           "lines": wl.beams.n_lines, "parallelism": f"{world} independent instances",
                           "l2": "flushed between timed steps (256 MiB write)", "options": tuned},
                "kernel_cell_updates_per_s": supp * value,
                "support_pairs_per_step": supp,
                "phases_ms": {k: float(v) for k, v in zip(PHASES, ph)},
                "phases_from": "as many steps again after the timed ones, with per-phase CUDA events",
                "roofline": roofline,
                "projection_variants": variants,
                "beam_quasistatic_call_ms": beam_ms,
                "cpu_baseline": cpu, "e2e": e2e, "clocks": clk,
                "gpu_launches": launches * world}
        print(json.dumps(line), flush=True)
    inst.close()
    if dist:
        dist.destroy_process_group()


def run_slab(a):
    """One flume (or canopy) split along x over the N ranks (strong scaling):
    each rank steps its slab, the ranks all-reduce the fixed-point partial
    weights (NCCL, int64 sum) between the two phases of the step."""
    import torch
    from paper_2609_39443_b300 import slab
    from paper_2609_39443_b300.ranks import max_over_ranks, rank_env
    world, rank, local = rank_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    wl = _workload(a.workload, 0, a.eps, a.reduced)       # the same instance on every rank
    sr = slab.SlabRank(wl, world, rank, device=f"cuda:{local}")
    glob = torch.zeros(max(wl.beams.n_points, 1), dtype=torch.int64, device=f"cuda:{local}")

    def step():
        sr.begin()
        glob.zero_()
        sr.partial(glob)
        if dist:
            dist.all_reduce(glob)
        sr.end(glob)

    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=f"cuda:{local}")
    for _ in range(a.warmup):
        step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = Clocks(local)
    clocks.start()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(a.steps)]
    launches0 = sr.inst.grid.launches()
    for e0, e1 in ev:
        flush.zero_()
        e0.record(stream)
        step()
        e1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clk = clocks.stop()
    launches = sr.inst.grid.launches() - launches0
    total_s = sum(e0.elapsed_time(e1) for e0, e1 in ev) / 1e3
    total_s = max_over_ranks([total_s], dist, f"cuda:{local}")[0]
    if rank == 0:
        p = sr.plan
        line = {"metric": "coupling steps/s", "value": a.steps / total_s, "unit": "steps/s", "n_gpus": world,
                "steps": a.steps, "warmup": a.warmup, "ms_per_step": 1e3 * total_s / a.steps,
                "higher_is_better": True, "scaling": "strong", "vs_baseline": None, "dtype": "f32",
                "data": "synthetic",
                "config": {"workload": wl.name, "cells": wl.grid.n_cells, "points": wl.beams.n_points,
                           "parallelism": f"x-slabs over {world} ranks, int64 all-reduce of partial weights",
                           "rank0_slab": {"owned": [p.x0, p.x1], "local": [p.lx0, p.lx1], "halo": p.halo,
                                          "lines": int(len(p.lines))},
                           "l2": "flushed between timed steps (256 MiB write)"},
                "clocks": clk, "gpu_launches": launches * world}
        print(json.dumps(line), flush=True)
    sr.close()
    if dist:
        dist.destroy_process_group()


def run_batched(a):
    """64 independent instances of uneven size: one batched launch sequence
    (CUDA graph) per step vs one launch sequence per instance."""
    import torch
    from paper_2609_39443_b300 import workloads as W
    from paper_2609_39443_b300.al import Batch, Instance
    from paper_2609_39443_b300.ranks import instance_seed, max_over_ranks, rank_env
    world, rank, local = rank_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    wls = W.make_batched(instance_seed(rank), a.instances)
    insts = [Instance(w, device=f"cuda:{local}") for w in wls]
    # tile sizes and weight pass: each instance tuned alone (used by the
    # per-instance launches), then the batch's brick height and persistent grid
    choices = [i.autotune(trials=1)[:2] for i in insts] if not a.no_tune else [(0, 8)] * len(insts)
    batch = Batch(insts, use_graph=True)
    batch_choice = batch.autotune(trials=1) if not a.no_tune else (8, 0)
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=f"cuda:{local}")

    def timed(fn, steps):
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for e0, e1 in ev:
            flush.zero_()
            e0.record(stream)
            fn()
            e1.record(stream)
        torch.cuda.synchronize()
        return sum(e0.elapsed_time(e1) for e0, e1 in ev) / 1e3

    def per_instance():
        for i in insts:
            i.step()

    for _ in range(a.warmup):
        batch.run()
        per_instance()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = Clocks(local)
    clocks.start()
    launches0 = batch.launches()
    t_batch = timed(batch.run, a.steps)
    launches = batch.launches() - launches0          # the library's own kernels (graph replays)
    t_plain = timed(per_instance, a.steps)
    clk = clocks.stop()
    t_batch, t_plain = max_over_ranks([t_batch, t_plain], dist, f"cuda:{local}")
    n = len(insts)
    value = world * n * a.steps / t_batch
    cells = sum(w.grid.n_cells for w in wls)
    pts = sum(w.beams.n_points for w in wls)
    if rank == 0:
        line = {"metric": "coupling steps/s", "value": value, "unit": "instance-steps/s", "n_gpus": world,
                "steps": a.steps, "warmup": a.warmup, "ms_per_step": 1e3 * t_batch / a.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                "data": "synthetic",
                "config": {"workload": f"batched_{n}_instances", "cells": cells, "points": pts,
                           "parallelism": f"{world} independent batches",
                           "l2": "flushed between timed steps (256 MiB write)"},
                "per_instance_launch_steps_per_s": world * n * a.steps / t_plain,
                "batched_speedup": t_plain / t_batch, "clocks": clk,
                "tuning": {"batch_brick_z": batch_choice[0], "batch_ctas_per_sm": batch_choice[1],
                           "instance_brick_z": {str(z): sum(1 for c in choices if c[1] == z) for z in (4, 8, 16)},
                           "instance_segment_weights": sum(1 for c in choices if c[0] == 1)},
                "gpu_launches": launches * world}
        print(json.dumps(line), flush=True)
    batch.close()
    for i in insts:
        i.close()


def run_serve(a):
    """Poisson-arriving coupling-step requests from many simulations (256 x
    100 steps by default): continuous batching through the library's server
    vs one request at a time.  A rate's run takes the first rate x --window
    seconds of its request stream (all of it when that is shorter), so that
    rates below saturation show service latency, not queueing, within
    minutes.  The batched form on the same simulations (one Batch of up to
    64, stepped back to back) gives the device's instance-steps/s for
    comparison."""
    import torch
    from paper_2609_39443_b300 import workloads as W
    from paper_2609_39443_b300.al import Batch, Instance, OPT_COLUMN
    from paper_2609_39443_b300.serve import BatchServer, PlainServer, Sim, poisson_arrivals
    local = int(os.environ.get("LOCAL_RANK", "0"))
    rank = int(os.environ.get("RANK", "0"))
    torch.cuda.set_device(local)
    wls = W.make_batched(1000 + rank, a.sims)
    sims = [Sim(w, a.sim_steps) for w in wls]
    budget = int(a.budget_gb * 2 ** 30)
    # the batched form on the same simulations (all of them in one batch, as
    # the server holds them resident)
    nb = len(sims)
    insts = [Instance(w, options={OPT_COLUMN: 0}) for w in wls[:nb]]
    batch = Batch(insts, use_graph=True)
    for _ in range(3):
        batch.run()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    for _ in range(10):
        batch.run()
    ev1.record()
    torch.cuda.synchronize()
    batched_rate = 10 * nb / (ev0.elapsed_time(ev1) / 1e3)
    batch.close()
    for i in insts:
        i.close()
    rows = []
    for rate in [float(x) for x in a.rates.split(",")]:
        arr = poisson_arrivals(sims, rate, seed=rate_seed(rate))
        n = min(len(arr), max(int(rate * a.window), 1))
        arr = arr[:n]
        used = sorted({s for _, s, _ in arr})
        remap = {s: i for i, s in enumerate(used)}
        sub = [Sim(sims[s].wl, sum(1 for _, x, _ in arr if x == s)) for s in used]
        arr_sub = [(t, remap[s], k) for t, s, k in arr]
        # two waves of up to half the slots in flight at once
        sb = BatchServer(sub, budget, n_slots=a.slots, max_wave=max(1, a.slots // 2), preadmit=True).run(arr_sub).summary()
        row = {"rate": rate, "requests": n, "simulations": len(sub), "batched": sb}
        if rate in (float(x) for x in a.plain_rates.split(",")):
            row["plain"] = PlainServer(sub, budget, preadmit=True).run(arr_sub).summary()
        rows.append(row)
    if rank == 0:
        best = max(rows, key=lambda r: r["batched"]["steps_per_s"])
        calm = min(rows, key=lambda r: r["rate"])
        line = {"metric": "coupling steps/s", "value": best["batched"]["steps_per_s"], "unit": "steps/s",
                "n_gpus": 1, "steps": best["requests"], "warmup": 0,
                "ms_per_step": 1e3 / best["batched"]["steps_per_s"], "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": f"serve_{a.sims}_sims_x_{a.sim_steps}_steps", "budget_bytes": budget,
                           "slots": a.slots, "window_s": a.window},
                "p50_ms": best["batched"]["p50_ms"], "p99_ms": best["batched"]["p99_ms"],
                "below_saturation": {"rate": calm["rate"], "p50_ms": calm["batched"]["p50_ms"],
                                     "p99_ms": calm["batched"]["p99_ms"]},
                "batched_form_instance_steps_per_s": batched_rate,
                "served_over_batched": best["batched"]["steps_per_s"] / batched_rate,
                "sweep": rows}
        print(json.dumps(line), flush=True)


def rate_seed(rate):
    return int(rate) % 100003


def _launch_ranks(n):
    """`--gpus N` without a torchrun environment: start N ranks on this node
    through torch.distributed.run (one process per GPU, rendezvous on
    127.0.0.1) with the same arguments; rank 0 prints the JSON line."""
    import socket
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", f"--nproc-per-node={n}",
           "--master-addr=127.0.0.1", f"--master-port={port}", os.path.abspath(__file__), *sys.argv[1:]]
    env = dict(os.environ, NCCL_DEBUG=os.environ.get("NCCL_DEBUG", "WARN"))
    return subprocess.call(cmd, env=env)


if __name__ == "__main__":
    args = _args()
    if args.gpus > 1 and "WORLD_SIZE" not in os.environ:
        sys.exit(_launch_ranks(args.gpus))
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batched":
        run_batched(args)
    elif args.workload == "serve":
        run_serve(args)
    elif args.split == "slab":
        run_slab(args)
    else:
        run_ours(args)
