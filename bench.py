"""Benchmark of the D3Q95 thermal BGK stream-collide on one GB300 (or N replicas).

Default workload: the precision-sweep setup, D3Q95, FP32 populations, 512 x 256 x 256
periodic box, omega 1.8, planar Riemann initial state (1, 1) | (0.5, 0.8) at
x = 256 with seeded density noise.  One bench "step" is one lattice time step over
the whole grid (one fused stream-collide launch).  The population arrays (2 x 12.75
GB) are two orders of magnitude larger than the 129 MB L2, so no L2 flush is needed
between steps and no step is served from the previous one's L2-resident output.

Prints one JSON line.  value = million lattice-cell updates per second (MLUPS)
over all ranks; roofline = algorithmic bytes (2 Q s per cell update) per launch
over the CUDA-event time of a launch, against the measured HBM copy bandwidth.
Secondary measurements in the same line: the 128 x 64 x 64 planar Riemann setup
(a 199 MB state, partly served from L2), the FP32 / FP16 / BF16 storage forms on
the 512 x 256 x 256 grid, the cost of the adjoint relative to the forward on the
128^3 adjoint workload, the 768 x 384 x 384 FP16 oblique problem (undivided, and as
two slabs with halo messages on this one GPU), an end-to-end run
through the public API from host buffers, and the FP64 oracle timed on the host
cores (cpu_baseline).

--impl reference times the FP64 CPU oracle (there is no reference program) on a
bounded sub-box sample of the same workload per step and prints the same JSON keys.

Multi-GPU (torchrun, N > 1): every rank runs an independent replica of the
workload (replicas only, weak scaling); the time is the maximum over ranks.  The
slab decomposition of the library is timed on one GPU (the `slabs` leg: two slabs
of the 768 x 384 x 384 FP16 workload with device-to-device halo messages).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "D3Q95 MLUPS and % of HBM roofline; FP16 vs FP32 form at stated error; adjoint cost"
BYTES = {"fp64": 8, "fp32": 4, "fp16": 2, "bf16": 2}
FALLBACK_HBM_GBS = 6800.0


def parse_args(argv=None):
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5000)
    p.add_argument("--warmup", type=int, default=20)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--storage", default="fp32", choices=["fp32", "fp16", "bf16", "fp64"])
    p.add_argument("--grid", default="512x256x256", help="NXxNYxNZ of the D3Q95 workload")
    p.add_argument("--setup", default="sweep", choices=["sweep", "riemann"],
                   help="sweep: omega 1.8, (1, 1) | (0.5, 0.8); riemann: omega 1.6, (1, 1) | (0.6, 0.75)")
    p.add_argument("--variant", default="auto", choices=["auto", "direct", "tma", "split", "pair"],
                   help="stream-collide kernel of the timed workload (auto: the library's choice)")
    p.add_argument("--no-extras", action="store_true", help="skip the forms / adjoint / cpu legs")
    p.add_argument("--leg", default=None, choices=["forms", "adjoint", "large", "moments", "d2q33",
                                                   "slabs",
                                                   "l2_assisted"],
                   help="run one secondary leg alone (for profiling) and print its JSON")
    return p.parse_args(argv)


# ------------------------------------------------------------------ distributed helpers
def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", str(rank)))
    return rank, world, local


def reduce_max_sum(elapsed_s, units, backend_device=None):
    """(max elapsed over ranks, sum of units over ranks); identity when not distributed."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return elapsed_s, units
    dev = backend_device or torch.device("cpu")
    t = torch.tensor([elapsed_s], dtype=torch.float64, device=dev)
    u = torch.tensor([float(units)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), u.item()


# ------------------------------------------------------------------ peaks, clocks, profiles
def hbm_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.proc = None
        self.gpu = gpu_index
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(gpu_index), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out = ""
        rows = [r.split(",") for r in out.strip().splitlines() if r.count(",") >= 8]
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx = float(r[2])
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if r[5 + k].strip().lower().startswith("active"):
                    reasons.add(nm)
        sm.sort()
        med = sm[len(sm) // 2] if sm else None
        return {"sm_mhz": med, "sm_max_mhz": mx, "samples": len(sm), "reasons": sorted(reasons)}


def kernel_source_hash():
    h = hashlib.sha256()
    for fn in ("kernels.cuh", "velset.cuh", "k_storage.inl", "common.h", "stream_collide_tma.cuh",
               "stream_collide_pair.cuh"):
        with open(os.path.join(ROOT, "paper_1303_4624_gb300", "csrc", fn), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def profile_record(workload_key, field):
    """A number recorded in a committed summary under profiles/, if that summary was
    taken on the current kernel source; else None.  A record is a 'workload_key:'
    line followed (before the next record) by a 'source_hash:' line that matches
    the current sources and a '<field>:' line."""
    d = os.path.join(ROOT, "profiles")
    if not os.path.isdir(d):
        return None
    src = kernel_source_hash()
    for fn in sorted(os.listdir(d)):
        if not fn.endswith(".md"):
            continue
        with open(os.path.join(d, fn)) as f:
            text = f.read()
        for block in re.split(r"(?=workload_key:)", text)[1:]:
            m_key = re.match(r"workload_key:\s*(\S+)", block)
            m_hash = re.search(r"source_hash:\s*([0-9a-f]+)", block)
            m_val = re.search(field + r":\s*([0-9.eE+-]+)", block)
            if m_key and m_hash and m_val and m_key.group(1) == workload_key \
                    and m_hash.group(1) == src:
                return float(m_val.group(1))
    return None


def profiled_traffic(workload_key):
    """DRAM bytes per launch of the stream-collide kernel from the committed ncu summary."""
    return profile_record(workload_key, "traffic_bytes_per_launch")


# ------------------------------------------------------------------ our arm
def time_steps(lbm, lat, steps, warmup, stream):
    import torch
    lbm.lbm_step(lat.ctx, warmup)
    torch.cuda.synchronize()
    start = torch.cuda.Event(enable_timing=True)
    stop = torch.cuda.Event(enable_timing=True)
    start.record(stream)
    lbm.lbm_step(lat.ctx, steps)
    stop.record(stream)
    torch.cuda.synchronize()
    return start.elapsed_time(stop) / 1e3


GRAPH_STEPS = 32     # steps per CUDA-graph replay in lbm_step (captured before timing)


VARIANTS = {"auto": 0, "direct": 1, "tma": 2, "split": 3, "pair": 4}


def make_lattice(lbm, wl, fields, storage=None, variant="auto"):
    lat = lbm.Lattice(wl.model, wl.dims, wl.omega, storage or wl.storage)
    if VARIANTS[variant]:
        lbm.lbm_set_variant(lat.ctx, VARIANTS[variant])
    lbm.lbm_set_graph_steps(lat.ctx, GRAPH_STEPS)
    lat.init(fields.rho, fields.U, fields.theta * lat.info["T0"])
    return lat


def workload_config(wl, Q):
    """The workload description both arms print (the reference arm times a sub-box
    sample of this workload per step and says so outside this object)."""
    state_mb = wl.cells * Q * BYTES[wl.storage] / 1e6
    return {"workload": wl.name, "model": wl.model,
            "storage": "%s (deviation h = f/w - 1)" % wl.storage,
            "grid": "%dx%dx%d" % wl.dims, "omega": wl.omega, "cells": wl.cells,
            "l2": ("inputs larger than L2 (2 x %.0f MB state vs 129 MB L2)" % state_mb
                   if 2 * state_mb > 129 else
                   "L2-resident (2 x %.0f MB state vs 129 MB L2): no roofline claim" % state_mb)}


def l2_assisted_leg(lbm, W, stream, steps=2000):
    """The 128 x 64 x 64 planar Riemann setup (omega 1.6), FP32: its 199 MB state is
    only 1.5x the L2, and consecutive steps walk the grid in opposite orders, so part
    of each step's input is still in L2 (DRAM traffic below the algorithmic bytes):
    reported beside the headline, not as an HBM roofline claim."""
    wl, fields = W.d3q95_riemann()
    lat = make_lattice(lbm, wl, fields)
    dt = time_steps(lbm, lat, steps, 20, stream)
    lat.close()
    peak, _ = hbm_peak()
    alg = wl.cells * 2 * 95 * 4
    gbs = alg / (dt / steps) / 1e9
    return {"workload": wl.name, "steps": steps, "mlups": round(wl.cells * steps / dt / 1e6, 1),
            "algorithmic_gbs": round(gbs, 1), "frac_of_measured_hbm": round(gbs / peak, 4),
            "dram_bytes_per_launch": profiled_traffic("d3q95_fp32_128x64x64"),
            "algorithmic_bytes_per_launch": alg,
            "note": "L2-assisted: DRAM traffic per launch below the algorithmic bytes"}


def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1 and not dist.is_initialized():
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import __graft_entry__
    if rank == 0 or world == 1:
        __graft_entry__.build()
    if world > 1:
        dist.barrier()
    from paper_1303_4624_gb300 import lbm
    from paper_1303_4624_gb300 import workloads as W

    stream = torch.cuda.current_stream()
    if args.leg:
        fn = {"forms": forms_leg, "adjoint": adjoint_leg, "large": large_leg, "slabs": slabs_leg,
              "moments": moments_leg, "d2q33": d2q33_leg, "l2_assisted": l2_assisted_leg}[args.leg]
        if rank == 0:
            print(json.dumps({"leg": args.leg, "result": fn(lbm, W, stream)}), flush=True)
        return
    nx, ny, nz = (int(v) for v in args.grid.lower().split("x"))
    make = W.d3q95_sweep if args.setup == "sweep" else W.d3q95_riemann
    wl, fields = make(nx, ny, nz, storage=args.storage)
    Q = lbm.lbm_model_info(wl.model)["Q"]
    lat = make_lattice(lbm, wl, fields, variant=args.variant)
    audit0 = lat.audit()
    launches0 = lbm.lbm_launch_count(lat.ctx)

    # ---- timed region: K fused stream-collide launches on the resident state
    lbm.lbm_step(lat.ctx, args.warmup)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks = ClockSampler(local)
    time.sleep(0.15)
    start = torch.cuda.Event(enable_timing=True)
    stop = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    start.record(stream)
    lbm.lbm_step(lat.ctx, args.steps)
    stop.record(stream)
    torch.cuda.synchronize()
    elapsed = start.elapsed_time(stop) / 1e3
    clk = clocks.stop()
    if world > 1:
        dist.barrier()
    gpu_launches = lbm.lbm_launch_count(lat.ctx) - launches0 - args.warmup
    t_max, units = reduce_max_sum(elapsed, wl.cells * args.steps,
                                  torch.device("cuda", local) if world > 1 else None)
    audit = lat.audit()
    value = units / t_max / 1e6
    per_launch = elapsed / args.steps
    alg_bytes = wl.cells * 2 * Q * BYTES[wl.storage]
    achieved = alg_bytes / per_launch / 1e9
    peak, peak_kind = hbm_peak()
    line = {
        "metric": METRIC,
        "value": round(value, 1),
        "unit": "MLUPS",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(t_max / args.steps * 1e3, 5),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64" if wl.storage == "fp64" else "f32",
        "data": "synthetic (seeded planar Riemann state, SplitMix64 noise)",
        "config": workload_config(wl, Q),
        "parallelism": "replicas" if world > 1 else "single GPU",
        "launch": "CUDA graphs of %d steps (programmatic dependent launch between steps), "
                  "remainder launched directly" % GRAPH_STEPS,
        "kernel_variant": args.variant,
        "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                     "frac": round(achieved / peak, 4), "peak_source": peak_kind + " (MEASURED_PEAKS.json hbm_gbs)"
                     if peak_kind == "measured" else "fallback 6.8 TB/s",
                     "traffic": profiled_traffic("d3q95_%s_%dx%dx%d" % ((wl.storage,) + wl.dims)),
                     "algorithmic_bytes_per_launch": alg_bytes,
                     "launch_ms": round(per_launch * 1e3, 5)},
        "clocks": clk,
        "gpu_launches": int(gpu_launches),
        "audit_after": {"nonfinite": audit["nonfinite"], "mass": audit["mass"],
                        "mass_drift_rel": audit["mass"] / audit0["mass"] - 1.0,
                        "energy_drift_rel": audit["energy"] / audit0["energy"] - 1.0,
                        "momentum_over_mass": float(max(abs(m) for m in audit["momentum"]))
                                              / audit["mass"],
                        "steps": args.warmup + args.steps},
    }
    if rank == 0 and not args.no_extras:
        line["moments"] = moments_leg(lbm, W, stream, lat=lat, wl=wl)
    # free the headline state before the other legs (the large adjoint leg sizes its
    # stored-state budget from the free device memory)
    lat.close()
    torch.cuda.empty_cache()
    if rank == 0 and not args.no_extras:
        line["l2_assisted"] = l2_assisted_leg(lbm, W, stream)
        line["e2e"] = e2e_leg(lbm, W, wl, fields, args.steps, stream,
                              reps=5 if args.steps <= 1000 else 3)
        line["forms"] = forms_leg(lbm, W, stream)
        line["d2q33"] = d2q33_leg(lbm, W, stream)
        line["adjoint"] = adjoint_leg(lbm, W, stream)
        del fields
        torch.cuda.empty_cache()
        line["large"] = large_leg(lbm, W, stream)
        line["slabs"] = slabs_leg(lbm, W, stream,
                                  undivided=line["large"].get("mlups") if line["large"] else None)
        line["cpu_baseline"] = cpu_baseline_leg()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


def e2e_leg(lbm, W, wl, fields, steps, stream, reps=5):
    """Whole job through the public API from pinned host buffers: lbm_init from
    host fields, `steps` steps, lbm_moments back to host; timed on the host clock."""
    import numpy as np
    import torch
    D = 3
    rho = torch.from_numpy(fields.rho).pin_memory().numpy()
    U = torch.from_numpy(np.ascontiguousarray(fields.U)).pin_memory().numpy()
    lat = lbm.Lattice(wl.model, wl.dims, wl.omega, wl.storage)
    lbm.lbm_set_graph_steps(lat.ctx, GRAPH_STEPS)
    T = torch.from_numpy(fields.theta * lat.info["T0"]).pin_memory().numpy()
    out_r = torch.empty(fields.rho.shape, dtype=torch.float64).pin_memory().numpy()
    out_U = torch.empty((D,) + fields.rho.shape, dtype=torch.float64).pin_memory().numpy()
    out_T = torch.empty(fields.rho.shape, dtype=torch.float64).pin_memory().numpy()
    lat.init(rho, U, T)   # warm-up of the path
    lbm.lbm_moments(lat.ctx, out_r, out_U, out_T)
    torch.cuda.synchronize()
    runs = []
    for _ in range(reps):
        t0 = time.perf_counter()
        lat.init(rho, U, T)
        lat.step(steps)
        lbm.lbm_moments(lat.ctx, out_r, out_U, out_T)
        runs.append(time.perf_counter() - t0)
    lat.close()
    dt = sorted(runs)[len(runs) // 2]
    h2d = rho.nbytes + U.nbytes + T.nbytes
    d2h = out_r.nbytes + out_U.nbytes + out_T.nbytes
    return {"value": round(wl.cells * steps / dt / 1e6, 1), "unit": "MLUPS",
            "h2d_bytes_per_step": round(h2d / steps, 1), "d2h_bytes_per_step": round(d2h / steps, 1),
            "runs_ms": [round(r * 1e3, 2) for r in runs],
            "note": "one lbm_init from host fields + %d steps + lbm_moments to host, host clock; "
                    "median of %d runs" % (steps, reps)}


def moments_leg(lbm, W, stream, lat=None, wl=None, calls=200):
    """lbm_moments into device buffers (rho, U, T in FP64) on the resident state:
    reads Q populations and writes D + 2 doubles per cell."""
    import torch
    own = lat is None
    if own:
        wl, fields = W.d3q95_riemann()
        lat = make_lattice(lbm, wl, fields)
        lat.step(10)
    D, Q = lat.info["D"], lat.info["Q"]
    shape = lat.shape
    rho = torch.empty(shape, dtype=torch.float64, device="cuda")
    U = torch.empty((D,) + shape, dtype=torch.float64, device="cuda")
    T = torch.empty(shape, dtype=torch.float64, device="cuda")
    for _ in range(5):
        lbm.lbm_moments(lat.ctx, rho, U, T)
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record(stream)
    for _ in range(calls):
        lbm.lbm_moments(lat.ctx, rho, U, T)
    b.record(stream)
    torch.cuda.synchronize()
    per_call = a.elapsed_time(b) / 1e3 / calls
    alg = wl.cells * (Q * BYTES[wl.storage] + (D + 2) * 8)
    peak, _ = hbm_peak()
    gbs = alg / per_call / 1e9
    if own:
        lat.close()
    return {"workload": wl.name, "storage": wl.storage, "calls": calls,
            "us_per_call": round(per_call * 1e6, 2),
            "mcells_per_s": round(wl.cells / per_call / 1e6, 1),
            "algorithmic_bytes_per_call": alg, "gbs": round(gbs, 1),
            "frac_of_measured_hbm": round(gbs / peak, 4)}


def d2q33_leg(lbm, W, stream, steps=300):
    """The 2D model on a grid larger than L2 (4096 x 2048, the D2Q33 workload's
    states, omega 1.5): FP32 and FP16 MLUPS and fraction of the HBM roofline."""
    import torch
    peak, _ = hbm_peak()
    out = {"grid": "4096x2048", "steps": steps}
    for st in ("fp32", "fp16"):
        fields = W.riemann_planar(2, 4096, 2048, 1, 2048, (1.0, 1.0), (0.5, 0.8), seed=1)
        lat = lbm.Lattice("D2Q33", (4096, 2048, 1), 1.5, st)
        lbm.lbm_set_graph_steps(lat.ctx, GRAPH_STEPS)
        lat.init(fields.rho, fields.U, fields.theta * lat.info["T0"])
        dt = time_steps(lbm, lat, steps, 5, stream)
        cells = 4096 * 2048
        gbs = cells * 2 * 33 * BYTES[st] / (dt / steps) / 1e9
        out[st] = {"mlups": round(cells * steps / dt / 1e6, 1), "gbs": round(gbs, 1),
                   "frac_of_measured_hbm": round(gbs / peak, 4)}
        lat.close()
        del fields
        torch.cuda.empty_cache()
    return out


def forms_leg(lbm, W, stream, steps=200):
    """FP32 vs FP16 / BF16 deviation storage on the 512 x 256 x 256 precision-sweep grid."""
    import torch
    out = {"grid": "512x256x256", "steps": steps, "omega": 1.8}
    for st in ("fp32", "fp16", "bf16"):
        wl, fields = W.d3q95_sweep(storage=st)
        lat = make_lattice(lbm, wl, fields)
        dt = time_steps(lbm, lat, steps, 5, stream)
        Q = lat.info["Q"]
        mlups = wl.cells * steps / dt / 1e6
        out[st] = {"mlups": round(mlups, 1),
                   "gbs": round(wl.cells * 2 * Q * BYTES[st] / (dt / steps) / 1e9, 1)}
        lat.close()
        del fields
        torch.cuda.empty_cache()
    out["fp16_over_fp32"] = round(out["fp16"]["mlups"] / out["fp32"]["mlups"], 3)
    out["bf16_over_fp32"] = round(out["bf16"]["mlups"] / out["fp32"]["mlups"], 3)
    err = {}
    for st in ("fp32", "fp16", "bf16"):
        r = profile_record("precision_d3q95_sweep_128x32x32_200", st + "_rho")
        t = profile_record("precision_d3q95_sweep_128x32x32_200", st + "_T")
        err[st] = None if r is None else {"rho": r, "T": t}
    out["error_vs_fp64_oracle"] = err
    out["error_source"] = ("max relative rho / T error after 200 steps on the 128x32x32 run of "
                           "the identical setup, from tests/test_gpu_precision.py, recorded in "
                           "profiles/precision_forms_d3q95_128x32x32.md for this kernel source "
                           "(null if the kernels changed since)")
    return out


def large_leg(lbm, W, stream, steps=300):
    """The 768 x 384 x 384 oblique Riemann workload, FP16 deviation storage: the
    forward, then the adjoint of the final-density MSE (target: the same setup's
    initial density from seed 2) with the memory-bounded reverse schedule, whose
    stored-state budget is what fits next to the two FP32 adjoint buffers."""
    import torch
    free, _ = torch.cuda.mem_get_info()
    if free < 60e9:
        return {"skipped": "needs 60 GB free device memory, %.0f GB free" % (free / 1e9)}
    wl, fields = W.d3q95_oblique()
    lat = make_lattice(lbm, wl, fields)
    dt = time_steps(lbm, lat, steps, 5, stream)
    a = lat.audit()
    key = "precision_d3q95_oblique_96x48x48_300"
    err = profile_record(key, "fp16_rho")
    out = {"workload": wl.name, "storage": "fp16", "steps": steps,
           "mlups": round(wl.cells * steps / dt / 1e6, 1),
           "gbs": round(wl.cells * 2 * 95 * 2 / (dt / steps) / 1e9, 1),
           "nonfinite_after": a["nonfinite"],
           "error_vs_fp64_oracle": None if err is None else
           {"rho": err, "T": profile_record(key, "fp16_T"),
            "source": "300 steps of the same setup (without density noise) on the 96x48x48 "
                      "stand-in grid, tests/test_gpu_precision.py, recorded in "
                      "profiles/precision_forms_d3q95_128x32x32.md for this kernel source"}}
    # adjoint of L = mean (rho_N - rho*)^2
    state_b = wl.cells * 95 * 2
    lam_b = 2 * wl.cells * 95 * 4
    free, _ = torch.cuda.mem_get_info()
    budget = int((free - lam_b - 12e9) // state_b)
    if budget < 2:
        out["adjoint"] = {"skipped": "%.0f GB free is too little" % (free / 1e9)}
    else:
        max_states = min(budget, 12)
        target = torch.from_numpy(W.d3q95_oblique(seed=2)[1].rho).to("cuda")
        lat.init(fields.rho, fields.U, fields.theta * lat.info["T0"])
        del fields
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        ev[0].record(stream)
        lbm.lbm_record_bounded(lat.ctx, steps, max_states)
        ev[1].record(stream)
        rhoN = torch.empty_like(target)
        lbm.lbm_moments(lat.ctx, rhoN, None, None)
        g = 2.0 * (rhoN - target) / rhoN.numel()
        loss = float(((rhoN - target) ** 2).mean())
        d_rho = torch.empty_like(target)
        torch.cuda.synchronize()
        ev[2].record(stream)
        d_om = lbm.lbm_backward(lat.ctx, g, d_rho, None, None)
        ev[3].record(stream)
        torch.cuda.synchronize()
        fw = ev[0].elapsed_time(ev[1]) / 1e3
        bw = ev[2].elapsed_time(ev[3]) / 1e3
        out["adjoint"] = {"loss": loss, "dL_domega": d_om,
                          "dL_drho0_rms": float(d_rho.pow(2).mean().sqrt()),
                          "max_states": max_states, "forward_s": round(fw, 3),
                          "backward_s": round(bw, 3), "backward_over_forward": round(bw / fw, 2),
                          "schedule": "%d stored FP16 states (S_0 included), placed to "
                                      "minimise the recomputed steps" % max_states}
        del target, rhoN, g, d_rho
    lbm.lbm_release_record(lat.ctx)
    lat.close()
    torch.cuda.empty_cache()
    return out


def slabs_leg(lbm, W, stream, undivided=None, nslabs=2, steps=20, warmup=3):
    """The 768 x 384 x 384 FP16 oblique workload decomposed into z-slabs on this one
    device (paper_1303_4624_gb300/slabs.py): every step advances each slab (interior
    and ghost planes) and then packs and unpacks the halo messages of both faces of
    every slab with device-to-device buffers.  MLUPS counts the grid's cells; against
    the undivided grid's rate this is the cost of the ghost planes and the halo
    kernels (the transport between GPUs is not part of it: one device)."""
    import numpy as np
    import torch
    from paper_1303_4624_gb300 import slabs as SL
    free, _ = torch.cuda.mem_get_info()
    if free < 60e9:
        return {"skipped": "needs 60 GB free device memory, %.0f GB free" % (free / 1e9)}
    wl, fields = W.d3q95_oblique()
    nz = wl.dims[2]
    splits = [nz // nslabs + (1 if k < nz % nslabs else 0) for k in range(nslabs)]
    sg = SL.SlabGrid(wl.model, wl.dims, wl.omega, wl.storage, splits)
    try:
        T0 = lbm.lbm_model_info(wl.model)["T0"]
        sg.init(fields.rho, fields.U, fields.theta * T0)
        del fields
        sg.step(warmup)
        torch.cuda.synchronize()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        ev[0].record(stream)
        sg.step(steps)
        ev[1].record(stream)
        torch.cuda.synchronize()
        dt = ev[0].elapsed_time(ev[1]) / 1e3
        h = lbm.lbm_halo_info(sg.ctxs[0])
        ml = wl.cells * steps / dt / 1e6
        out = {"workload": wl.name, "storage": wl.storage, "slabs": nslabs, "splits": splits,
               "ghost_planes_per_side": h["ghost"], "face_bytes": h["face_bytes"],
               "steps": steps, "mlups": round(ml, 1),
               "of_undivided": None if not undivided else round(ml / undivided, 4),
               "note": "all slabs on one GPU, halos by device-to-device buffers; MLUPS over "
                       "the grid's cells"}
    finally:
        sg.close()
        torch.cuda.empty_cache()
    return out


def adjoint_leg(lbm, W, stream, n=128, steps=500, k=22):
    """Cost of lbm_backward (replay + adjoint) over lbm_record (checkpointed forward)."""
    import numpy as np
    import torch
    wl, fields = W.d3q95_adjoint(n)
    lat = lbm.Lattice(wl.model, wl.dims, wl.omega, "fp32")
    lat.init(fields.rho, fields.U, fields.theta * lat.info["T0"])
    g = torch.zeros(fields.rho.shape, dtype=torch.float64, device="cuda")
    g += 1.0 / fields.rho.size
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    lbm.lbm_record(lat.ctx, 20, 5)       # warm-up (allocations)
    lbm.lbm_backward(lat.ctx, g)
    torch.cuda.synchronize()
    ev[0].record(stream)
    lbm.lbm_record(lat.ctx, steps, k)
    ev[1].record(stream)
    lbm.lbm_backward(lat.ctx, g)
    ev[2].record(stream)
    torch.cuda.synchronize()
    fwd = ev[0].elapsed_time(ev[1]) / 1e3
    bwd = ev[1].elapsed_time(ev[2]) / 1e3
    lbm.lbm_release_record(lat.ctx)
    lat.close()
    torch.cuda.empty_cache()
    # the backward replays every segment but the last (kept by the record) once
    replay = steps - (steps + k - 1) // k - (min(k, steps) - 1)
    t_step = fwd / steps
    adj_per_step = (bwd - replay * t_step) / steps
    return {"workload": wl.name, "steps": steps, "ckpt_every": k, "forward_s": round(fwd, 4),
            "backward_s": round(bwd, 4), "backward_over_forward": round(bwd / fwd, 3),
            "replayed_steps": replay,
            "adjoint_step_over_forward_step": round(adj_per_step / t_step, 3),
            "forward_mlups": round(wl.cells * steps / fwd / 1e6, 1)}


CPU_SAMPLE = """
import json, os, sys, time
sys.path.insert(0, %r)
from oracle import lbm
from oracle.model import get_model
from paper_1303_4624_gb300 import workloads as W
mdl = get_model("D3Q95")
wl, f = W.d3q95_sweep(nx=%d, ny=%d, nz=%d)
S = lbm.init_populations(mdl, f.rho, f.U, f.theta * mdl.T0)
for _ in range(max(1, %d)):
    S = lbm.step(mdl, S, wl.omega)
n = 0
t0 = time.perf_counter()
while True:
    S = lbm.step(mdl, S, wl.omega)
    n += 1
    dt = time.perf_counter() - t0
    if n >= %d or dt > %f:
        break
print(json.dumps({"steps": n, "seconds": dt, "cells": wl.cells}))
"""

# The oracle sample: the headline workload's setup (omega 1.8, diaphragm at x = 256 of a
# 512-cell tube, the same seeded noise recipe) on a 512 x ny x nz sub-box; the
# x extent is kept so that the sample holds both Riemann fans of the periodic tube.
SAMPLE_NX = 512


def run_oracle_sample(ny, nz, max_steps, budget_s, warmup=1, threads=None):
    env = dict(os.environ)
    cores = threads or os.cpu_count() or 1
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[k] = str(cores)
    code = CPU_SAMPLE % (ROOT, SAMPLE_NX, ny, nz, warmup, max_steps, budget_s)
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env,
                       timeout=budget_s * 4 + 120)
    if r.returncode != 0:
        raise RuntimeError(r.stderr[-2000:])
    res = json.loads(r.stdout.strip().splitlines()[-1])
    res["cores"] = cores
    return res


def cpu_baseline_leg():
    res = run_oracle_sample(16, 8, 10 ** 9, 15.0)
    one = run_oracle_sample(16, 8, 10 ** 9, 8.0, threads=1)
    return {"value": round(res["cells"] * res["steps"] / res["seconds"] / 1e6, 4), "unit": "MLUPS",
            "cores": res["cores"], "kind": "oracle",
            "sample": "FP64 numpy oracle, the same D3Q95 setup on a %dx16x8 sub-box, "
                      "%d steps in %.1f s, BLAS threads = cores"
                      % (SAMPLE_NX, res["steps"], res["seconds"]),
            "single_thread": {"value": round(one["cells"] * one["steps"] / one["seconds"] / 1e6, 4),
                              "unit": "MLUPS", "cores": 1,
                              "sample": "same sub-box, %d steps in %.1f s, one BLAS thread"
                                        % (one["steps"], one["seconds"])}}


# ------------------------------------------------------------------ reference arm (the oracle)
def run_reference(args):
    """The FP64 oracle on the host cores: every step is one oracle step of the
    headline workload's setup on a 512 x ny x nz sub-box, sized so that the warm-up
    and timed steps take about two minutes; MLUPS counts the sub-box's cells."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    total = args.steps + args.warmup
    budget = 120.0
    cells = max(SAMPLE_NX, min(SAMPLE_NX * 32 * 32, int(budget / (total * 1.2e-5))))
    ny = nz = max(1, int(math.sqrt(cells / SAMPLE_NX)))
    res = run_oracle_sample(ny, nz, args.steps, budget * 1.5, warmup=args.warmup)
    value = res["cells"] * res["steps"] / res["seconds"] / 1e6
    sample = ("FP64 numpy oracle: each step is one step of the same setup on a %dx%dx%d "
              "sub-box (%d cells), %d timed steps" % (SAMPLE_NX, ny, nz, res["cells"], res["steps"]))
    line = {
        "impl": "reference",
        "metric": METRIC,
        "value": round(value, 4),
        "unit": "MLUPS",
        "n_gpus": world,
        "steps": res["steps"],
        "warmup": args.warmup,
        "ms_per_step": round(res["seconds"] / res["steps"] * 1e3, 3),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64",
        "data": "synthetic (seeded planar Riemann state, SplitMix64 noise)",
        "config": reference_config(args),
        "sample_grid": "%dx%dx%d" % (SAMPLE_NX, ny, nz),
        "cpu_baseline": {"value": round(value, 4), "unit": "MLUPS", "cores": res["cores"],
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": round(value, 4), "unit": "MLUPS", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def reference_config(args):
    """Our arm's config object for the same arguments (no GPU needed to build it)."""
    from paper_1303_4624_gb300 import workloads as W
    nx, ny, nz = (int(v) for v in args.grid.lower().split("x"))
    name = ("d3q95_sweep_%dx%dx%d" if args.setup == "sweep" else "d3q95_riemann_%dx%dx%d") % (nx, ny, nz)
    omega = 1.8 if args.setup == "sweep" else 1.6
    wl = W.Workload(name, "D3Q95", args.storage, (nx, ny, nz), 0, omega)
    return workload_config(wl, 95)


def main(argv=None):
    args = parse_args(argv)
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
