#!/usr/bin/env python
"""Throughput of the DD-CCLB time step on GB300 (MLUPS and HBM roofline).

Default workload: the 4096 x 4096, N = 4 porous-imbibition problem
(2000 seeded solid circles embedded by psi, contact angles per circle,
seeded droplets) in FP32 with g_0 stored as g_0 - rho0; one step is one
full DD-CCLB update of every node (order parameters, chemical potentials,
mobility flux, force, velocity/pressure, both collisions, streaming and the
lagged fields).  The FP64 step of the same workload is timed beside it.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  Under torchrun every rank runs the same
workload on its own GPU (replicas: the method needs no data exchange
between independent problems), ``value`` sums the ranks' node updates over
the slowest rank's time.
"""
from __future__ import annotations

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

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "MLUPS & % HBM roofline: FP32 vs FP64 DD-LB step at stated error; adjoint/fwd"
UNIT = "MLUPS"


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--err-steps", type=int, default=20000,
                    help="steps of the FP32-vs-FP64 error statement (emulsion 1024^2; its "
                         "configuration asks for 2 x 10^4)")
    ap.add_argument("--adj-steps", type=int, default=2000,
                    help="steps T of the adjoint cost measurement (wavy wall; its configuration "
                         "asks for T = 2000 with a checkpoint every 100 steps)")
    ap.add_argument("--precision", choices=["fp32", "fp64"], default="fp32",
                    help="precision of the main line (the FP64 step is timed beside the FP32 "
                         "one either way)")
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--size", type=int, default=4096, help="grid edge of the workload")
    ap.add_argument("--fp64-steps", type=int, default=10)
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the FP64 leg, e2e leg and CPU baseline")
    ap.add_argument("--path", choices=["tile", "sweep"], default="tile",
                    help="step kernels: the TMA-staged tile kernels (default) or the row sweep")
    ap.add_argument("--workload", choices=["imbibition", "sphere3d"], default="imbibition",
                    help="imbibition: the 2D headline workload; sphere3d: the Sec. 4.4 "
                         "compound drop on a sphere, 3D (D3Q7 / D3Q15), --size^3 nodes")
    return ap.parse_args()


# ----------------------------------------------------------------------------
# helpers
# ----------------------------------------------------------------------------

def step_floats_per_node(N, theta_field):
    """Algorithmic floats a step must move per node: populations read and
    written (18 N), psi (1), the contact-angle field (N-1 if per node) and
    the lagged fields read and written (a, psi C_i u, T, psi m.u: 2N+3)."""
    return 18 * N + 1 + ((N - 1) if theta_field else 0) + 2 * (2 * N + 3)


def collide_floats_per_node(N, theta_field, fused=True):
    """The tile collide-stream kernel's own algorithmic floats.  The fused
    kernel (order parameters formed from the staged phase populations) and
    the row sweep move exactly the step's floats; the unfused tile kernel
    also reads the order parameters (N-1)."""
    return step_floats_per_node(N, theta_field) + (0 if fused else N - 1)


def order_param_floats_per_node(N):
    """Order-parameter kernel: reads the phase populations and psi, writes C."""
    return 9 * (N - 1) + 1 + (N - 1)


def step_bytes_per_node_3d(N, theta_field, es):
    """Algorithmic bytes of one 3D step per node at element size es: the
    D3Q7 populations (7 (N-1)) and the D3Q15 populations (15) read and
    written, psi, the angle field (N-1 if per node) and the 3N + 7 lagged
    fields read and written."""
    return es * (2 * (7 * (N - 1) + 15) + 1 + ((N - 1) if theta_field else 0) + 2 * (3 * N + 7))


def kernel_bytes_per_node_3d(N, theta_field, es):
    """Each 3D kernel's own algorithmic bytes per node: the volume-fraction
    pass (phase populations and psi in, C out), the chemical potentials (C,
    psi and angles in, mu out) and the node update (populations and lagged
    fields in and out, psi, C and mu in); the fused step moves the whole
    step's bytes (C and mu stay on chip)."""
    nt = (N - 1) if theta_field else 0
    return {"order_param": es * (7 * (N - 1) + 1 + (N - 1)),
            "chem_pot": es * ((N - 1) + 1 + nt + N),
            "update": es * (2 * (7 * (N - 1) + 15) + 2 * (3 * N + 7) + 1 + (N - 1) + N),
            "fused_step": step_bytes_per_node_3d(N, theta_field, es)}


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def kernel_source_hash(files=("ddcc_kernels.cu", "ddcc_sweep.cu", "ddcc_device.cuh", "ddcc_internal.h",
                              "ddcc_tma.cuh")):
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, "paper_2311_10314_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    from paper_2311_10314_gb300 import build as B
    # the flags without the include paths, which differ from machine to machine
    h.update(" ".join(f for f in B.FLAGS if not os.path.isabs(f)).encode())
    return h.hexdigest()[:16]


def ncu_record(kind, key, path=os.path.join(ROOT, "profiles", "ncu_traffic.json")):
    """A per-node figure of a kernel from a committed ncu summary, or None
    when the summary is missing or the kernel source changed since."""
    if not os.path.exists(path):
        return None
    with open(path) as fh:
        d = json.load(fh)
    entry = d.get(kind)
    files = ("ddcc3d.cu",) if "_3d" in kind else None
    if not entry or entry.get("source_hash") != (kernel_source_hash(files) if files else kernel_source_hash()):
        return None
    return float(entry[key])


def ncu_traffic_per_node(kind):
    """DRAM bytes per node of a kernel (ncu, one launch)."""
    return ncu_record(kind, "dram_bytes_per_node")


def ncu_fp64_flops_per_node():
    """FP64 flops the FP64 collide-stream kernel executes per node (ncu:
    2 x DFMA + DADD + DMUL thread instructions of one launch / nodes)."""
    return ncu_record("collide_stream_fp64", "fp64_flops_per_node",
                      os.path.join(ROOT, "profiles", "ncu_fp64.json"))


class ClockSampler:
    """nvidia-smi clock / throttle samples while the timed region runs."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + q,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as fh:
            for line in fh:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None

        def num(x):
            try:
                return float(x)
            except ValueError:
                return float("nan")
        sm = [num(r[1]) for r in rows if not math.isnan(num(r[1]))]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for k, name in enumerate(names):
                if r[5 + k].lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": num(rows[0][2]), "reasons": sorted(reasons),
                "samples": len(rows),
                "power_w_max": max(num(r[3]) for r in rows)}


def dist_setup():
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
    elif torch.cuda.is_available():
        torch.cuda.set_device(0)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def allreduce_max(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ----------------------------------------------------------------------------
# the oracle on the host cores (CPU baseline and the reference arm)
# ----------------------------------------------------------------------------

def oracle_sample(pb, crop=256, steps=2, threads=None):
    """Time the FP64 CPU oracle on a crop x crop window of the workload's
    own fields (psi, C0, contact angles), periodic, on `threads` host threads
    (all cores by default); returns (MLUPS, cores, description, seconds per
    step)."""
    import numpy as np
    import torch
    from oracle import Oracle
    torch.set_num_threads(threads or os.cpu_count() or 1)
    c = min(crop, pb.params["nx"], pb.params["ny"])
    prm = dict(pb.params)
    prm["nx"], prm["ny"] = c, c
    cf = None if pb.cos_theta_field is None else np.ascontiguousarray(pb.cos_theta_field[:, :c, :c])
    o = Oracle(prm, np.ascontiguousarray(pb.psi[:c, :c]), np.ascontiguousarray(pb.C0[:, :c, :c]),
               pb.cos_theta, cf)
    o.step(1)
    t0 = time.perf_counter()
    o.step(steps)
    dt = (time.perf_counter() - t0) / steps
    mlups = c * c / dt / 1e6
    desc = ("FP64 torch-CPU oracle, %dx%d window of the %s fields, %d timed steps after 1 "
            "warm-up step" % (c, c, pb.name, steps))
    return mlups, torch.get_num_threads(), desc, dt



def oracle_sample_3d(pb, crop=32, steps=2, threads=None):
    """Time the FP64 CPU 3D oracle on a crop^3 window of the workload's own
    fields, periodic; returns (MLUPS, cores, description, seconds per step)."""
    import numpy as np
    import torch
    from oracle.ddcc_oracle3d import Oracle3D
    torch.set_num_threads(threads or os.cpu_count() or 1)
    c = min(crop, pb.params["nx"])
    prm = dict(pb.params)
    prm["nx"] = prm["ny"] = prm["nz"] = c
    L = pb.params["nx"]
    o0 = L // 2 - c // 2
    win = (slice(o0, o0 + c),) * 3
    cf = None if pb.cos_theta_field is None else np.ascontiguousarray(pb.cos_theta_field[(slice(None),) + win])
    o = Oracle3D(prm, np.ascontiguousarray(pb.psi[win]), np.ascontiguousarray(pb.C0[(slice(None),) + win]),
                 pb.cos_theta, cf)
    o.step(1)
    t0 = time.perf_counter()
    o.step(steps)
    dt = (time.perf_counter() - t0) / steps
    desc = ("FP64 torch-CPU 3D oracle, %d^3 window at the centre of the %s fields, %d timed steps "
            "after 1 warm-up step" % (c, pb.name, steps))
    return c ** 3 / dt / 1e6, torch.get_num_threads(), desc, dt


# ----------------------------------------------------------------------------
# arms
# ----------------------------------------------------------------------------

def run_reference(args, world, rank):
    import workloads as W
    if rank != 0:
        return
    if getattr(args, "workload", "imbibition") == "sphere3d":
        size = args.size if args.size != 4096 else 256
        pb = W.config7_sphere(L=size)
        k = max(1, min(args.steps, 3))
        mlups_s, cores, desc, dt = oracle_sample_3d(pb, crop=32, steps=k)
        line = {
            "impl": "reference", "metric": METRIC, "value": round(mlups_s, 4), "unit": UNIT,
            "n_gpus": args.gpus, "steps": k, "warmup": 1, "ms_per_step": round(dt * 1e3, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": pb.name, "nodes_per_step": 32 ** 3, "sample": "32^3 window"},
            "cpu_baseline": {"value": round(mlups_s, 4), "unit": UNIT, "cores": cores,
                             "kind": "oracle", "sample": desc},
            "e2e": {"value": round(mlups_s, 4), "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0},
        }
        print(json.dumps(line), flush=True)
        return
    pb = W.config4_imbibition(nx=args.size, ny=args.size)
    # each timed step is one oracle step on the bounded window
    crop = 256
    mlups_s, cores, desc, dt = oracle_sample(pb, crop=crop, steps=max(1, min(args.steps, 3)))
    line = {
        "impl": "reference", "metric": METRIC, "value": round(mlups_s, 4), "unit": UNIT,
        "n_gpus": args.gpus, "steps": max(1, min(args.steps, 3)), "warmup": 1,
        "ms_per_step": round(dt * 1e3, 3), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": pb.name, "nodes_per_step": crop * crop,
                   "sample": "%dx%d window" % (crop, crop)},
        "cpu_baseline": {"value": round(mlups_s, 4), "unit": UNIT, "cores": cores,
                         "kind": "oracle", "sample": desc},
        "e2e": {"value": round(mlups_s, 4), "unit": UNIT, "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def timed_steps(D, sim, steps, warmup, world, profile=True):
    import torch
    from paper_2311_10314_gb300 import _lib
    stream = sim.stream
    sim.step(warmup)
    torch.cuda.synchronize()
    barrier(world)
    torch.cuda.synchronize()
    if profile:
        _lib.ddcc_profile(sim.h, True)
        _lib.ddcc_kernel_times(sim.h)            # clear
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    sim.step(steps)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    kt = _lib.ddcc_kernel_times(sim.h) if profile else {}
    if profile:
        _lib.ddcc_profile(sim.h, False)
    return ms, kt


def fp32_error_statement(D, W, steps):
    """FP32 against FP64 on the 1024^2 three-phase emulsion (body force,
    porous matrix): max |dC_i| on psi >= 0.5 and max |du| at a few steps, and
    each precision's relative drift of every phase's FP64-reduced mass, scaled
    to 10^4 steps."""
    import numpy as np
    import torch
    pb = W.config3_emulsion()
    marks = sorted({max(1, steps // 8), max(1, steps // 4), max(1, steps // 2), steps})
    sims = [D.Sim(pb.params, pb.psi, pb.C0, pb.cos_theta, pb.cos_theta_field, precision=pr)
            for pr in (D.DDCC_FP32, D.DDCC_FP64)]
    m0 = [s_.mass() for s_ in sims]
    bulk = pb.psi >= 0.5
    curve = []
    t = 0
    for mk in marks:
        for s_ in sims:
            s_.step(mk - t)
        t = mk
        f32, f64 = sims[0].fields(), sims[1].fields()
        curve.append({"step": mk,
                      "max_dC_bulk": float(np.abs(f32["C"] - f64["C"])[:, bulk].max()),
                      "max_du": float(max(np.abs(f32["ux"] - f64["ux"]).max(),
                                          np.abs(f32["uy"] - f64["uy"]).max()))})
    drift = []
    for s_, m in zip(sims, m0):
        d = (np.abs(s_.mass() - m) / np.abs(m)).max()
        drift.append(float(d) * 1e4 / steps)
    for s_ in sims:
        s_.close()
    torch.cuda.empty_cache()
    return {"workload": pb.name, "steps": steps, "curve": curve,
            "mass_drift_per_1e4_steps": {"fp32": drift[0], "fp64": drift[1]},
            "targets": {"max_dC_bulk": 1e-4, "fp32_mass_drift_per_1e4_steps": 1e-6}}


def fp32_error_statement_3d(D, W, size, steps):
    """FP32 against FP64 on the 3D sphere workload at size^3 (N = 3): max
    |dC_i| on psi >= 0.5 and max |du| at a few steps, and each precision's
    relative drift of every phase's FP64-reduced mass, scaled to 10^4 steps."""
    import numpy as np
    import torch
    pb = W.config7_sphere(L=size)
    marks = sorted({max(1, steps // 4), max(1, steps // 2), steps})
    sims = [D.Sim3D(pb.params, pb.psi, pb.C0, pb.cos_theta, precision=pr)
            for pr in (D.DDCC_FP32, D.DDCC_FP64)]
    m0 = [s_.mass() for s_ in sims]
    bulk = pb.psi >= 0.5
    curve = []
    t = 0
    for mk in marks:
        for s_ in sims:
            s_.step(mk - t)
        t = mk
        f32, f64 = sims[0].fields(), sims[1].fields()
        curve.append({"step": mk,
                      "max_dC_bulk": float(np.abs(f32["C"] - f64["C"])[:, bulk].max()),
                      "max_du": float(max(np.abs(f32[k] - f64[k]).max() for k in ("ux", "uy", "uz")))})
    drift = []
    for s_, m in zip(sims, m0):
        drift.append(float((np.abs(s_.mass() - m) / np.abs(m)).max()) * 1e4 / steps)
    for s_ in sims:
        s_.close()
    torch.cuda.empty_cache()
    return {"workload": pb.name, "steps": steps, "curve": curve,
            "mass_drift_per_1e4_steps": {"fp32": drift[0], "fp64": drift[1]},
            "targets": {"max_dC_bulk": 1e-4, "fp32_mass_drift_per_1e4_steps": 1e-6}}


def adjoint_cost(D, W, steps):
    """Reverse sweep (checkpoint every 100 steps, segment recompute included,
    pipelined where two sets of segment buffers fit) against forward steps
    on the wavy-wall drop, CUDA events on the stream."""
    import torch
    from paper_2311_10314_gb300 import adjoint as A
    out = []
    for n, prec in ((256, D.DDCC_FP32), (256, D.DDCC_FP64), (1024, D.DDCC_FP32), (1024, D.DDCC_FP64)):
        pb = W.config5_wavy_wall(nx=n, ny=n)
        e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        sim = D.Sim(pb.params, pb.psi, pb.C0, cos_theta_field=pb.cos_theta_field, precision=prec)
        sim.step(20)
        e[0].record(sim.stream)
        sim.step(steps)
        e[1].record(sim.stream)
        torch.cuda.synchronize()
        fwd = e[0].elapsed_time(e[1]) / steps
        sim.close()
        run = A.CheckpointedRun(pb.params, pb.psi, pb.C0, pb.cos_theta_field, steps, ckpt=100, precision=prec)
        stream = torch.cuda.current_stream()
        e[2].record(stream)
        run.reverse()
        e[3].record(stream)
        torch.cuda.synchronize()
        rev = e[2].elapsed_time(e[3]) / steps
        run.close()
        torch.cuda.empty_cache()
        out.append({"grid": "%dx%d" % (n, n), "dtype": "f32" if prec == D.DDCC_FP32 else "f64",
                    "forward_ms_per_step": round(fwd, 4), "reverse_ms_per_step": round(rev, 4),
                    "reverse_over_forward": round(rev / fwd, 3)})
    # the 4096^2 four-phase imbibition, whose 100-state segments (3.2 GB a
    # state) do not fit: two-level checkpointing, one more forward step per
    # reversed step
    pb = W.config4_imbibition()
    T4 = 200
    e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    sim = D.Sim(pb.params, pb.psi, pb.C0, cos_theta_field=pb.cos_theta_field, precision=D.DDCC_FP32)
    sim.step(5)
    e[0].record(sim.stream)
    sim.step(T4)
    e[1].record(sim.stream)
    torch.cuda.synchronize()
    fwd = e[0].elapsed_time(e[1]) / T4
    sim.close()
    run = A.CheckpointedRun(pb.params, pb.psi, pb.C0, pb.cos_theta_field, T4, ckpt=100,
                            precision=D.DDCC_FP32, sub=10)
    stream = torch.cuda.current_stream()
    e[2].record(stream)
    run.reverse()
    e[3].record(stream)
    torch.cuda.synchronize()
    rev = e[2].elapsed_time(e[3]) / T4
    run.close()
    torch.cuda.empty_cache()
    out.append({"grid": "4096x4096", "dtype": "f32", "workload": "imbibition_N4", "T": T4,
                "checkpointing": "two-level: every 100 steps, then every 10 within a segment",
                "forward_ms_per_step": round(fwd, 4), "reverse_ms_per_step": round(rev, 4),
                "reverse_over_forward": round(rev / fwd, 3)})
    return {"workload": "wavy_wall_N2 (drop on a sinusoidal wall, per-node theta field)",
            "objective": "phase-1 x-centroid after T steps; d/dcos(theta)(x), d/dpsi(x)",
            "T": steps, "checkpoint_every": 100,
            "reverse": "segment recompute (buffer to buffer, on a second stream beside the reverse of the "
                       "later segment where two buffer sets fit) + adjoint kernels", "runs": out}


def fp64_roofline_3d(kt64, ms_step, nodes):
    """The 3D FP64 step (three kernels) against the FP64 pipe: FP64 flops per
    node of each kernel (ncu counters of one launch each, committed under
    profiles/) times the nodes, over the CUDA-event times, against the FP64
    FMA rate measured on this GPU."""
    import torch
    from paper_2311_10314_gb300 import _lib
    path = os.path.join(ROOT, "profiles", "ncu_fp64.json")
    fpn = {kk: ncu_record(kk + "_3d_fp64", "fp64_flops_per_node", path) for kk in ("order_param", "chem_pot", "update")}
    sink = torch.zeros(8 * torch.cuda.get_device_properties(0).multi_processor_count,
                       dtype=torch.float64, device="cuda")
    peak = _lib.ddcc_measure_fp64_peak(torch.cuda.current_stream().cuda_stream, sink.data_ptr())
    out = {"kernels": "order_param + chem_pot + update", "bound": "fp64", "unit": "TFLOP/s",
           "peak": round(peak, 3), "peak_kind": "measured (ddcc_measure_fp64_peak)",
           "flops_per_node": None, "achieved": None, "frac": None, "per_kernel": {}}
    for kk, f in fpn.items():
        ms, n = kt64.get(kk, (0.0, 0))
        if f is None or not n:
            continue
        ach = f * nodes / (ms / n * 1e-3) / 1e12
        out["per_kernel"][kk] = {"flops_per_node": f, "achieved": round(ach, 3), "frac": round(ach / peak, 4)}
    if all(v is not None for v in fpn.values()):
        tot = sum(fpn.values())
        out["flops_per_node"] = round(tot, 1)
        out["achieved"] = round(tot * nodes / (ms_step * 1e-3) / 1e12, 3)
        out["frac"] = round(out["achieved"] / peak, 4)
    return out


def three_d_step(D, W, size, steps, warmup, fp64_steps, world, peak, peak_kind, sampler=None, fp32=True):
    """FP32 (and FP64) steps of the Sec. 4.4 sphere workload at size^3, N = 3:
    MLUPS, the per-kernel record and the roofline of the dominant kernel
    (the FP64 step against the FP64 pipe)."""
    import torch
    from paper_2311_10314_gb300 import _lib
    pb = W.config7_sphere(L=size)
    N = pb.params["nphase"]
    nodes = size ** 3
    tf = pb.cos_theta_field is not None
    out = {"workload": pb.name, "nodes": nodes, "nphase": N}
    for prec, k, w in ((D.DDCC_FP32, steps if fp32 else 0, warmup), (D.DDCC_FP64, fp64_steps, 2)):
        if k <= 0:
            continue
        sim = D.Sim3D(pb.params, pb.psi, pb.C0, pb.cos_theta, pb.cos_theta_field, precision=prec)
        sim.step(w)
        torch.cuda.synchronize()
        barrier(world)
        torch.cuda.synchronize()
        _lib.ddcc3d_profile(sim.h, True)
        _lib.ddcc3d_kernel_times(sim.h)
        if sampler is not None and prec == D.DDCC_FP32:
            sampler.start()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(sim.stream)
        sim.step(k)
        e1.record(sim.stream)
        torch.cuda.synchronize()
        barrier(world)
        torch.cuda.synchronize()
        if sampler is not None and prec == D.DDCC_FP32:
            out["clocks"] = sampler.stop()
        ms = allreduce_max(e0.elapsed_time(e1), world)
        kt = _lib.ddcc3d_kernel_times(sim.h)
        finite = bool(torch.isfinite(torch.tensor(sim.mass())).all())
        sim.close()
        del sim
        torch.cuda.empty_cache()
        es = 4 if prec == D.DDCC_FP32 else 8
        step_bytes = step_bytes_per_node_3d(N, tf, es) * nodes
        kb = {kk: v * nodes for kk, v in kernel_bytes_per_node_3d(N, tf, es).items()}
        total = sum(v[0] for v in kt.values())
        rec = {"value": round(world * nodes * k / (ms * 1e-3) / 1e6, 2), "unit": UNIT,
               "steps": k, "warmup": w, "ms_per_step": round(ms / k, 4), "mass_finite": finite,
               "gpu_launches": sum(v[1] for v in kt.values()),
               "kernels": {kk: {"launches": v[1], "avg_ms": round(v[0] / v[1], 4),
                                "share": round(v[0] / total, 4),
                                "algorithmic_GBps": round(kb[kk] / (v[0] / v[1] * 1e-3) / 1e9, 1)}
                           for kk, v in kt.items() if v[1]},
               "whole_step": {"algorithmic_bytes": step_bytes,
                              "achieved": round(step_bytes / (ms / k * 1e-3) / 1e9, 1),
                              "frac": round(step_bytes / (ms / k * 1e-3) / 1e9 / peak, 4)}}
        if prec == D.DDCC_FP32:
            kind = "fused_step" if kt.get("fused_step", (0, 0))[1] else "update"
            ms_u, n_u = kt[kind]
            ach = kb[kind] / (ms_u / n_u * 1e-3) / 1e9
            tpn = ncu_traffic_per_node(kind + "_3d")
            rec["roofline"] = {"kernel": kind + "_3d", "bound": "hbm", "achieved": round(ach, 1),
                               "peak": peak, "unit": "GB/s", "frac": round(ach / peak, 4),
                               "peak_kind": peak_kind,
                               "traffic": round(tpn * nodes) if tpn else None,
                               "algorithmic_bytes": kb[kind],
                               "avg_launch_ms": round(ms_u / n_u, 4),
                               "share_of_step": round(ms_u / total, 4)}
            out["fp32"] = rec
        else:
            rec["roofline"] = fp64_roofline_3d(kt, ms / k, nodes)
            out["fp64"] = rec
    if "fp32" in out and "fp64" in out:
        out["fp32_speedup_over_fp64"] = round(out["fp32"]["value"] / out["fp64"]["value"], 3)
    return out


def run_ours_3d(args, world, rank, local):
    """--workload sphere3d: one JSON line for the 3D sphere workload."""
    import workloads as W
    import __graft_entry__ as G
    G.build()
    import paper_2311_10314_gb300 as D
    peak, peak_kind = load_peaks()
    size = args.size if args.size != 4096 else 256
    sampler = ClockSampler(local)
    if args.precision == "fp64":
        # the FP64 step alone (three kernels) as the line, against the FP64 pipe
        r = three_d_step(D, W, size, 0, args.warmup, args.steps, world, peak, peak_kind, fp32=False)
        if rank == 0:
            f = r["fp64"]
            print(json.dumps({
                "metric": METRIC, "value": f["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": 2, "ms_per_step": f["ms_per_step"], "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": r["workload"], "nx": size, "ny": size, "nz": size,
                           "nphase": r["nphase"], "lattices": "D3Q7 phase, D3Q15 flow", "precision": "FP64",
                           "parallelism": "replicas" if world > 1 else "single GPU"},
                "roofline": f["roofline"], "whole_step": f["whole_step"], "kernels": f["kernels"],
                "cpu_baseline": None, "e2e": None, "gpu_launches": f["gpu_launches"],
                "mass_finite": f["mass_finite"]}), flush=True)
        return
    r = three_d_step(D, W, size, args.steps, args.warmup, 0 if args.no_extras else args.fp64_steps,
                     world, peak, peak_kind, sampler)
    if rank != 0:
        return
    f = r["fp32"]
    line = {
        "metric": METRIC, "value": f["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": f["ms_per_step"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": r["workload"], "nx": size, "ny": size, "nz": size,
                   "nphase": r["nphase"], "lattices": "D3Q7 phase, D3Q15 flow",
                   "precision": "FP32, g0 - rho0",
                   "l2": "state %.1f GB per step, larger than L2" % (
                       step_bytes_per_node_3d(r["nphase"], False, 4) * r["nodes"] / 1e9),
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "roofline": f["roofline"], "whole_step": f["whole_step"], "kernels": f["kernels"],
        "cpu_baseline": None, "e2e": None, "gpu_launches": f["gpu_launches"],
        "clocks": r.get("clocks"), "mass_finite": f["mass_finite"],
    }
    if "fp64" in r:
        line["fp64"] = {k: r["fp64"][k] for k in ("value", "unit", "ms_per_step", "kernels", "roofline")}
        line["fp32_speedup_over_fp64"] = r["fp32_speedup_over_fp64"]
    if not args.no_extras:
        line["e2e"] = e2e_3d(D, W, size, args.steps, world)
        if rank == 0:
            line["fp32_error"] = fp32_error_statement_3d(D, W, 128, 2000)
        if world == 1:
            pb3 = W.config7_sphere(L=size)
            mlups_c, cores, desc, _ = oracle_sample_3d(pb3, crop=32, steps=2)
            mlups_1 = oracle_sample_3d(pb3, crop=32, steps=1, threads=1)[0]
            line["cpu_baseline"] = {"value": round(mlups_c, 4), "unit": UNIT, "cores": cores,
                                    "kind": "oracle", "sample": desc,
                                    "value_1_thread": round(mlups_1, 4)}
    print(json.dumps(line), flush=True)


def e2e_3d(D, W, size, steps, world):
    """The 3D step end to end through the C ABI: ddcc3d_create from pinned
    host psi and C0 (H2D and the initial state), K steps, ddcc3d_read of
    every C_i (D2H) and the FP64 masses."""
    import torch
    from paper_2311_10314_gb300 import _lib
    pb = W.config7_sphere(L=size)
    N = pb.params["nphase"]
    nodes = size ** 3

    def pinned(a):
        t = torch.empty(a.shape, dtype=torch.float64, pin_memory=True)
        t.numpy()[...] = a
        return t
    ppsi, pc0 = pinned(pb.psi), pinned(pb.C0)
    out = [torch.empty((size, size, size), dtype=torch.float64, pin_memory=True) for _ in range(N)]
    torch.cuda.synchronize()
    barrier(world)
    t0 = time.perf_counter()
    sim = D.Sim3D(pb.params, ppsi.numpy(), pc0.numpy(), pb.cos_theta, precision=D.DDCC_FP32)
    sim.step(steps)
    for i in range(N):
        _lib.ddcc3d_read(sim.h, _lib.FIELD_C + i, out[i].numpy())
    sim.mass()
    t1 = time.perf_counter()
    sim.close()
    del sim
    torch.cuda.empty_cache()
    dt = allreduce_max(t1 - t0, world)
    return {"value": round(world * nodes * steps / dt / 1e6, 2), "unit": UNIT,
            "h2d_bytes_per_step": int((pb.psi.nbytes + pb.C0.nbytes) / steps),
            "d2h_bytes_per_step": int((N * nodes * 8 + (N - 1) * 8) / steps),
            "steps_per_run": steps,
            "what": "ddcc3d_create from pinned host psi/C0 (H2D + init), ddcc3d_step x K, "
                    "ddcc3d_read of every C_i (D2H), ddcc3d_mass"}


def fp64_roofline(D, kt64, nodes, N, theta_field, hbm_peak):
    """The FP64 step against the FP64 pipe: the FP64 flops its collide-stream
    kernel executes per node (ncu counters of one launch, committed under
    profiles/) times the nodes, over the kernel's CUDA-event time, against
    the FP64 FMA rate measured on this GPU; and the same kernel's
    algorithmic bytes against the HBM peak."""
    import torch
    from paper_2311_10314_gb300 import _lib
    ms, n = kt64.get("collide_stream", (0.0, 0))
    if not n:
        return None
    sink = torch.zeros(8 * torch.cuda.get_device_properties(0).multi_processor_count,
                       dtype=torch.float64, device="cuda")
    peak = _lib.ddcc_measure_fp64_peak(torch.cuda.current_stream().cuda_stream, sink.data_ptr())
    t = ms / n * 1e-3
    fpn = ncu_fp64_flops_per_node()
    hbm = collide_floats_per_node(N, theta_field) * 8 * nodes / t / 1e9
    out = {"kernel": "collide_stream", "bound": "fp64", "unit": "TFLOP/s",
           "peak": round(peak, 3), "peak_kind": "measured (ddcc_measure_fp64_peak)",
           "avg_launch_ms": round(ms / n, 4),
           "flops_per_node": fpn,
           "achieved": round(fpn * nodes / t / 1e12, 3) if fpn else None,
           "frac": round(fpn * nodes / t / 1e12 / peak, 4) if fpn else None,
           "hbm_GBps": round(hbm, 1), "hbm_frac": round(hbm / hbm_peak, 4)}
    return out


def run_ours(args, world, rank, local):
    import numpy as np
    import torch
    import workloads as W
    import __graft_entry__ as G
    G.build()
    import paper_2311_10314_gb300 as D
    from paper_2311_10314_gb300 import _lib

    pb = W.config4_imbibition(nx=args.size, ny=args.size)
    N = pb.params["nphase"]
    nodes = pb.nodes
    theta_field = pb.cos_theta_field is not None
    peak, peak_kind = load_peaks()

    main_prec = D.DDCC_FP64 if args.precision == "fp64" else D.DDCC_FP32
    sim = D.Sim(pb.params, pb.psi, pb.C0, pb.cos_theta, pb.cos_theta_field, precision=main_prec,
                path=args.path)
    path = sim.path
    sampler = ClockSampler(local)
    sim.step(args.warmup)
    torch.cuda.synchronize()
    sampler.start()
    ms, kt = timed_steps(D, sim, args.steps, 0, world)
    clocks = sampler.stop()
    ms_max = allreduce_max(ms, world)
    ms_step = ms_max / args.steps
    value = world * nodes * args.steps / (ms_max * 1e-3) / 1e6
    mass_ok = bool(np.isfinite(sim.mass()).all())
    sim.close()
    del sim
    torch.cuda.empty_cache()

    # roofline of the dominant kernel (the row sweep, or the tile kernels)
    es = 8 if main_prec == D.DDCC_FP64 else 4
    step_bytes = step_floats_per_node(N, theta_field) * es * nodes
    fused = kt.get("order_param", (0.0, 0))[1] == 0
    per_launch_bytes = {
        "row_sweep": step_bytes,
        "collide_stream": collide_floats_per_node(N, theta_field, fused) * es * nodes,
        "order_param": order_param_floats_per_node(N) * es * nodes,
        "ghost_fill": None,       # copies of the ghost frame, no method bytes
    }
    kinds = {k: v for k, v in kt.items() if v[1] > 0}
    dom = max((k for k in kinds if per_launch_bytes[k]), key=lambda k: kinds[k][0])
    ms_d, n_d = kinds[dom]
    achieved = per_launch_bytes[dom] / (ms_d / n_d * 1e-3) / 1e9
    total_ms = sum(v[0] for v in kinds.values())
    traffic_pn = ncu_traffic_per_node(dom)
    roofline = {
        "kernel": dom, "bound": "hbm",
        "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
        "frac": round(achieved / peak, 4), "peak_kind": peak_kind,
        "traffic": round(traffic_pn * nodes) if traffic_pn else None,
        "algorithmic_bytes": per_launch_bytes[dom],
        "avg_launch_ms": round(ms_d / n_d, 4),
        "share_of_step": round(ms_d / total_ms, 4),
        "kernels": {k: {"launches": v[1], "avg_ms": round(v[0] / v[1], 4),
                        "share": round(v[0] / total_ms, 4),
                        "algorithmic_GBps": (round(per_launch_bytes[k] / (v[0] / v[1] * 1e-3) / 1e9, 1)
                                             if per_launch_bytes[k] else None)}
                    for k, v in kinds.items()},
        "whole_step": {"algorithmic_bytes": step_bytes,
                       "achieved": round(step_bytes / (ms_step * 1e-3) / 1e9, 1),
                       "frac": round(step_bytes / (ms_step * 1e-3) / 1e9 / peak, 4)},
    }

    extras = {}
    e2e = None
    cpu = None
    if not args.no_extras:
        # FP64 step of the same workload
        sim = D.Sim(pb.params, pb.psi, pb.C0, pb.cos_theta, pb.cos_theta_field,
                    precision=D.DDCC_FP64, path=args.path)
        path64 = sim.path
        ms64, kt64 = timed_steps(D, sim, args.fp64_steps, 2, world)
        sim.close()
        del sim
        torch.cuda.empty_cache()
        ms64 = allreduce_max(ms64, world)
        fp64_value = world * nodes * args.fp64_steps / (ms64 * 1e-3) / 1e6
        extras["fp64"] = {"value": round(fp64_value, 2), "unit": UNIT,
                          "ms_per_step": round(ms64 / args.fp64_steps, 3), "step_path": path64,
                          "kernel_ms": {k: round(v[0] / max(v[1], 1), 4) for k, v in kt64.items()}}
        extras["fp64"]["roofline"] = fp64_roofline(D, kt64, nodes, N, theta_field, peak)
        extras["fp32_speedup_over_fp64"] = round(value / fp64_value, 3)

        # end to end through the C ABI with host buffers: upload of psi, C0
        # and the angle field from pinned memory, init, K steps, read-back of
        # every volume fraction and the FP64 masses
        def pinned(a):
            t = torch.empty(a.shape, dtype=torch.float64, pin_memory=True)
            t.numpy()[...] = a
            return t
        ppsi, pc0 = pinned(pb.psi), pinned(pb.C0)
        pcf = pinned(pb.cos_theta_field) if theta_field else None
        out = [torch.empty((pb.params["ny"], pb.params["nx"]), dtype=torch.float64,
                           pin_memory=True) for _ in range(N)]
        torch.cuda.synchronize()
        barrier(world)
        t0 = time.perf_counter()
        sim = D.Sim(pb.params, ppsi.numpy(), pc0.numpy(), pb.cos_theta,
                    None if pcf is None else pcf.numpy(), precision=D.DDCC_FP32, path=args.path)
        torch.cuda.synchronize()
        t_create = time.perf_counter()
        sim.step(args.steps)
        torch.cuda.synchronize()
        t_steps = time.perf_counter()
        for i in range(N):
            _lib.ddcc_read(sim.h, _lib.FIELD_C + i, out[i].numpy())
        sim.mass()
        t1 = time.perf_counter()
        sim.close()
        del sim
        torch.cuda.empty_cache()
        dt = allreduce_max(t1 - t0, world)
        h2d = pb.psi.nbytes + pb.C0.nbytes + (pb.cos_theta_field.nbytes if theta_field else 0)
        d2h = N * nodes * 8 + (N - 1) * 8
        e2e = {"value": round(world * nodes * args.steps / dt / 1e6, 2), "unit": UNIT,
               "h2d_bytes_per_step": int(h2d / args.steps),
               "d2h_bytes_per_step": int(d2h / args.steps),
               "steps_per_run": args.steps,
               "create_s": round(t_create - t0, 4), "steps_s": round(t_steps - t_create, 4),
               "readback_s": round(t1 - t_steps, 4),
               "what": "ddcc_create from pinned host psi/C0/theta (H2D + init), "
                       "ddcc_step x K, ddcc_read of every C_i (D2H), ddcc_mass"}
        if rank == 0:
            extras["fp32_error"] = fp32_error_statement(D, W, args.err_steps)
            extras["adjoint"] = adjoint_cost(D, W, args.adj_steps)
        # the 3D variant (D3Q7 / D3Q15) on the 256^3 sphere workload
        r3 = three_d_step(D, W, 256, 200, 5, 5, world, peak, peak_kind)
        if rank == 0:
            extras["three_d"] = {"workload": r3["workload"], "fp32": {
                k: r3["fp32"][k] for k in ("value", "ms_per_step", "whole_step", "roofline")},
                "fp64": {k: r3["fp64"][k] for k in ("value", "ms_per_step", "roofline")},
                "fp32_speedup_over_fp64": r3["fp32_speedup_over_fp64"]}
        if rank == 0 and world == 1:
            mlups_c, cores, desc, _ = oracle_sample(pb, crop=256, steps=2)
            mlups_1 = oracle_sample(pb, crop=256, steps=1, threads=1)[0]
            cpu = {"value": round(mlups_c, 4), "unit": UNIT, "cores": cores, "kind": "oracle",
                   "sample": desc, "value_1_thread": round(mlups_1, 4)}

    if rank != 0:
        return
    line = {
        "metric": METRIC, "value": round(value, 2), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_step, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if main_prec == D.DDCC_FP64 else "f32",
        "data": "synthetic",
        "config": {"workload": pb.name, "nx": pb.params["nx"], "ny": pb.params["ny"],
                   "step_path": path,
                   "nphase": N, "theta": "per-circle field",
                   "precision": "FP64" if main_prec == D.DDCC_FP64 else "FP32, g0 - rho0",
                   "l2": "state %.1f GB per step, larger than L2" % (
                       (18 * N + 2 * (2 * N + 3)) * es * nodes / 1e9),
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "roofline": roofline,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": sum(v[1] for v in kt.values()),
        "clocks": clocks,
        "mass_finite": mass_ok,
    }
    line.update(extras)
    print(json.dumps(line), flush=True)


def main():
    args = parse_args()
    world, rank, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, world, rank)
    elif args.workload == "sphere3d":
        run_ours_3d(args, world, rank, local)
    else:
        run_ours(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
