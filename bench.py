#!/usr/bin/env python3
"""Throughput of the fused D2Q9 OReg-GEq step (arXiv 2602.21242, Eq. 1) on GB300.

One benchmark step = one pass of the whole hot path over the lattice: pull
streaming, moments, guided equilibrium, Onsager-regularised non-equilibrium,
compatibility and stress corrections, relaxation, store, and the fused FP64
diagnostics reduction (mass, momentum, kinetic energy, non-finite count).

Workload (default): 4096 x 4096 doubly periodic advected shear wave,
u_y = 0.01 sin(2 pi x / nx) on u_x = U = 0.1, rho = 1, theta = 1/3, nu = 0.005,
completely corrected model, FP64 storage and arithmetic. Inputs are larger than
L2 (two 1.2 GB population buffers vs 129 MB).

Prints ONE JSON line (rank 0). ``--impl reference`` times the FP64 CPU oracle
on the host cores instead (the reference arm).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "MLUPS and % of HBM roofline, D2Q9 OReg-GEq; FP32 vs FP64 at stated error"
BYTES_PER_NODE = {"f64": 144, "f32": 72, "f16": 36, "f64df": 144}
# Algorithmic FP64 operations per node of one fused step (each add, mul or FMA of
# the product-form collision is one operation, the exact power-of-two scalings
# too): 33 shared (moments 16, 1/rho 3, u 2, u^2 2, u/2 2, P 8), the model part
# (LBGK 22, OReg 55, partial 65, complete 85, the mu sum and Pi~ sharing u^2 - 1;
# complete with the Eq. 12 prefactor from f^neq 82) and the fused diagnostics (5:
# three sums and j.u by two FMAs).
FP64_OPS_PER_NODE = {"lbgk": 60, "oreg": 93, "partial": 103, "complete": 123, "complete_neq": 120}
# The FP64 form on GB300 is bound by the FP64 pipe, which carries only the sums and
# FMAs of that count: the products run on the integer pipes (correctly rounded
# binary64 products from the operands' bit fields, bit-identical to the FP64
# instruction) and the power-of-two scalings move exponent bits there too.
FP64_PIPE_OPS_PER_NODE = {"lbgk": 41, "oreg": 71, "partial": 73, "complete": 86, "complete_neq": 84}
INT_PIPE_PRODUCTS_PER_NODE = {"lbgk": 17, "oreg": 20, "partial": 24, "complete": 31, "complete_neq": 29}
FALLBACK_HBM_GBS = 6800.0
# DRAM bytes (read + write) per node of one step-kernel launch, from ncu captures of
# the current kernels: the FP64 kernel captured at 2048^2 and scaled to the lattice by
# node count (its traffic grows in proportion), the FP32 kernels (single steps, and two
# steps a launch) captured at 4096^2.
# Keyed by (storage, model, steps per launch).
PROFILED_TRAFFIC_B_PER_NODE = {("f64", "complete", 1): 133.7, ("f32", "complete", 1): 68.8,
                               ("f32", "complete", 2): 72.1}
MODEL_NAMES = ["lbgk", "oreg", "partial", "complete", "complete_neq"]
# the step kernel each storage form launches under its default launch shape
STEP_KERNEL = {"f64": "step_kernel_f64", "f64df": "step_kernel_df", "f32": "step_stream_persistent_kernel",
               "f16": "step_stream_kernel"}


def parse_args():
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--n", type=int, default=4096, help="lattice side (nx = ny)")
    ap.add_argument("--model", default="complete", choices=MODEL_NAMES)
    ap.add_argument("--prec", default="f64", choices=["f64", "f32", "f16", "f64df"])
    ap.add_argument("--no-forms", action="store_true", help="skip the per-model / per-precision sweep")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end host-buffer measurement")
    ap.add_argument("--precision-study", action="store_true",
                    help="run the 8192^2 shear-layer precision study instead of the benchmark")
    ap.add_argument("--study-steps", type=int, default=5000)
    ap.add_argument("--experiments", action="store_true",
                    help="run the paper's rotated-shear-wave and shear-layer experiments instead of the benchmark")
    ap.add_argument("--e2e-steps", type=int, default=50, help="lattice steps per end-to-end call")
    ap.add_argument("--e2e-calls", type=int, default=3)
    ap.add_argument("--batch-steps", type=int, default=1000, help="steps of the 256-domain batched workload")
    ap.add_argument("--batch-tile", default="", help="kind,bx,by,rows (or bx,by,rows for kind 0) of the batched tiles (default: autotuned)")
    ap.add_argument("--config-sweep", action="store_true",
                    help="time every model, U and theta of the 4096^2 shear-wave benchmark (FP64 and double-float)")
    ap.add_argument("--sweep-steps", type=int, default=200)
    ap.add_argument("--vjp-only", action="store_true",
                    help="run only the differentiation workload (gradient through lbm_vjp) and print its JSON")
    ap.add_argument("--vjp-steps", type=int, default=500, help="steps of the differentiation workload")
    ap.add_argument("--batch-only", action="store_true",
                    help="run only the 256-domain batched workload (graph and persistent modes) and print its JSON")
    return ap.parse_args()


def workload(n: int):
    theta, nu, U = 1.0 / 3.0, 0.005, 0.1
    return {"nx": n, "ny": n, "theta": theta, "nu": nu, "tau": nu / theta + 0.5, "U": U, "amp": 0.01}


def workload_name(w, model, prec):
    return (f"advected shear wave {w['nx']}x{w['ny']} periodic, u_y=0.01 sin(2 pi x/nx), U={w['U']}, "
            f"theta=1/3, nu={w['nu']}, {model} model, {prec} storage, diagnostics every step")


def hbm_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return FALLBACK_HBM_GBS, "fallback"


# ----------------------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi samples every 200 ms while the timed region runs."""

    FIELDS = ["index", "clocks.sm", "clocks.max.sm", "power.draw", "clocks_event_reasons.active",
              "clocks_event_reasons.hw_slowdown", "clocks_event_reasons.hw_thermal_slowdown",
              "clocks_event_reasons.sw_thermal_slowdown", "clocks_event_reasons.sw_power_cap"]

    def __init__(self, gpu_id: str):
        self.gpu_id = gpu_id
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "--query-gpu=" + ",".join(self.FIELDS), "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", self.gpu_id], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [ln for ln in out.splitlines() if ln.strip()]

    def summary(self):
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in getattr(self, "lines", []):
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < len(self.FIELDS):
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


# ----------------------------------------------------------------------------- CPU oracle

def oracle_mlups(w, model, target_s=12.0, nx=None, ny=None):
    """Time the FP64 oracle (all host cores) on the workload's flow; returns (mlups, cores, sample)."""
    import numpy as np
    from oracle import oracle as O
    from paper_2602_21242_gb300 import flows

    cores = O.set_threads(os.cpu_count() or 1)
    nx = nx or w["nx"]
    ny = ny or w["ny"]
    m = MODEL_NAMES.index(model)
    rho, ux, uy = flows.shear_wave(nx, ny, U=w["U"], amp=w["amp"])
    f = O.init(rho, ux, uy, w["theta"])
    del rho, ux, uy
    t0 = time.perf_counter()
    f = O.run(f, w["theta"], w["tau"], m, 1)  # calibration step
    t1 = time.perf_counter() - t0
    steps = max(1, int(target_s / max(t1, 1e-6)))
    t0 = time.perf_counter()
    f = O.run(f, w["theta"], w["tau"], m, steps)
    dt = time.perf_counter() - t0
    assert np.isfinite(f[:, :2, :2]).all()
    sample = f"{nx}x{ny} grid of the same flow, {steps} oracle steps of the {model} model, {dt:.1f} s"
    return nx * ny * steps / dt / 1e6, cores, sample


def oracle_single_thread_mlups(w, model, target_s=3.0, rows=64):
    """The FP64 oracle on one host thread over a band of `rows` rows of the workload's flow (the
    flow depends on x only, so a periodic band is the same flow); returns (mlups, sample)."""
    from oracle import oracle as O
    from paper_2602_21242_gb300 import flows

    prev = O.set_threads(0)
    O.set_threads(1)
    try:
        nx, ny = w["nx"], min(rows, w["ny"])
        m = MODEL_NAMES.index(model)
        f = O.init(*flows.shear_wave(nx, ny, U=w["U"], amp=w["amp"]), w["theta"])
        t0 = time.perf_counter()
        f = O.run(f, w["theta"], w["tau"], m, 1)  # calibration step
        steps = max(1, int(target_s / max(time.perf_counter() - t0, 1e-6)))
        t0 = time.perf_counter()
        f = O.run(f, w["theta"], w["tau"], m, steps)
        dt = time.perf_counter() - t0
    finally:
        O.set_threads(prev)
    return nx * ny * steps / dt / 1e6, f"{nx}x{ny} periodic band of the same flow, {steps} oracle steps, {dt:.1f} s"


# ----------------------------------------------------------------------------- GPU arm

def run_gpu(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2602_21242_gb300 import capi, flows
    from paper_2602_21242_gb300.lattice import Lattice

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    capi.load()
    stream = torch.cuda.current_stream(dev)

    w = workload(args.n)
    n = w["nx"] * w["ny"]
    rho, ux, uy = flows.shear_wave(w["nx"], w["ny"], U=w["U"], amp=w["amp"])
    fields = [torch.from_numpy(a).to(dev) for a in (rho, ux, uy)]

    def barrier():
        torch.cuda.synchronize(dev)
        if world > 1:
            dist.barrier()

    # ---- headline: timed region
    lat = Lattice(w["nx"], w["ny"], w["theta"], w["tau"], args.model, args.prec, device=dev, stream=stream)
    lat.init(*fields)
    lat.set_diagnostics_interval(1)
    # steps per launch: 2 under launch kind 2 (the FP32 default where it applies), timed per launch
    # (kind 2 applies where nx is a multiple of the 16-byte chunk)
    chunk = {"f32": 4, "f16": 8}.get(args.prec, 0)
    spl = 2 if capi.lbm_get_launch_ex(lat.ctx)[0] == 2 and chunk and w["nx"] % chunk == 0 else 1
    for _ in range(args.warmup):
        lat.step(spl)
    lat.sync()
    props = torch.cuda.get_device_properties(dev)
    gpu_id = str(getattr(props, "uuid", local))
    if gpu_id and not gpu_id.startswith("GPU-") and len(gpu_id) == 36:
        gpu_id = "GPU-" + gpu_id
    launches = -(-args.steps // spl)
    args.steps = launches * spl
    events = [torch.cuda.Event(enable_timing=True) for _ in range(launches + 1)]
    barrier()
    with ClockSampler(gpu_id) as clocks:
        events[0].record(stream)
        for k in range(launches):
            lat.step(spl)
            events[k + 1].record(stream)
        barrier()
    total_ms = events[0].elapsed_time(events[-1])
    per_launch = [events[k].elapsed_time(events[k + 1]) for k in range(launches)]
    diag, t_diag, status = lat.step_diagnostics()
    total_ms = max_over_ranks(total_ms, world, dev)
    mlups = aggregate_mlups(n, args.steps, total_ms, world)
    launch_ms = statistics.mean(per_launch)
    step_ms = launch_ms / spl

    # ---- roofline of the step kernel (fused step + its tiny diagnostics finalisation); a
    # two-step launch reads and writes the state once, so its algorithmic bytes per launch
    # are one step's
    peak_hbm, hbm_src = hbm_peak()
    bytes_launch = BYTES_PER_NODE[args.prec] * n
    hbm_gbs = bytes_launch / (launch_ms * 1e-3) / 1e9
    tpn = PROFILED_TRAFFIC_B_PER_NODE.get((args.prec, args.model, spl))
    traffic = round(tpn * n) if tpn is not None else None
    roof = {"bound": "hbm", "achieved": round(hbm_gbs, 1), "peak": peak_hbm, "unit": "GB/s",
            "frac": round(hbm_gbs / peak_hbm, 4), "traffic": traffic,
            "peak_source": f"{hbm_src} copy bandwidth (MEASURED_PEAKS.json hbm_gbs)" if hbm_src == "measured"
            else "profiling-recipe fallback 6.8 TB/s",
            "kernel": f"{'step2_stream_kernel' if spl == 2 else STEP_KERNEL[args.prec]}<{args.model},diag>",
            "ms_per_launch": round(launch_ms, 4), "steps_per_launch": spl}
    alu = None
    if args.prec == "f64":
        peak_ops = capi.lbm_measure_peak(0) / 2.0  # FMA instructions per second (2 FLOP each)
        ops = FP64_PIPE_OPS_PER_NODE[args.model] * n / (step_ms * 1e-3)
        alu = {"bound": "alu", "achieved": round(ops / 1e12, 4), "peak": round(peak_ops / 1e12, 4),
               "unit": "Top/s (FP64-pipe add/fma)", "frac": round(ops / peak_ops, 4), "traffic": traffic,
               "peak_source": "FP64 FMA issue rate measured live on this GPU (lbm_measure_peak / 2)",
               "ops_per_node": FP64_PIPE_OPS_PER_NODE[args.model],
               "method_ops_per_node": FP64_OPS_PER_NODE[args.model],
               "integer_pipe_products_per_node": INT_PIPE_PRODUCTS_PER_NODE[args.model],
               "method_ops_rate": round(FP64_OPS_PER_NODE[args.model] * n / (step_ms * 1e-3) / 1e12, 4),
               "kernel": roof["kernel"], "ms_per_launch": round(step_ms, 4)}
        if alu["frac"] > roof["frac"]:
            roof, alu = alu, roof
    lat.close()
    del lat

    out = {"metric": METRIC, "value": round(mlups, 2), "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": round(total_ms / args.steps, 4), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None,
           "dtype": {"f64": "f64", "f64df": "f32x2 double-float (FP64 storage)"}.get(args.prec, "f32"),
           "data": "synthetic",
           "config": {"workload": workload_name(w, args.model, args.prec), "nx": w["nx"], "ny": w["ny"],
                      "collision": args.model, "storage": args.prec, "theta": w["theta"], "nu": w["nu"],
                      "tau": w["tau"], "U": w["U"],
                      "l2": f"inputs larger than L2: two {lat_bytes(args.prec, n)/1e9:.2f} GB population buffers",
                      "parallelism": f"one independent lattice per GPU (replicas), {world} GPU(s)"},
           "roofline": roof, "roofline_other": alu,
           "gpu_launches": launches * (1 + spl),
           "gpu_launches_note": f"per launch: 1 fused step kernel ({spl} step(s)) + {spl} diagnostics finalisation "
                                f"kernel(s)",
           "clocks": clocks.summary(),
           "final_diagnostics": {"t": t_diag, "mass": diag[0], "mom_x": diag[1], "mom_y": diag[2],
                                 "kinetic": diag[3], "nonfinite": diag[4]}}

    # ---- end to end through the host-buffer entry point
    if not args.no_e2e:
        host = [torch.from_numpy(a).pin_memory() for a in (rho, ux, uy)]
        res = [torch.empty((w["ny"], w["nx"]), dtype=torch.float64).pin_memory() for _ in range(3)]
        lat = Lattice(w["nx"], w["ny"], w["theta"], w["tau"], args.model, args.prec, device=dev, stream=stream)
        lat.set_diagnostics_interval(1)
        ptrs = [h.data_ptr() for h in host] + [r.data_ptr() for r in res]
        capi.lbm_run_host(lat.ctx, *ptrs[:3], 2, *ptrs[3:], want_diag=True)  # warm-up (staging allocation)
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.e2e_calls):
            capi.lbm_run_host(lat.ctx, *ptrs[:3], args.e2e_steps, *ptrs[3:], want_diag=True)
        barrier()
        dt = max_over_ranks(time.perf_counter() - t0, world, dev)
        lat.close()
        out["e2e"] = {"value": round(world * n * args.e2e_steps * args.e2e_calls / dt / 1e6, 2), "unit": "MLUPS",
                      "h2d_bytes_per_step": round(3 * 8 * n / args.e2e_steps),
                      "d2h_bytes_per_step": round((3 * 8 * n + 5 * 8) / args.e2e_steps),
                      "call": f"lbm_run_host: upload rho0,u0 (pinned) -> init -> {args.e2e_steps} steps with "
                              f"diagnostics -> download rho,u and diagnostics; {args.e2e_calls} calls timed"}

    # ---- per-model / per-precision sweep on the same flow, and the batched workload
    if not args.no_forms:
        out["forms"] = forms_sweep(w, fields, dev, stream, peak_hbm)
        out["forms"].update(batch_sweep(dev, stream, peak_hbm, steps=args.batch_steps))
        out["forms"].update(vjp_sweep(dev, stream, steps=args.vjp_steps))

    # ---- CPU baseline (oracle) on rank 0 at N = 1
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, cores, sample = oracle_mlups(w, args.model)
        out["cpu_baseline"] = {"value": round(v, 3), "unit": "MLUPS", "cores": cores, "kind": "oracle",
                               "sample": sample}
        v1, sample1 = oracle_single_thread_mlups(w, args.model)
        out["cpu_baseline"]["single_thread"] = {"value": round(v1, 3), "unit": "MLUPS", "cores": 1,
                                                "sample": sample1}
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


def max_over_ranks(x: float, world: int, device) -> float:
    """Largest value of x over the ranks of the default process group (x itself when world == 1)."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist

    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_mlups(nodes_per_rank: int, steps: int, max_ms: float, world: int) -> float:
    """Whole-job MLUPS: every rank advances its own lattice (weak scaling), timed by the slowest rank."""
    return world * nodes_per_rank * steps / (max_ms * 1e-3) / 1e6


def lat_bytes(prec, n):
    return BYTES_PER_NODE[prec] // 2 * n


def forms_sweep(w, fields, dev, stream, peak_hbm, steps=100, warm=5, err_steps=200):
    """MLUPS of every model in FP64 and in the double-float form (FP64 storage, FP32-pair
    arithmetic), and of the complete model in the shifted FP32 / FP16 forms, with the velocity
    error of the non-FP64 forms against FP64 after err_steps steps."""
    import torch

    from paper_2602_21242_gb300.lattice import Lattice

    n = w["nx"] * w["ny"]
    res = {}

    from paper_2602_21242_gb300 import capi

    def timed(model, prec, diag_every=1, launch=None):
        lat = Lattice(w["nx"], w["ny"], w["theta"], w["tau"], model, prec, device=dev, stream=stream)
        if launch is not None:
            capi.lbm_set_launch_ex(lat.ctx, *launch)
        kind = capi.lbm_get_launch_ex(lat.ctx)[0]
        lat.init(*fields)
        lat.set_diagnostics_interval(diag_every)
        lat.step(warm)
        lat.sync()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        lat.step(steps)
        e1.record(stream)
        lat.sync()
        ms = e0.elapsed_time(e1) / steps
        lat.close()
        mlups = n / (ms * 1e-3) / 1e6
        if kind == 2:
            # two steps a launch: the state is read and written once per two steps, so the
            # algorithmic traffic of a step is half the single step's; the rate is also
            # given against the single-step HBM roof
            bpn = BYTES_PER_NODE[prec] / 2
            gbs = bpn * n / (ms * 1e-3) / 1e9
            return {"mlups": round(mlups, 1), "ms_per_step": round(ms, 4), "launch": "two steps a launch (kind 2)",
                    "bytes_per_node_step": bpn, "hbm_gbs": round(gbs, 1), "hbm_frac": round(gbs / peak_hbm, 4),
                    "vs_single_step_hbm_roof": round(2 * gbs / peak_hbm, 4)}
        gbs = BYTES_PER_NODE[prec] * n / (ms * 1e-3) / 1e9
        return {"mlups": round(mlups, 1), "ms_per_step": round(ms, 4), "hbm_gbs": round(gbs, 1),
                "hbm_frac": round(gbs / peak_hbm, 4)}

    for model in MODEL_NAMES:
        res[f"{model}/f64"] = timed(model, "f64")
    for model in MODEL_NAMES:
        res[f"{model}/f64df"] = timed(model, "f64df")
    for prec in ("f32", "f16"):
        res[f"complete/{prec}"] = timed("complete", prec)
        res[f"complete/{prec}/diagnostics_every_100"] = timed("complete", prec, 100)
    # FP32 single steps (the persistent pipeline on 4-row tiles) beside the default two-step launch
    res["complete/f32/single_step"] = timed("complete", "f32", 1, (1, 64, 1, 4))

    # velocity error of the double-float and shifted forms against FP64 on the same flow
    finals = {}
    for prec in ("f64", "f64df", "f32", "f16"):
        lat = Lattice(w["nx"], w["ny"], w["theta"], w["tau"], "complete", prec, device=dev, stream=stream)
        lat.init(*fields)
        lat.step(err_steps)
        finals[prec] = [t.clone() for t in lat.moments()]
        lat.close()
    for prec in ("f64df", "f32", "f16"):
        du = max(float((finals[prec][k] - finals["f64"][k]).abs().max()) for k in (1, 2))
        dr = float((finals[prec][0] - finals["f64"][0]).abs().max())
        res[f"complete/{prec}"]["error_vs_f64"] = {
            "steps": err_steps, "max_abs_du_over_U": du / w["U"], "max_abs_drho": dr}
    return res


def batch_sweep(dev, stream, peak_hbm, steps=1000, tile=None):
    """Batched workload: 256 independent Taylor-Green domains, N ~ U{64..512}, theta ~ U[0.25, 0.4],
    nu ~ U[0.002, 0.02], u0 ~ U[0.02, 0.1], completely corrected model, FP32 shifted storage, `steps`
    steps per call; tile shape from the autotuner; graph mode (fused per-domain diagnostics every
    step) and persistent mode (one cooperative launch, no fused diagnostics)."""
    import torch

    from paper_2602_21242_gb300 import flows, tune
    from paper_2602_21242_gb300.batch import Batch

    doms = flows.batch_domains(256)
    ns = [d.n for d in doms]
    thetas = [d.theta for d in doms]
    taus = [d.nu / d.theta + 0.5 for d in doms]
    fields = [flows.taylor_green(d.n, d.n, d.u0, d.theta) for d in doms]
    rho, ux, uy = ([f[j] for f in fields] for j in range(3))
    res = {}
    with Batch(ns, ns, thetas, taus, "complete", "f32", device=dev, stream=stream) as b:
        if tile is None:
            shape, _ = tune.tune_batch(b, steps=10, use_cache=False)
        else:
            shape = tuple(tile)
            b.set_launch(*shape)
        nodes = b.total_nodes
        for mode in ("graph", "persistent"):
            b.set_mode(mode)
            b.set_diagnostics_interval(1 if mode == "graph" else 0)
            b.init(rho, ux, uy)
            b.step(steps)  # warm-up (graph capture)
            b.sync()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            b.step(steps)
            e1.record(stream)
            b.sync()
            ms = e0.elapsed_time(e1) / steps
            d = b.diagnostics()
            mass = sum(x[0] for x in d)
            # a kind 2 batch runs two steps a launch (graph mode) or a pair of steps between grid
            # barriers (persistent mode): 36 B a node-step
            two = shape[0] == 2
            bpn = 36 if two else 72
            res[f"batch256/complete/f32/{mode}"] = {
                "mlups": round(nodes / (ms * 1e-3) / 1e6, 1), "ms_per_step": round(ms, 4),
                "bytes_per_node_step": bpn, "hbm_gbs": round(bpn * nodes / (ms * 1e-3) / 1e9, 1),
                "hbm_frac": round(bpn * nodes / (ms * 1e-3) / 1e9 / peak_hbm, 4),
                "vs_single_step_hbm_roof": round(72 * nodes / (ms * 1e-3) / 1e9 / peak_hbm, 4),
                "steps_per_launch": 2 if two else 1,
                "domains": 256, "nodes": nodes, "steps": steps, "tile": list(shape),
                "fused_diagnostics": mode == "graph", "mass_rel_drift": abs(mass - sum(rho_k.sum() for rho_k in rho)) / mass}
    return res


def vjp_sweep(dev, stream, n=1024, steps=500, ckpt=50):
    """Differentiation workload: 1024^2 periodic, initial velocity from random Fourier modes
    |k| <= 8 scaled to max |u| = 0.02, theta = 1/3, nu = 0.01, 500 steps, completely corrected
    model; loss = 1/2 sum (rho_T - rho_target)^2 against a target run from the next seed;
    gradient with respect to (rho0, u0) through lbm_vjp with checkpoints every 50 steps, in
    FP64, in the double-float form and in the FP32 form, with each gradient's relative error
    against FP64."""
    import torch

    from paper_2602_21242_gb300 import flows
    from paper_2602_21242_gb300.lattice import Lattice, run

    theta, nu = 1.0 / 3.0, 0.01
    tau = nu / theta + 0.5
    x0 = [torch.from_numpy(a).to(dev) for a in flows.random_modes(n, seed=flows.SEED_BASE + 4)]
    tgt = [torch.from_numpy(a).to(dev) for a in flows.random_modes(n, seed=flows.SEED_BASE + 5)]
    with Lattice(n, n, theta, tau, "complete", "f64", device=dev, stream=stream) as lat:
        lat.init(*tgt)
        lat.step(steps)
        rho_t = lat.moments()[0].clone()
    res, grads = {}, {}
    for prec in ("f64", "f64df", "f32"):
        with Lattice(n, n, theta, tau, "complete", prec, device=dev, stream=stream) as lat:
            for rep in range(2):  # first pass allocates the work memory
                x = [t.clone().requires_grad_(True) for t in x0]
                e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
                e0.record(stream)
                rho, _, _ = run(lat, *x, steps, ckpt_every=ckpt)
                loss = 0.5 * ((rho - rho_t) ** 2).sum()
                e1.record(stream)
                loss.backward()
                e2.record(stream)
                torch.cuda.synchronize(dev)
            fwd_ms, bwd_ms = e0.elapsed_time(e1), e1.elapsed_time(e2)
            grads[prec] = [t.grad.detach() for t in x]
            res[f"vjp1024/complete/{prec}"] = {
                "forward_ms": round(fwd_ms, 2), "backward_ms": round(bwd_ms, 2), "loss": float(loss.detach()),
                "gradient_mlups": round(n * n * steps / ((fwd_ms + bwd_ms) * 1e-3) / 1e6, 1),
                "steps": steps, "ckpt_every": ckpt,
                "note": "forward = lbm_vjp_forward (checkpoints kept); backward = segment recomputes + adjoint steps"}
    den = sum(float((b ** 2).sum()) for b in grads["f64"])
    for prec in ("f64df", "f32"):
        num = sum(float(((a - b) ** 2).sum()) for a, b in zip(grads[prec], grads["f64"]))
        res[f"vjp1024/complete/{prec}"]["grad_rel_l2_error_vs_f64"] = (num / den) ** 0.5
    return res


# ----------------------------------------------------------------------------- reference arm

def run_reference(args):
    """The FP64 CPU oracle, as it stands, timed on the host cores (the reference arm)."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from oracle import oracle as O
    from paper_2602_21242_gb300 import flows

    w = workload(args.n)
    cores = O.set_threads(os.cpu_count() or 1)
    m = MODEL_NAMES.index(args.model)
    # bounded sample per step: a band of rows of the same flow, sized to ~1 s of oracle work
    band = min(w["ny"], 256)
    rho, ux, uy = flows.shear_wave(w["nx"], band, U=w["U"], amp=w["amp"])
    f = O.init(rho, ux, uy, w["theta"])
    t0 = time.perf_counter()
    f = O.run(f, w["theta"], w["tau"], m, 1)
    t1 = time.perf_counter() - t0
    band = max(8, min(w["ny"], int(band * 1.0 / max(t1, 1e-6))))
    rho, ux, uy = flows.shear_wave(w["nx"], band, U=w["U"], amp=w["amp"])
    f = O.init(rho, ux, uy, w["theta"])
    for _ in range(args.warmup):
        f = O.run(f, w["theta"], w["tau"], m, 1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        f = O.run(f, w["theta"], w["tau"], m, 1)
    dt = time.perf_counter() - t0
    nodes = w["nx"] * band
    mlups = nodes * args.steps / dt / 1e6
    sample = f"per step: one oracle step on a {w['nx']}x{band} periodic band of the same flow"
    out = {"impl": "reference", "metric": METRIC, "value": round(mlups, 3), "unit": "MLUPS", "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(dt / args.steps * 1e3, 3),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic",
           "config": {"workload": workload_name(w, args.model, "f64"), "nx": w["nx"], "ny": w["ny"],
                      "collision": args.model, "storage": "f64", "theta": w["theta"], "nu": w["nu"],
                      "tau": w["tau"], "U": w["U"]},
           "cpu_baseline": {"value": round(mlups, 3), "unit": "MLUPS", "cores": cores, "kind": "oracle",
                            "sample": sample},
           "e2e": {"value": round(mlups, 3), "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def config_sweep(args):
    """The bandwidth benchmark's full matrix: 4096^2 advected shear wave with u_x = U in {0, 0.1, 0.2},
    theta in {0.25, 1/3, 0.4}, nu = 0.005, every model, FP64 and the double-float form; MLUPS over
    `--sweep-steps` steps with fused diagnostics every step, and whether the state stayed finite."""
    import torch

    from paper_2602_21242_gb300 import flows
    from paper_2602_21242_gb300.lattice import Lattice

    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    n, nu, steps = 4096, 0.005, args.sweep_steps
    table = {}
    for U in (0.0, 0.1, 0.2):
        fields = [torch.from_numpy(a).to(dev) for a in flows.shear_wave(n, n, U=U, amp=0.01)]
        for theta in (0.25, 1.0 / 3.0, 0.4):
            for prec in ("f64", "f64df"):
                for model in MODEL_NAMES:
                    with Lattice(n, n, theta, nu / theta + 0.5, model, prec, device=dev, stream=stream) as lat:
                        lat.init(*fields)
                        lat.set_diagnostics_interval(1)
                        lat.step(5)
                        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                        e0.record(stream)
                        lat.step(steps)
                        e1.record(stream)
                        torch.cuda.synchronize(dev)
                        ms = e0.elapsed_time(e1) / steps
                        d, t, status = lat.step_diagnostics(raise_nonfinite=False)
                    table[f"U={U}/theta={theta:.3f}/{prec}/{model}"] = {
                        "mlups": round(n * n / (ms * 1e-3) / 1e6, 1), "finite": status == 0 and d[4] == 0}
    print(json.dumps({"sweep": "4096^2 advected shear wave, nu=0.005", "steps": steps, "results": table}),
          flush=True)


def precision_study(args):
    """8192^2 doubly periodic shear layer (u_x = 0.1 tanh((y - ny/4)/80), mirrored; u_y = 0.005
    sin(2 pi x / nx)), theta = 0.3, nu = 1e-3, completely corrected model, `--study-steps` steps in
    FP64, FP64 storage with double-float arithmetic, FP32-shifted and FP16-shifted storage; prints
    the velocity and density error of the other forms against FP64 and each form's throughput. LBGK is run in FP64 alongside to record
    whether it stays finite at this Reynolds number (U N / nu = 8.2e5)."""
    import torch

    from paper_2602_21242_gb300 import flows
    from paper_2602_21242_gb300.lattice import Lattice

    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    n, theta, nu, U = 8192, 0.3, 1e-3, 0.1
    tau = nu / theta + 0.5
    fields = [torch.from_numpy(a).to(dev) for a in flows.shear_layer(n, n, U=U, width=80.0, delta_amp=0.005)]
    res, final = {}, {}
    for model, prec in (("complete", "f64"), ("complete", "f64df"), ("complete", "f32"), ("complete", "f16"),
                        ("lbgk", "f64")):
        with Lattice(n, n, theta, tau, model, prec, device=dev, stream=stream) as lat:
            lat.init(*fields)
            lat.set_diagnostics_interval(100)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            lat.step(args.study_steps)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            ms = e0.elapsed_time(e1)
            d, t, status = lat.step_diagnostics(raise_nonfinite=False)
            if model == "complete":
                final[prec] = [x.clone() for x in lat.moments()]
            res[f"{model}/{prec}"] = {"mlups": round(n * n * args.study_steps / (ms * 1e-3) / 1e6, 1),
                                      "finite": status == 0 and d[4] == 0, "mass": d[0], "t_diag": t}
    for prec in ("f64df", "f32", "f16"):
        du = max(float((final[prec][k] - final["f64"][k]).abs().max()) for k in (1, 2))
        du_rms = max(float(((final[prec][k] - final["f64"][k]) ** 2).mean().sqrt()) for k in (1, 2))
        dr = float((final[prec][0] - final["f64"][0]).abs().max())
        res[f"complete/{prec}"].update({"max_abs_du_over_U": du / U, "rms_du_over_U": du_rms / U,
                                         "max_abs_drho": dr})
    print(json.dumps({"study": "shear-layer precision, 8192^2, theta=0.3, nu=1e-3, U=0.1",
                      "steps": args.study_steps, "results": res}), flush=True)


def paper_experiments(args):
    """Sec. 5.1: nu~/nu of the rotated decaying shear wave (N = 200, nu = 1e-3, 1200 steps) for every
    model (with both readings of the LBGK equilibrium), theta in {0.25, 1/3, 0.4, 0.5}, Ma = 0.1 .. 1.0
    (0 = the run became non-finite), for the wave along y on a column and along the lattice diagonal,
    and for two fitting windows.
    Sec. 5.3: the doubly periodic shear layer (kappa = 80, delta = 0.05, u0 = 0.04, Re = 3e4) to one
    turnover time for N in {128, 256, 512}, theta in {0.4, 0.6}: whether each model stays finite.
    Sec. 5.2: the isothermal shocktube (800 x 1, bounce-back walls, 400 steps) at (theta, nu) =
    (0.4, 1e-12) and (0.55, 1e-9): range and total variation of the density (the comparison with the
    exact isothermal Riemann solution is made by the tests, on the oracle side)."""
    import torch

    from paper_2602_21242_gb300 import experiments

    torch.cuda.set_device(0)
    models = ["lbgk", "oreg", "partial", "complete", "complete_neq"]
    mas = [round(0.1 * k, 1) for k in range(1, 11)]
    # two orientations of the wave, both readings of the LBGK equilibrium (GEq and the polynomial one),
    # and two fitting windows of nu~ (the default t = 200 .. 1200 and a later one, t = 600 .. 1200)
    table = {}
    for orientation in ("axis", "diagonal"):
        for t_fit in (200, 600):
            for theta in experiments.SHEAR_WAVE_THETAS:
                for model in models + ["lbgk_poly"]:
                    if t_fit != 200 and model not in ("lbgk", "lbgk_poly", "oreg"):
                        continue
                    table[f"{orientation}/t_fit={t_fit}/{model}/theta={theta:.3f}"] = [
                        round(experiments.rotated_shear_wave_viscosity(model, theta, ma, t_fit=t_fit,
                                                                       orientation=orientation), 4) for ma in mas]
    layer = {}
    for theta in experiments.SHEAR_LAYER_THETAS:
        for n in experiments.SHEAR_LAYER_GRIDS:
            for model in models + ["lbgk_poly"]:
                finite, steps, w = experiments.shear_layer_run(model, theta, n)
                layer[f"{model}/theta={theta}/N={n}"] = {
                    "finite": finite, "steps": steps,
                    "max_abs_vorticity": None if w is None else float(abs(w).max())}
    tube = {}
    for theta, nu in experiments.SHOCKTUBE_CASES:
        for model in models + ["lbgk_poly"]:
            r = experiments.shocktube_run(model, theta, nu)
            entry = {"finite": r["finite"]}
            if r["finite"]:
                mid = r["rho"][len(r["rho"]) // 2]
                entry.update({"rho_min": float(r["rho"].min()), "rho_max": float(r["rho"].max()),
                              "ux_max": float(r["ux"].max()), "rho_at_jump": float(mid),
                              "tv_rho": float(abs(r["rho"][1:] - r["rho"][:-1]).sum())})
            tube[f"{model}/theta={theta}/nu={nu:g}"] = entry
    print(json.dumps({"experiments": "paper Sec. 5.1, 5.2 and 5.3",
                      "rotated_shear_wave": {"Ma": mas, "nu_ratio": table}, "shear_layer": layer,
                      "shocktube": {"grid": "800 x 1, fullway bounce-back walls at x = 0 and 799, 400 steps",
                                    "rho_l_rho_r": list(experiments.SHOCKTUBE_RHO), "runs": tube}}), flush=True)


def main():
    args = parse_args()
    if args.experiments:
        paper_experiments(args)
        return
    if args.precision_study:
        precision_study(args)
        return
    if args.config_sweep:
        config_sweep(args)
        return
    if args.vjp_only:
        import torch

        torch.cuda.set_device(0)
        stream = torch.cuda.Stream()
        print(json.dumps(vjp_sweep(torch.device("cuda", 0), stream, steps=args.vjp_steps)), flush=True)
        return
    if args.batch_only:
        import torch

        torch.cuda.set_device(0)
        stream = torch.cuda.Stream()
        tile = tuple(int(v) for v in args.batch_tile.split(",")) if args.batch_tile else None
        print(json.dumps(batch_sweep(torch.device("cuda", 0), stream, hbm_peak()[0], args.batch_steps, tile)),
              flush=True)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
