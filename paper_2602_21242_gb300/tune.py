"""Autotuner for the launch shape of the step kernels.

For a lattice (or a batch) it times candidate shapes (threads bx x by, rows per
thread) with CUDA events on the object's own stream, keeps the fastest, and
caches it in a JSON file keyed by GPU name, kind, size class, storage form and
collision model, so the measurement runs once per configuration class.

Cache file: $OLBM_TUNE_CACHE, else ~/.cache/olbm/tune.json.
"""
from __future__ import annotations

import itertools
import json
import math
import os
import threading

import torch

from . import capi, flows

_lock = threading.Lock()

# (kind, bx, by, rows): kind 0 = column kernel; kind 1 = bulk-copy pipeline (shifted forms)
# with bx = CTAs per SM (0 = one CTA per tile); kind 2 = two steps a launch
LATTICE_CANDIDATES = [(0, bx, by, rows) for (bx, by), rows in itertools.product(
    [(32, 4), (32, 8), (64, 2), (64, 4), (128, 1), (128, 2), (128, 4), (256, 1), (256, 2)], [4, 8, 16, 32])]
PIPELINE_CANDIDATES = [(1, ctas, 1, rows) for ctas in (0, 2, 64) for rows in (4, 8, 16, 32, 64)]
# kind 2: two steps a launch (shifted forms), one CTA per tile of `rows` rows
TWO_STEP_CANDIDATES = [(2, 0, 1, rows) for rows in (8, 16, 32, 64)]
BATCH_CANDIDATES = [(0, bx, by, rows) for (bx, by), rows in itertools.product(
    [(32, 4), (32, 8), (64, 2), (64, 4), (128, 2)], [2, 4, 8, 16])]
# kind 1: the pipeline with bx consumer threads (0 = default) on tiles of 2 bx columns x rows
# (shifted forms; widths a form does not offer are skipped)
BATCH_PIPELINE_CANDIDATES = [(1, nc, 1, rows) for nc in (0, 32, 64, 128) for rows in (16, 32, 64)]
# kind 2: two steps a launch (graph mode) on tiles of the default width
BATCH_TWO_STEP_CANDIDATES = [(2, 0, 1, rows) for rows in (8, 16, 32, 64)]


def cache_path() -> str:
    return os.environ.get("OLBM_TUNE_CACHE") or os.path.join(os.path.expanduser("~"), ".cache", "olbm", "tune.json")


def _load_cache(path: str) -> dict:
    try:
        with open(path) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


def _store(path: str, key: str, value) -> None:
    with _lock:
        data = _load_cache(path)
        data[key] = value
        os.makedirs(os.path.dirname(path), exist_ok=True)
        tmp = f"{path}.tmp{os.getpid()}"
        with open(tmp, "w") as fh:
            json.dump(data, fh, indent=1, sort_keys=True)
        os.replace(tmp, path)


def _key(kind: str, nodes: int, prec: int, model: int, extra: str = "") -> str:
    gpu = torch.cuda.get_device_name(torch.cuda.current_device()).replace(" ", "_")
    size_class = int(round(math.log2(max(nodes, 1))))
    return f"{gpu}|{kind}|2^{size_class}{extra}|prec{prec}|model{model}"


def _timing_fields(nx: int, ny: int):
    """(rho, ux, uy) host arrays the candidates are timed on: the advected shear wave of the
    bandwidth benchmark (u_x = 0.1, u_y = 0.01 sin(2 pi x / nx)). A fluid at rest would time
    another code path of the FP64 form, whose products take zero operands on a slower path."""
    return flows.shear_wave(nx, ny, U=0.1, amp=0.01)


def _time(step, sync, stream, steps: int) -> float:
    step(steps)  # warm-up with the same count (a batch captures its graph here)
    sync()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    step(steps)
    e1.record(stream)
    sync()
    return e0.elapsed_time(e1) / steps


def tune_lattice(lat, candidates=None, steps: int = 10, use_cache: bool = True, path: str | None = None):
    """Pick and apply the fastest launch (kind, bx, by, rows) for `lat` (a Lattice). Timing
    runs on a temporary lattice of the same size, storage and model started from the
    advected shear wave of `_timing_fields`, so `lat`'s state is untouched. Candidates may
    be given as (bx, by, rows) for kind 0 or as (kind, bx, by, rows). Returns ((kind, bx, by, rows), ms_per_step or None if cached)."""
    from .lattice import Lattice

    path = path or cache_path()
    key = _key("lattice", lat.nx * lat.ny, lat.prec, lat.model, f"|nx={lat.nx}")
    if use_cache:
        hit = _load_cache(path).get(key)
        if hit:
            capi.lbm_set_launch_ex(lat.ctx, *hit["shape"])
            return tuple(hit["shape"]), None
    if candidates is None:
        candidates = list(LATTICE_CANDIDATES)
        if lat.prec != capi.LBM_F64_DF:  # shapes a form does not take are skipped below
            candidates += PIPELINE_CANDIDATES + TWO_STEP_CANDIDATES
    best = None
    with Lattice(lat.nx, lat.ny, lat.theta, lat.tau, lat.model, lat.prec, device=lat.device,
                 stream=lat.stream) as tmp:
        tmp.init(*(torch.from_numpy(a).to(lat.device) for a in _timing_fields(lat.nx, lat.ny)))
        tmp.set_diagnostics_interval(1)
        for shape in candidates:
            shape = tuple(shape) if len(shape) == 4 else (0,) + tuple(shape)
            try:
                capi.lbm_set_launch_ex(tmp.ctx, *shape)
            except capi.LBMError:
                continue
            ms = _time(tmp.step, tmp.sync, tmp.stream, steps)
            if best is None or ms < best[1]:
                best = (shape, ms)
    capi.lbm_set_launch_ex(lat.ctx, *best[0])
    _store(path, key, {"shape": list(best[0]), "ms_per_step": best[1]})
    return tuple(best[0]), best[1]


def tune_batch(batch, candidates=None, steps: int = 10, use_cache: bool = True, path: str | None = None):
    """Pick and apply the fastest tile shape for `batch` (a Batch). The timing steps the
    batch itself from the advected shear wave of `_timing_fields`: call it before Batch.init.
    Candidates are (kind, bx, by, rows) or (bx, by, rows) for kind 0; the default set
    adds the pipeline shapes for the shifted forms. Returns ((kind, bx, by, rows),
    ms_per_step or None if cached)."""
    path = path or cache_path()
    key = _key("batch", batch.total_nodes, batch.prec, batch.model, f"|n{batch.n}|k")
    if use_cache:
        hit = _load_cache(path).get(key)
        if hit:
            batch.set_launch(*hit["shape"])
            return tuple(hit["shape"]), None
    rho, ux, uy = zip(*(_timing_fields(nx, ny) for nx, ny in zip(batch.nx, batch.ny)))
    best = None
    if candidates is None:
        candidates = BATCH_CANDIDATES + (BATCH_PIPELINE_CANDIDATES + BATCH_TWO_STEP_CANDIDATES
                                         if batch.prec != capi.LBM_F64 else [])
    for shape in candidates:
        shape = tuple(shape) if len(shape) == 4 else (0,) + tuple(shape)
        try:
            batch.set_launch(*shape)
        except capi.LBMError:
            continue
        batch.init(rho, ux, uy)
        ms = _time(batch.step, batch.sync, batch.stream, steps)
        if best is None or ms < best[1]:
            best = (shape, ms)
    batch.set_launch(*best[0])
    batch.init(rho, ux, uy)
    _store(path, key, {"shape": list(best[0]), "ms_per_step": best[1]})
    return tuple(best[0]), best[1]
