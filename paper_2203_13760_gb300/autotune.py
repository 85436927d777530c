"""Autotuner of libjf launch variants (tile shape, z chunk, batch tile).

For a Solver or a Batch, ``tune`` times every compiled launch variant
(jf_variant_info / jf_set_variant) with CUDA events on the current stream,
keeps the fastest and records it in a JSON cache keyed by the device name and
the configuration (kind, dimensionality, physics, dtype, size class), so that
later handles of the same kind pick it without timing.  Timing uses copies of
the caller's fields; the caller's data is not modified.

  from paper_2203_13760_gb300 import autotune
  best = autotune.tune(solver, U)            # or autotune.tune(batch, fields)
  autotune.apply(solver)                     # cached choice, no timing
"""
from __future__ import annotations

import json
import math
import os
import threading

_LOCK = threading.Lock()
DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "jf_autotune.json")


def cache_path() -> str:
    return os.environ.get("JF_AUTOTUNE_CACHE", DEFAULT_CACHE)


def _load(path):
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(path, data):
    os.makedirs(os.path.dirname(path) or ".", exist_ok=True)
    tmp = f"{path}.tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def _size_class(cells: int) -> int:
    """Power-of-two bucket of the cell count (variants rank alike within one)."""
    return int(round(math.log2(max(cells, 1))))


def config_key(obj) -> str:
    import torch
    from . import jf
    dev = torch.cuda.get_device_name(torch.cuda.current_device()).replace(" ", "_")
    sch = obj.scheme
    dtype = "f32" if sch.dtype == jf.JF_F32 else "f64"
    visc = int(bool(sch.viscous or sch.heat) and obj.gas.mu > 0)
    if isinstance(obj, jf.Batch):
        g0 = obj.grids[0]
        dim = 3 if g0.nz > 1 else (2 if g0.ny > 1 else 1)
        cells = sum(g.nx * g.ny * g.nz for g in obj.grids)
        kind = f"batch{obj.nsim}"
    else:
        g = obj.grid
        dim = 3 if g.nz > 1 else (2 if g.ny > 1 else 1)
        cells = g.nx * g.ny * g.nz
        kind = "single"
    return f"{dev}|{kind}|{dim}d|visc{visc}|{dtype}|2^{_size_class(cells)}"


def _time_variant(obj, fields, steps: int, reps: int) -> float:
    import torch
    from . import jf
    stream = torch.cuda.current_stream()
    best = float("inf")
    if isinstance(obj, jf.Batch):
        work = [f.clone() for f in fields]
        obj.step(work, steps)  # capture
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            obj.step(work, steps)
            e1.record(stream)
            torch.cuda.synchronize()
            best = min(best, e0.elapsed_time(e1))
    else:
        work = fields.clone()
        dt = obj.compute_dt(work)
        obj.run(work, steps, dt)  # capture
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            obj.run(work, steps, dt)
            e1.record(stream)
            torch.cuda.synchronize()
            best = min(best, e0.elapsed_time(e1))
    obj.sync()
    return best


def tune(obj, fields, steps: int = 3, reps: int = 3, path: str | None = None) -> dict:
    """Time every variant of ``obj`` (a jf.Solver with its field, or a
    jf.Batch with its list of fields), select the fastest and cache it.
    Returns {"key", "variant", "description", "ms": {variant: ms}}."""
    path = path or cache_path()
    names = obj.variants()
    times = {}
    for v in range(len(names)):
        obj.set_variant(v)
        times[v] = _time_variant(obj, fields, steps, reps)
    best = min(times, key=times.get)
    obj.set_variant(best)
    key = config_key(obj)
    rec = {"variant": best, "description": names[best], "ms": {names[v]: t for v, t in times.items()},
           "steps": steps}
    with _LOCK:
        data = _load(path)
        data[key] = rec
        _store(path, data)
    return dict(rec, key=key)


def apply(obj, path: str | None = None):
    """Select the cached variant for ``obj``'s configuration, if any.
    Returns the variant index used, or None (default kept)."""
    rec = _load(path or cache_path()).get(config_key(obj))
    if not rec:
        return None
    names = obj.variants()
    v = rec.get("variant")
    if v is None or v >= len(names) or names[v] != rec.get("description"):
        return None  # stale entry (the compiled variant table changed)
    obj.set_variant(v)
    return v
