"""Autotuner for the pair kernels' launch shapes.

The density and force kernels are persistent launches whose speed depends on
the shape of the work: how many candidates a warp's neighbourhood holds (the
stage size decides whether it fits or streams in chunks), how finely cells
are ordered inside (sub-cells), how many warps share an SM (block size and
the shared memory each warp's stage takes), and the order of the work queue
(cell order, or the costliest items first for uneven occupancy).  The tuner
times the real kernels on the caller's particles with CUDA events and keeps
the fastest shape:

  1. the binning choices (sub-cells per cell edge, queue order), each timed
     as density + force at the current launch shapes;
  2. with those fixed, the block size and stage size of each kernel,
     density and force measured separately (each kernel launches with its
     own block size).

Results are cached in a JSON file keyed by the device and a signature of the
workload (particle count, cell grid, occupancy, storage formats, Newton
steps), so repeated runs on the same kind of input skip the search.
"""
from __future__ import annotations

import json
import os
import statistics

SPACE = {
    "subcells": (1, 2),
    "item_order": (0, 1),
    "block_threads": (32, 64, 128),
    "stage_density": (64, 128, 256, 512),
    "stage_force": (96, 128, 160, 192),
}


def default_cache_path() -> str:
    return os.environ.get("SPH_TUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "sph_gb300_tuning.json"))


def signature(device: str, n: int, ncell: int, max_occupancy: int, prec: dict | None, newton_steps: int) -> str:
    """Cache key: device name and the workload features the best shape depends on
    (mean occupancy to one significant figure, the largest cell's occupancy as a
    power of two)."""
    mean_occ = n / max(ncell, 1)
    occ = float(f"{mean_occ:.1g}")
    peak = 1 << max(0, int(max_occupancy).bit_length() - 1)
    fmts = ",".join(f"{k}:{v}" for k, v in sorted((prec or {}).items()))
    return f"{device}|n={n}|ncell={ncell}|occ~{occ}|peak~{peak}|fmt={fmts}|newton={newton_steps}"


def load_cache(path: str) -> dict:
    try:
        with open(path) as f:
            data = json.load(f)
        return data if isinstance(data, dict) else {}
    except (OSError, ValueError):
        return {}


def save_cache(path: str, cache: dict) -> None:
    d = os.path.dirname(path)
    if d:
        os.makedirs(d, exist_ok=True)
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def _timer(torch, stream, reps: int):
    def run(fn):
        fn()                                   # warm-up (also the first launch's attribute setup)
        ts = []
        for _ in range(reps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        return statistics.median(ts)
    return run


def tune(s, cell_edge: float, prec: dict | None = None, newton_steps: int = 5, reps: int = 3,
         cache_path: str | None = None, use_cache: bool = True) -> dict:
    """Search the launch shapes for Sph context `s` on its current AoS and
    apply the best.  The AoS is not modified (no write-back).  Returns
    {"tuning": {...}, "ms": {"density": .., "force": ..}, "cached": bool,
    "trials": [...]}."""
    import torch
    from . import FIELDS_FORCE, SphError

    stream = s.stream
    timer = _timer(torch, stream, reps)
    cache_path = cache_path or default_cache_path()

    def prepare():
        s.bin_cells(cell_edge)
        s.aos_to_soa(FIELDS_FORCE, prec)

    with torch.cuda.stream(stream):
        prepare()
        st = s.stats()
        ncell = st["ncell"][0] * st["ncell"][1] * st["ncell"][2]
        key = signature(torch.cuda.get_device_name(), s.n, ncell, st["max_occupancy"], prec, newton_steps)
        cache = load_cache(cache_path) if use_cache else {}
        if key in cache:
            best = cache[key]["tuning"]
            s.set_tuning(**best)
            prepare()
            return {"tuning": best, "ms": cache[key]["ms"], "cached": True, "trials": [], "key": key}

        trials = []

        def measure(kind):
            if kind == "density":
                return timer(lambda: s.density(newton_steps))
            s.density(newton_steps)
            return timer(lambda: s.force())

        # 1. binning choices at the current launch shapes
        best_bin, best_t = None, float("inf")
        for sub in SPACE["subcells"]:
            for order in SPACE["item_order"]:
                s.set_tuning(subcells=sub, item_order=order, class_launches=0)
                prepare()
                t = measure("density") + measure("force")
                trials.append({"subcells": sub, "item_order": order, "ms": t})
                if t < best_t:
                    best_bin, best_t = (sub, order), t
        s.set_tuning(subcells=best_bin[0], item_order=best_bin[1], class_launches=0)
        prepare()

        # 2. block size and stage, per kernel (each kernel takes its own
        # block size)
        dens, forc = None, None
        for bt in SPACE["block_threads"]:
            for sd in SPACE["stage_density"]:
                try:
                    s.set_tuning(block_threads=bt, stage_density=sd)
                except SphError:
                    continue                         # does not fit in shared memory
                t = measure("density")
                trials.append({"block_threads": bt, "stage_density": sd, "density_ms": t})
                if dens is None or t < dens[0]:
                    dens = (t, bt, sd)
        for bt in SPACE["block_threads"]:
            for sf in SPACE["stage_force"]:
                try:
                    s.set_tuning(block_threads_force=bt, stage_force=sf)
                except SphError:
                    continue
                t = measure("force")
                trials.append({"block_threads_force": bt, "stage_force": sf, "force_ms": t})
                if forc is None or t < forc[0]:
                    forc = (t, bt, sf)
        best = {"block_threads": dens[1], "stage_density": dens[2], "block_threads_force": forc[1],
                "stage_force": forc[2], "subcells": best_bin[0], "item_order": best_bin[1], "class_launches": 0}
        ms = {"density": dens[0], "force": forc[0]}
        s.set_tuning(**best)
        prepare()
    if use_cache:
        cache[key] = {"tuning": best, "ms": ms}
        save_cache(cache_path, cache)
    return {"tuning": best, "ms": ms, "cached": False, "trials": trials, "key": key}
