"""Launch-shape autotuning with a JSON cache.

`egpe_autotune` (C ABI) times every kernel of one solver attempt with each
candidate launch shape -- rows per block of the row (x) passes, TMA-fed or plain
tile loads of the column (y/z) passes -- and keeps the fastest in the handle.
This module runs it once per (device, build, precision, grid, preconditioner)
and stores the choices in a JSON file; later handles on the same device and
build apply the stored shapes with `egpe_set_tuning` instead of re-timing.
Instances of a handle that share a grid share one tuning.

The shapes change only how work is split over thread blocks, not the
arithmetic; the grouping of per-block partial sums (and so the last bits of a
reduction) can differ between shapes.
"""
from __future__ import annotations

import json
import os
from typing import Callable, Dict, List, Optional, Sequence

from . import build as _build
from . import egpe as E

DEFAULT_CACHE = os.environ.get("EGPE_TUNE_CACHE",
                               os.path.join(os.path.dirname(os.path.abspath(__file__)), "_tune_cache.json"))

ENGINE_NAMES = {0: "fp64", 1: "fp32"}


def engines_of(prec: int) -> List[int]:
    """Engines (0 FP64, 1 FP32) a handle of precision prec holds."""
    if prec == E.EGPE_FP64:
        return [0]
    if prec == E.EGPE_FP32:
        return [1]
    return [0, 1]


def cache_key(device: str, engine: int, n: Sequence[int], precond: int, digest: Optional[str] = None) -> str:
    d = digest if digest is not None else _build._digest()[:16]
    return f"{device}|{d}|{ENGINE_NAMES[engine]}|{n[0]}x{n[1]}x{n[2]}|pc{precond}"


def load_cache(path: str) -> Dict[str, list]:
    try:
        with open(path) as f:
            data = json.load(f)
        return data if isinstance(data, dict) else {}
    except (OSError, ValueError):
        return {}


def save_cache(path: str, data: Dict[str, list]) -> None:
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def tune_handle(h: int, grids: Sequence[Sequence[int]], prec: int, precond: int,
                make_psi: Callable[[int, int], object], device: str, reps: int = 5,
                cache_path: Optional[str] = DEFAULT_CACHE, digest: Optional[str] = None,
                tuner=None, setter=None) -> Dict[str, list]:
    """Tunes (or applies cached shapes to) every instance of handle h.

    grids[i] is instance i's (nx, ny, nz); make_psi(i, engine) returns a device
    field of that engine's precision for instance i (the state the timing runs
    from).  Returns {cache key: tuning entries} for the grids of the handle.
    tuner / setter default to egpe_autotune / egpe_set_tuning (replaceable for
    host-side tests)."""
    tuner = tuner or E.egpe_autotune
    setter = setter or E.egpe_set_tuning
    cache = load_cache(cache_path) if cache_path else {}
    used: Dict[str, list] = {}
    changed = False
    for eng in engines_of(prec):
        for i, n in enumerate(grids):
            key = cache_key(device, eng, n, precond, digest)
            if key not in used:
                if key in cache:
                    used[key] = cache[key]
                else:
                    used[key] = tuner(h, i, eng, make_psi(i, eng), precond, reps)
                    cache[key] = used[key]
                    changed = True
            setter(h, i, eng, used[key])
    if cache_path and changed:
        save_cache(cache_path, cache)
    return used
