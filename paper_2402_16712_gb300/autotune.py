"""Autotuner of the pair kernel's launch.

The planner in the library picks warps per CTA, CTAs per SM, k per CTA and the
width of the first selection bracket from the shape alone.  This module times
alternatives on the caller's own call and keeps the fastest per (GPU, dtype,
call kind, power-of-two buckets of n, m and the number of lambdas) in a JSON
cache; a later call of the same bucket applies the cached tuning with
l1line.set_tuning.  Tunings never change results (every decision of the
selection is exact), only the time.

Cache file: $L1LINE_AUTOTUNE_CACHE, else ~/.cache/l1line/autotune.json.
"""
from __future__ import annotations

import json
import os
import statistics
import threading
from typing import Callable, Optional

from . import l1line

CACHE_ENV = "L1LINE_AUTOTUNE_CACHE"
_lock = threading.Lock()


def cache_path() -> str:
    return os.environ.get(CACHE_ENV) or os.path.join(os.path.expanduser("~"), ".cache", "l1line",
                                                     "autotune.json")


def bucket(x: int) -> int:
    """The power of two at or above x."""
    x = int(x)
    return 1 if x <= 1 else 1 << (x - 1).bit_length()


def _gpu_name() -> str:
    import torch
    return torch.cuda.get_device_name() if torch.cuda.is_available() else "cpu"


def key(dtype, n: int, m: int, nl: int, kind: str = "fit", gpu: Optional[str] = None) -> str:
    dt = "f32" if l1line._dt(dtype) == l1line.DTYPE_F32 else "f64"
    return (f"{gpu if gpu is not None else _gpu_name()}|{dt}|{kind}|n{bucket(n)}|m{bucket(m)}"
            f"|l{bucket(nl)}")


def load_cache(path: Optional[str] = None) -> dict:
    p = path or cache_path()
    try:
        with open(p) as f:
            d = json.load(f)
        return d if isinstance(d, dict) else {}
    except (OSError, ValueError):
        return {}


def store(k: str, tuning: dict, ms: float, path: Optional[str] = None) -> None:
    p = path or cache_path()
    with _lock:
        d = load_cache(p)
        d[k] = {"tuning": tuning, "ms": ms}
        os.makedirs(os.path.dirname(os.path.abspath(p)), exist_ok=True)
        tmp = f"{p}.tmp{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(d, f, indent=1, sort_keys=True)
        os.replace(tmp, p)


def candidates(base: dict, kchunk: bool = True, classes: bool = False):
    """Coordinate sweeps around the planner's plan `base` (l1line.plan):
    k per CTA (unless kchunk is False), the number of size classes of a
    batched call (if classes), the bracket width, the other placement of
    x_ijhat, then warps x CTAs per SM."""
    kc = max(1, base["kchunk"])
    for div in ((2, 3, 4, 6) if kchunk else ()):
        yield {"kchunk": max(1, -(-kc // div))}
    for k in ((1, 2, 3) if classes else ()):
        yield {"batch_classes": k}
    for d0 in (3, 4, 5, 7, 8, 10):
        yield {"d0": d0}
    # after the bracket width: which placement is faster depends on it
    for c in (1, 2):
        if c != base.get("column"):
            yield {"column": c}
    for warps, ctas in ((16, 2), (8, 3), (16, 1), (8, 2), (12, 1), (6, 3), (4, 3), (8, 1)):
        yield {"warps": warps, "ctas_per_sm": ctas}


def _time(run: Callable[[], None], reps: int, flush) -> float:
    import torch
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(reps)]
    run()  # warm-up (first launch of a configuration)
    for a, b in ev:
        if flush is not None:
            flush.fill_(3)
        a.record()
        run()
        b.record()
    torch.cuda.synchronize()
    return statistics.median(a.elapsed_time(b) for a, b in ev)


def tune(run: Callable[[], None], dtype, n: int, m: int, nj: Optional[int] = None, reps: int = 3,
         flush=None, log=None, kchunk: bool = True, classes: bool = False):
    """Time `run` (a call on the current stream) under the planner's plan and
    the candidate tunings; returns (best tuning dict, its ms, table).  Each
    sweep keeps the best value found so far and varies one knob."""
    l1line.set_tuning(None)
    base = l1line.plan(dtype, n, m, nj)
    best, best_ms = {}, _time(run, reps, flush)
    table = [({}, best_ms)]
    for cand in candidates(base, kchunk, classes):
        t = dict(best)
        t.update(cand)
        try:
            l1line.set_tuning(t)
            l1line.plan(dtype, n, m, nj)  # raises if the lists do not fit
            ms = _time(run, reps, flush)
        except l1line.L1LineError:
            continue
        finally:
            l1line.set_tuning(None)
        table.append((t, ms))
        if log:
            log(f"  {t}: {ms:.3f} ms")
        if ms < best_ms * 0.995:
            best, best_ms = t, ms
    return best, best_ms, table


def apply(dtype, n: int, m: int, nl: int = 1, kind: str = "fit", run=None, nj=None, flush=None,
          path: Optional[str] = None, log=None) -> dict:
    """Set this thread's tuning for a call of this shape: from the cache, or
    (when `run` is given and the bucket is not cached) by tuning on `run` and
    storing the result.  Returns the tuning applied ({} = the planner)."""
    k = key(dtype, n, m, nl, kind)
    hit = load_cache(path).get(k)
    if hit is None and run is not None:
        # a batched call gives every CTA a whole column: k per CTA is not a
        # knob, the number of size classes is
        t, ms, _ = tune(run, dtype, n, m, nj=nj, flush=flush, log=log, kchunk=kind != "batch",
                        classes=kind == "batch")
        store(k, t, ms, path)
        hit = {"tuning": t}
    t = hit["tuning"] if hit else {}
    l1line.set_tuning(t or None)
    return t
