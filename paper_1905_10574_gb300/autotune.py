"""Tile-size autotuner for batched solves.

The tile size t trades the length of the chain of diagonal-tile solves and the
per-update overhead against the work per tile; the best t depends on the size
mix of a batch and on the GPU.  ``tune_batch`` times ``sylv_batch_execute`` on
the caller's batch (CUDA events, median of a few runs, right-hand sides refilled
from a saved copy between runs) for candidate tile sizes, first one size for
all equations, then per size bucket (max(m, n) <= 64, 128, 256, 512, larger) with
the other buckets held at their best, and returns a tile per equation.  Results
are cached per GPU name, precision and size-mix signature in a JSON file
(``$XDG_CACHE_HOME/sylv_gb300/autotune.json``, else ``~/.cache/...``).
"""
from __future__ import annotations

import json
import os

CANDIDATES = (16, 24, 32, 48, 64)
BUCKETS = (64, 128, 256, 512, 1 << 30)


def _cache_path() -> str:
    base = os.environ.get("XDG_CACHE_HOME") or os.path.join(os.path.expanduser("~"), ".cache")
    return os.path.join(base, "sylv_gb300", "autotune.json")


def bucket_of(m: int, n: int) -> int:
    mx = max(m, n)
    for i, b in enumerate(BUCKETS):
        if mx <= b:
            return i
    return len(BUCKETS) - 1


def signature(shapes) -> str:
    counts = [0] * len(BUCKETS)
    for m, n in shapes:
        counts[bucket_of(m, n)] += 1
    return "b" + "-".join(str(c) for c in counts)


def _load_cache() -> dict:
    try:
        with open(_cache_path()) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _save_cache(c: dict) -> None:
    path = _cache_path()
    try:
        os.makedirs(os.path.dirname(path), exist_ok=True)
        tmp = path + f".tmp{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(c, f, indent=1)
        os.replace(tmp, path)
    except OSError:
        pass


def _time_plan(sy, torch, shapes, As, Bs, Cs, C0s, tiles, reps=3, precision="fp64", tol=0.0) -> float:
    stream = torch.cuda.current_stream()
    o = sy.make_opts(stream=stream.cuda_stream, precision=precision, tol=tol)
    plan = sy.sylv_batch_create([m for m, _ in shapes], [n for _, n in shapes], [a.data_ptr() for a in As],
                                [a.stride(1) for a in As], [b.data_ptr() for b in Bs], [b.stride(1) for b in Bs],
                                [c.data_ptr() for c in Cs], [c.stride(1) for c in Cs], o, tiles=tiles)
    ts = []
    try:
        for r in range(reps + 1):
            for c, c0 in zip(Cs, C0s):
                c.copy_(c0)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            rc = sy.sylv_batch_execute(plan, stream.cuda_stream)
            e1.record(stream)
            torch.cuda.synchronize()
            if rc:
                raise sy.SylvError(rc, "sylv_batch_execute")
            if r:
                ts.append(e0.elapsed_time(e1))
    finally:
        sy.sylv_batch_destroy(plan)
    ts.sort()
    return ts[len(ts) // 2]


def tune_batch(As, Bs, Cs, *, precision="fp64", tol=0.0, use_cache=True, reps=3, log=None):
    """Tile size per equation for this batch (lists of column-major float64 CUDA
    tensors; Cs are overwritten during tuning and restored at the end), tuned for the
    given precision ("fp64" or "fp32_refine" at stop tolerance tol): the binary32
    correction solves favour other tiles than the FP64 solve."""
    import torch

    from . import sylv as sy
    shapes = [(int(c.shape[0]), int(c.shape[1])) for c in Cs]
    key = f"{torch.cuda.get_device_name()}|{precision}|{tol!r}|{signature(shapes)}"
    cache = _load_cache() if use_cache else {}
    if key in cache:
        per_bucket = cache[key]["per_bucket"]
        return [per_bucket[bucket_of(m, n)] for m, n in shapes]
    C0s = [c.clone() for c in Cs]
    best_t, best_ms = None, float("inf")
    for t in CANDIDATES:
        ms = _time_plan(sy, torch, shapes, As, Bs, Cs, C0s, [t] * len(shapes), reps, precision, tol)
        if log:
            log(f"all t={t}: {ms:.2f} ms")
        if ms < best_ms:
            best_t, best_ms = t, ms
    per_bucket = [best_t] * len(BUCKETS)
    present = sorted({bucket_of(m, n) for m, n in shapes})
    for b in present:
        for t in CANDIDATES:
            if t == per_bucket[b]:
                continue
            trial = list(per_bucket)
            trial[b] = t
            ms = _time_plan(sy, torch, shapes, As, Bs, Cs, C0s, [trial[bucket_of(m, n)] for m, n in shapes], reps,
                            precision, tol)
            if log:
                log(f"bucket {b} t={t}: {ms:.2f} ms")
            if ms < best_ms * 0.98:
                per_bucket, best_ms = trial, ms
    for c, c0 in zip(Cs, C0s):
        c.copy_(c0)
    if use_cache:
        cache = _load_cache()
        cache[key] = {"per_bucket": per_bucket, "ms": best_ms}
        _save_cache(cache)
    return [per_bucket[bucket_of(m, n)] for m, n in shapes]
