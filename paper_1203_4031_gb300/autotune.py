"""Autotuner of the batched solves (gbf_batch_solve): picks, per arithmetic
path, the number of concurrent workers (handle + stream each: how many
problems' kernels overlap on the GPU) and, per size bucket of n, the LU
panel / trailing-update width fpm(43) (the k of the tensor-core trailing
updates and the size of the inverted diagonal blocks), by timing the real
batched solve on a sample of the workload, and persists the choice as JSON.

    from paper_1203_4031_gb300 import autotune
    table = autotune.tune(sample_problems)      # list of DeviceProblem
    autotune.save(table)                        # tuning/batch_<gpu>.json
    rc, outs = autotune.batch_solve(problems)   # uses the saved table

Timing only; every solve runs the library's kernels.  Results of a solve do
not depend on the worker count; they depend on fpm(43) only through the
rounding of the FP32 / FP64-class products.
"""
from __future__ import annotations

import json
import os
import time

from . import DeviceProblem, batch_solve as _batch_solve, lib  # noqa: F401

HERE = os.path.dirname(os.path.abspath(__file__))
TUNING_DIR = os.path.join(HERE, "tuning")
WORKERS = (4, 6, 8, 12, 16)
WIDTHS = (0, 16)          # fpm(43): 0 = default 32 columns, or 16
BUCKETS = (128, 256, 512, 1024, 1 << 30)   # upper bounds of n per bucket
DEFAULT = {"workers": {"0": 8, "1": 8}, "width": {}}


def gpu_name():
    import torch

    return torch.cuda.get_device_name().replace(" ", "_")


def path_for(name=None):
    return os.path.join(TUNING_DIR, f"batch_{name or gpu_name()}.json")


def bucket_of(n):
    for b in BUCKETS:
        if n <= b:
            return str(b)
    return str(BUCKETS[-1])


def _timed(problems, nworkers):
    import torch

    torch.cuda.synchronize()
    t0 = time.perf_counter()
    rc, outs = _batch_solve(problems, nworkers=nworkers)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    if rc != 0 or any(r.info != 0 for r in outs):
        return float("inf"), 0
    return dt, sum(r.M for r in outs)


def _with_width(problems, width):
    for q in problems:
        q.p.fpm[42] = int(width)
    return problems


def tune(problems, workers=WORKERS, widths=WIDTHS, reps=2):
    """problems: DeviceProblem list (one arithmetic path per call, the fpm of
    the first problem decides it).  Returns the table entry for that path:
    {"workers": w, "width": {bucket: fpm43}, "timings": {...}}."""
    prec = str(int(problems[0].p.fpm[41]))
    saved = [int(q.p.fpm[42]) for q in problems]
    _batch_solve(problems[: min(len(problems), 4)], nworkers=4)   # warm-up: workspaces, modules
    timings = {}
    # 1. worker count with the default width
    _with_width(problems, 0)
    best_w, best_t = workers[0], float("inf")
    for w in workers:
        t = min(_timed(problems, w)[0] for _ in range(reps))
        timings[f"workers={w}"] = t
        if t < best_t:
            best_w, best_t = w, t
    # 2. per size bucket, the trailing-update width at that worker count
    width = {}
    by_bucket = {}
    for q in problems:
        by_bucket.setdefault(bucket_of(q.p.n), []).append(q)
    for b, qs in sorted(by_bucket.items(), key=lambda kv: int(kv[0])):
        best_k, best_tk = 0, float("inf")
        for k in widths:
            _with_width(qs, k)
            t = min(_timed(qs, best_w)[0] for _ in range(reps))
            timings[f"bucket={b},width={k}"] = t
            if t < best_tk:
                best_k, best_tk = k, t
        width[b] = best_k
        _with_width(qs, 0)
    for q, s in zip(problems, saved):
        q.p.fpm[42] = s
    return {"prec": prec, "workers": best_w, "width": width, "timings": timings}


def merge(entries, name=None):
    table = {"gpu": name or gpu_name(), "workers": {}, "width": {}, "timings": {}}
    for e in entries:
        table["workers"][e["prec"]] = e["workers"]
        table["width"][e["prec"]] = e["width"]
        table["timings"][e["prec"]] = e["timings"]
    return table


def save(table, path=None):
    path = path or path_for(table.get("gpu"))
    os.makedirs(os.path.dirname(path), exist_ok=True)
    with open(path, "w") as f:
        json.dump(table, f, indent=1, sort_keys=True)
    return path


def load(path=None):
    try:
        with open(path or path_for()) as f:
            return json.load(f)
    except (OSError, ValueError):
        return DEFAULT


def apply(problems, table=None):
    """Sets fpm(43) of each problem from the table (its path and size
    bucket) and returns the worker count for the batch."""
    table = table or load()
    prec = str(int(problems[0].p.fpm[41])) if problems else "0"
    widths = table.get("width", {}).get(prec, {})
    for q in problems:
        q.p.fpm[42] = int(widths.get(bucket_of(q.p.n), 0))
    return int(table.get("workers", {}).get(prec, 8))


def batch_solve(problems, table=None):
    """gbf_batch_solve with the tuned worker count and widths."""
    return _batch_solve(problems, nworkers=apply(problems, table))
