"""Autotuner of the batched labelling launch.

Searches the launch shape of a batch object — pixels per strip (the tile of the
shared-memory union pass), threads per block, a cap on resident blocks per SM, and the
merge schedule (how many waves of blocks a frame's flatten tasks trail its strip tasks)
— by timing flic_label_batch with CUDA events on the caller's frames, applies the
fastest and persists it as JSON keyed by the device name and the workload's frame-shape
mix.  Results never depend on these settings (the GPU tests check many shapes), only the
speed does.
"""
from __future__ import annotations

import hashlib
import itertools
import json
import os
import time

SPACE = {
    "px_per_cta": [8192, 16384, 32768],
    "threads": [256, 512],
    "ctas_per_sm": [0, 1],
    "p3_delay": [2, 4, 8, 16],
}
DEFAULT = {"px_per_cta": 16384, "threads": 512, "ctas_per_sm": 0, "p3_delay": 8}


def configs(space: dict = SPACE):
    """Every combination of the search space, as dicts, default first."""
    keys = list(space)
    out = [dict(DEFAULT)]
    for vals in itertools.product(*(space[k] for k in keys)):
        c = dict(zip(keys, vals))
        if c != DEFAULT:
            out.append(c)
    return out


def signature(shapes, device_name: str) -> str:
    """Key of a workload: the device and the multiset of (rows, cols, skip) of its frames."""
    hist = {}
    for s in shapes:
        k = "x".join(str(int(v)) for v in s)
        hist[k] = hist.get(k, 0) + 1
    text = device_name + "|" + ",".join(f"{k}:{hist[k]}" for k in sorted(hist))
    return hashlib.sha256(text.encode()).hexdigest()[:20]


def cache_path() -> str:
    return os.environ.get("FLIC_AUTOTUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "flic", "autotune.json"))


def load(sig: str, path: str | None = None):
    path = path or cache_path()
    try:
        with open(path) as fh:
            return json.load(fh).get(sig)
    except (OSError, ValueError):
        return None


def save(sig: str, entry: dict, path: str | None = None) -> None:
    path = path or cache_path()
    os.makedirs(os.path.dirname(path), exist_ok=True)
    try:
        with open(path) as fh:
            data = json.load(fh)
    except (OSError, ValueError):
        data = {}
    data[sig] = entry
    tmp = path + f".tmp{os.getpid()}"
    with open(tmp, "w") as fh:
        json.dump(data, fh, indent=1, sort_keys=True)
    os.replace(tmp, path)


def apply(flic, batch, cfg: dict) -> None:
    flic.flic_batch_set_tuning(batch, cfg["px_per_cta"], cfg["threads"], 0, cfg["ctas_per_sm"])
    flic.flic_batch_set_schedule(batch, cfg["p3_delay"])


def tune_batch(flic, batch, args, shapes, stream=None, reps: int = 10, use_cache: bool = True,
               space: dict = SPACE) -> dict:
    """Time every configuration on these frames (args: flic.BatchArgs; shapes: (rows, cols,
    skip) per frame), apply the fastest to `batch` and return
    {"config", "ms", "searched", "from_cache", "seconds"}."""
    import torch
    t0 = time.perf_counter()
    sig = signature(shapes, torch.cuda.get_device_name())
    if use_cache:
        hit = load(sig)
        if hit:
            apply(flic, batch, hit["config"])
            return {**hit, "from_cache": True, "seconds": round(time.perf_counter() - t0, 3)}
    stream = stream or torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    best, results = None, []
    for cfg in configs(space):
        try:
            apply(flic, batch, cfg)
            for _ in range(2):
                flic.flic_label_batch(batch, args, stream)
            e0.record(stream)
            for _ in range(reps):
                flic.flic_label_batch(batch, args, stream)
            e1.record(stream)
            torch.cuda.synchronize()
        except flic.FlicError:
            continue  # the shape does not fit these frames
        ms = e0.elapsed_time(e1) / reps
        results.append((ms, cfg))
        if best is None or ms < best[0]:
            best = (ms, cfg)
    apply(flic, batch, best[1])
    entry = {"config": best[1], "ms": round(best[0], 4), "searched": len(results)}
    if use_cache:
        save(sig, entry)
    return {**entry, "from_cache": False, "seconds": round(time.perf_counter() - t0, 3)}
