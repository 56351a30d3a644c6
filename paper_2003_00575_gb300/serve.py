"""Serving driver: simulated sensors with Poisson arrivals feeding the libflic server.

Four sensors (16x1800, 32x1024, 64x2048, 128x2048) emit frames at a Poisson rate; half
of the frames are range images, half raw xyz clouds of 30k-260k points that need the
projection.  The aggregate rate is swept over log-spaced steps (default 100 -> 20,000
frames/s over 60 s).  The server (flic_server_* in libflic, a native dispatcher thread)
admits frames into device-memory slots as they free up, batches whatever has arrived into
one labelling launch and overlaps batches on two streams; this driver only submits at the
scheduled times and reads the completion records.  Per step it reports p50/p99 latency
(submission to labels in host memory), achieved frames/s and admitted/rejected counts.

    python -m paper_2003_00575_gb300.serve --seconds 60 --steps 12
"""
from __future__ import annotations

import argparse
import gc
import json
import math
import time

import numpy as np


# ----------------------------------------------------------------------- host logic

def rate_steps(lo: float, hi: float, n: int) -> list[float]:
    """n aggregate rates spaced evenly in log scale from lo to hi (frames/s)."""
    if n == 1:
        return [float(hi)]
    return [float(lo * (hi / lo) ** (i / (n - 1))) for i in range(n)]


def poisson_schedule(rate: float, seconds: float, nsensors: int, seed: int):
    """Arrivals of nsensors independent Poisson sensors sharing the aggregate rate:
    a time-sorted list of (t, sensor, kind), kind 0 = range image, 1 = cloud (alternating
    per sensor, so half of each sensor's frames are clouds)."""
    g = np.random.Generator(np.random.PCG64(seed))
    out = []
    per = rate / nsensors
    for s in range(nsensors):
        t, k = 0.0, 0
        while True:
            t += g.exponential(1.0 / per)
            if t >= seconds:
                break
            out.append((t, s, k & 1))
            k += 1
    out.sort()
    return out


def summarize(records, t0: float, t1: float) -> dict:
    """Latency percentiles (ms) and throughput of completion records (dicts or structs
    with t_submit, t_launch, t_done, batch_size, status).  The latency splits into the wait
    in the admission queue (submission to the launch of the frame's batch) and the service
    time (the batch's launch to its results in host memory: enqueueing, copies, kernels)."""
    if not records:
        return {"completed": 0}
    lat = np.array([(r.t_done - r.t_submit) * 1e3 for r in records])
    wait = np.array([(r.t_launch - r.t_submit) * 1e3 for r in records])
    svc = np.array([(r.t_done - r.t_launch) * 1e3 for r in records])
    bs = np.array([r.batch_size for r in records])
    ok = sum(1 for r in records if r.status == 0)
    span = max(t1 - t0, 1e-9)

    def pc(x, q):
        return round(float(np.percentile(x, q)), 3)
    return {"completed": len(records), "ok": ok, "frames_per_s": round(len(records) / span, 1),
            "latency_ms_p50": pc(lat, 50), "latency_ms_p99": pc(lat, 99),
            "latency_ms_max": round(float(lat.max()), 3),
            "queue_ms_p50": pc(wait, 50), "queue_ms_p99": pc(wait, 99),
            "service_ms_p50": pc(svc, 50), "service_ms_p99": pc(svc, 99),
            "mean_batch": round(float(bs.mean()), 2)}


# ----------------------------------------------------------------------- GPU side

class FramePool:
    """Pinned host copies of a few pre-generated frames per sensor and kind, and output
    buffers used round-robin."""

    def __init__(self, sensors, per_kind: int = 4, outputs: int = 256, seed: int = 1000):
        import torch
        from . import synth
        self.inputs = []   # [sensor][kind] -> list of pinned tensors
        self.outputs = []  # [sensor][kind] -> list of pinned int32 tensors
        self.max_points = []
        for si, s in enumerate(sensors):
            ins, outs, mp = [[], []], [[], []], 0
            for j in range(per_kind):
                f = synth.c5_frame(s, seed + 100 * si + 2 * j, as_cloud=False)
                ins[0].append(torch.from_numpy(f.range.reshape(-1)).pin_memory())
                c = synth.c5_frame(s, seed + 100 * si + 2 * j + 1, as_cloud=True)
                ins[1].append(torch.from_numpy(c.xyz.reshape(-1)).pin_memory())
                mp = max(mp, c.xyz.shape[0])
            npix = s.rows * s.cols
            outs[0] = [torch.empty(npix, dtype=torch.int32).pin_memory() for _ in range(outputs)]
            outs[1] = [torch.empty(260_001, dtype=torch.int32).pin_memory() for _ in range(outputs)]
            self.inputs.append(ins)
            self.outputs.append(outs)
            self.max_points.append(260_001)
        self.k = 0

    def pick(self, sensor: int, kind: int):
        ins = self.inputs[sensor][kind]
        outs = self.outputs[sensor][kind]
        self.k += 1
        x = ins[self.k % len(ins)]
        n = x.numel() // 3 if kind == 1 else x.numel()
        return x, outs[self.k % len(outs)][:n]


def run_step(flic, srv, pool: FramePool, rate: float, seconds: float, seed: int) -> dict:
    """Submit a Poisson schedule at its times and summarize the completions.  The garbage
    collector is off while the schedule is paced: a full collection over the growing list
    of completion records stalls this thread for tens of milliseconds, and the frames due
    meanwhile would then arrive as one burst that the schedule never had."""
    sched = poisson_schedule(rate, seconds, len(pool.inputs), seed)
    records, rejected = [], 0
    gc.collect()
    gc.disable()
    try:
        t_start = time.perf_counter()
        c0 = flic.flic_server_clock()
        late = np.empty(len(sched))  # how far behind its schedule each submission was
        for i, (t, s, kind) in enumerate(sched):
            while True:
                now = time.perf_counter() - t_start
                if now >= t:
                    break
            late[i] = now - t
            x, y = pool.pick(s, kind)
            if flic.flic_server_submit(srv, s, kind, x, y, i) != flic.FLIC_OK:
                rejected += 1
            if i % 64 == 0:
                records += flic.flic_server_poll(srv)
        flic.flic_server_drain(srv, 120.0)
        records += flic.flic_server_poll(srv)
    finally:
        gc.enable()
    c1 = max([r.t_done for r in records], default=c0)
    out = summarize(records, c0, c1)
    out.update({"rate_offered": round(rate, 1), "submitted": len(sched), "rejected": rejected})
    if len(sched):
        # the load generator's own delays: a submission made late by a pause of this
        # thread arrives in a burst with the ones due during the pause
        out.update({"submit_late_ms_p99": round(float(np.percentile(late, 99)) * 1e3, 3),
                    "submit_late_ms_max": round(float(late.max()) * 1e3, 3),
                    "submit_late_over_1ms": int((late > 1e-3).sum())})
    return out


def main(argv=None):
    p = argparse.ArgumentParser()
    p.add_argument("--seconds", type=float, default=60.0, help="total over all steps")
    p.add_argument("--steps", type=int, default=12)
    p.add_argument("--lo", type=float, default=100.0)
    p.add_argument("--hi", type=float, default=20000.0)
    p.add_argument("--streams", type=int, default=2)
    p.add_argument("--max-batch", type=int, default=256)
    p.add_argument("--mem-gb", type=float, default=4.0)
    p.add_argument("--only-top", type=int, default=0,
                   help="run only the last N rate steps (each seconds/steps long)")
    args = p.parse_args(argv)
    import torch
    from . import flic, synth
    torch.cuda.set_device(0)
    sensors = synth.c5_sensors()
    handles = [flic.flic_create(s.rows, s.cols, s.elevation, s.az_step, 0.5, 3) for s in sensors]
    pool = FramePool(sensors)
    srv = flic.flic_server_create(handles, pool.max_points, nstreams=args.streams,
                                  max_batch=args.max_batch, mem_budget=int(args.mem_gb * 2**30))
    warm = run_step(flic, srv, pool, 200.0, 0.5, 999)  # first launches capture graphs
    steps = []
    rates = rate_steps(args.lo, args.hi, args.steps)
    for i, rate in enumerate(rates):
        if args.only_top and i < len(rates) - args.only_top:
            continue
        r = run_step(flic, srv, pool, rate, args.seconds / args.steps, 1000 + i)
        steps.append(r)
        print(json.dumps(r), flush=True)
    print(json.dumps({"server": flic.flic_server_stats(srv), "warmup": warm}), flush=True)
    srv.close()
    for h in handles:
        h.close()
    return steps


if __name__ == "__main__":
    main()
