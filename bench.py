#!/usr/bin/env python
"""Benchmark of the FLIC hot path (arXiv 2003.00575) on GB300.

Workload (the batched configuration the throughput metric is quoted on): 256 synthetic
frames of uneven shape drawn from {16x1800, 32x1024, 64x2048, 128x2048}, each with its
own elevation table, delta in 0.3-0.6 m and skip S in 1..5, labelled by one persistent
kernel launch replayed from a CUDA graph.  One step = one pass of the labelling path
(neighbour test + union-find CCL + flatten) over the whole batch.

Reported (one JSON line on rank 0):
  value        batched labelled Mpixel/s over all ranks, inputs resident in HBM
  e2e          the same through the host-buffer batch call (flic_label_batch_host) on
               pinned packed buffers: per step every range image goes up and every label
               comes back; 4 groups of frames overlap their copies with the labelling of
               the others and a step's uploads run under the previous step's downloads
               (times for other group counts, and with every call ordered on the stream,
               reported beside it)
  per_frame    the same 256 frames as 256 flic_label launches (frames/s, Mpixel/s,
               p50/p99 latency of one launch) and the batched/per-frame ratio
  roofline     flic_label_kernel: algorithmic bytes (4 B range in + 4 B label out per
               pixel) / mean launch time vs the measured HBM copy bandwidth
  projection   flic_project + flic_label + flic_scatter on the 128x2048 occlusion frame
               with 262,144 xyz points
  projection_batch  a c5 batch of 96 clouds (30k-260k points each) through
               flic_project_batch + flic_label_batch + flic_scatter_batch, with the HBM
               rooflines of the batched projection and scatter
  edges        flic_edges (the 16-byte word pass) on a 512x4096 frame, S = 3 and 5, GB/s
  serving      a short sweep of the continuous-batching server (four Poisson sensors,
               half of the frames as xyz clouds) at 1,000 / 5,000 / 20,000 frames/s:
               p50/p99 latency from submission to labels in host memory
  cpu_baseline the CPU oracle (sequential BFS, 1 thread) on all 256 frames once
The launch shape is autotuned on the batch first (paper_2003_00575_gb300/autotune.py,
cached as JSON) unless --tuning or --no-autotune is given; config.tuning records it.
L2 policy: three copies of the batch's buffers (~700 MB, > 129 MB L2) are used in
rotation, so no step finds its inputs in L2.

--impl reference times the CPU oracle (the plain sequential labeller) instead: one frame of
the same batch per step, cycling, on the host cores of rank 0.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import platform
import re
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "labelled Mpixel/s & frames/s, batched vs per-frame; p50/p99 frame latency"
UNIT = "Mpixel/s"
WORKLOAD = ("c4 batch: 256 frames of uneven shape {16x1800, 32x1024, 64x2048, 128x2048}, "
            "per-frame elevation table, delta U(0.3,0.6) m, skip U{1..5}, c2-style scenes; "
            "one persistent launch under a CUDA graph")
BYTES_PER_PX = 8  # 4 B range read + 4 B label written
NCOPIES = 3
PROFILE_NOTE = os.path.join(ROOT, "profiles", "flic_label_kernel.c4_batch.md")
CSRC = os.path.join(ROOT, "paper_2003_00575_gb300", "csrc")


def parse_args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5000)
    p.add_argument("--warmup", type=int, default=20)
    p.add_argument("--impl", choices=["flic", "reference"], default="flic")
    p.add_argument("--frames", type=int, default=256)
    p.add_argument("--per-frame-reps", type=int, default=20)
    p.add_argument("--e2e-steps", type=int, default=100)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--tuning", type=str, default="",
                   help="px_per_cta,threads,max_strips,ctas_per_sm for the batch (skips autotuning)")
    p.add_argument("--no-autotune", action="store_true")
    p.add_argument("--proj-scale", type=int, default=1,
                   help="repeat the c3 cloud this many times in the projection section "
                        "(a cloud larger than L2 for DRAM counters)")
    p.add_argument("--serve-seconds", type=float, default=3.0,
                   help="short serving sweep (0 = skip); the full sweep is serve.py")
    return p.parse_args()


def host_cpu() -> str:
    """Model of the host CPU (x86 and Arm report it under different names)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.split(":")[0].strip() in ("Model name", "Model"):
                name = line.split(":", 1)[1].strip()
                if name and not name.isdigit():
                    return name
    except (OSError, subprocess.SubprocessError):
        pass
    return platform.machine()


def rank_first_seed(rank: int, frames: int) -> int:
    """Weak scaling: rank r labels the c4 frames with seeds 100 + r*frames ... (disjoint)."""
    return 100 + rank * frames


def reduce_max(dist, value: float, device) -> float:
    """Max over ranks of a per-rank time (the job is as slow as its slowest rank)."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


KERNEL_SOURCES = ("flic_label.cu", "flic_device.cuh")


def source_sha() -> str:
    """Hash of the labelling kernel's own sources (what its DRAM traffic depends on)."""
    h = hashlib.sha256()
    for fn in KERNEL_SOURCES:
        h.update(fn.encode())
        h.update(open(os.path.join(CSRC, fn), "rb").read())
    return h.hexdigest()[:16]


def committed_counter(name: str):
    """A per-launch counter from the committed ncu summary, if taken on these sources."""
    if not os.path.exists(PROFILE_NOTE):
        return None
    text = open(PROFILE_NOTE).read()
    sha = re.search(r"source_sha256_16:\s*([0-9a-f]+)", text)
    val = re.search(name + r":\s*([0-9.eE+]+)", text)
    if not sha or not val or sha.group(1) != source_sha():
        return None
    return float(val.group(1))


def committed_traffic():
    """DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum)."""
    return committed_counter("traffic_bytes_per_launch_full_batch")


def load_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 100 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,utilization.gpu,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    NAMES = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]

    def __init__(self, bus_id: str | None):
        self.bus_id = bus_id
        self.proc = None
        self.out = None

    def start(self):
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
               "-lms", "100"]
        if self.bus_id:
            cmd += ["-i", self.bus_id]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                                         text=True)
        except OSError:
            self.proc = None
        time.sleep(0.15)

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        time.sleep(0.15)
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        return self.parse(out)

    @classmethod
    def parse(cls, out: str) -> dict:
        """The clock record of nvidia-smi's CSV lines: median SM clock of the samples under
        load (utilisation >= 30 %, else all), the highest max clock, the throttle reasons
        seen active under load."""
        rows = []
        for line in out.strip().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), float(parts[4]),
                             [n for n, v in zip(cls.NAMES, parts[5:9]) if v == "Active"]))
            except ValueError:
                continue
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        loaded = [r for r in rows if r[2] >= 30] or rows
        reasons = sorted({n for r in loaded for n in r[3]})
        return {"sm_mhz": statistics.median(r[0] for r in loaded),
                "sm_max_mhz": max(r[1] for r in rows), "reasons": reasons,
                "samples": len(loaded)}


def pct(xs, q):
    return float(np.percentile(np.asarray(xs, dtype=np.float64), q))


# ------------------------------------------------------------------------ reference arm

def run_reference(args, world, rank):
    if rank != 0:
        return
    import oracle
    from paper_2003_00575_gb300 import synth
    frames = synth.config_c4(args.frames)
    oracle.build()
    times = []
    px = 0
    for i in range(args.warmup + args.steps):
        f = frames[i % len(frames)]
        t0 = time.perf_counter()
        oracle.label(f.range, f.sensor.elevation, f.sensor.az_step, f.delta, f.skip)
        dt = time.perf_counter() - t0
        if i >= args.warmup:
            times.append(dt)
            px += f.range.size
    total = sum(times)
    value = px / total / 1e6
    sample = (f"one c4 frame per step, cycling through the {len(frames)} frames "
              f"({args.steps} steps, {px} px), sequential C BFS labeller")
    line = {
        "impl": "reference", "metric": METRIC, "value": round(value, 3), "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(1e3 * total / args.steps, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "frames": len(frames), "impl_note": "CPU oracle"},
        "cpu_baseline": {"value": round(value, 3), "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": sample, "host_cpu": host_cpu()},
        "e2e": {"value": round(value, 3), "unit": UNIT, "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
        "frames_per_s": round(args.steps / total, 2),
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------------ flic arm

def fp64_flip_count(oracle, synth, c4_frames):
    """Edge decisions of the fp32 test (Eq. 3's constant, the one both the kernels and the
    oracle evaluate) that the exact double-precision Eq. 2 decides the other way, over every
    candidate pair of c1-c3 and of the c4 frames; every flip must lie within 1e-5 m of delta."""
    out = {}
    sets = {"c1": [synth.config_c1()], "c2": [synth.config_c2()],
            "c3": [synth.config_c3(with_xyz=False)], "c4": c4_frames}
    for name, fr in sets.items():
        pairs = flips = lit_flips = lit_far = 0
        dev = lit_dev = 0.0
        for f in fr:
            p, n, d = oracle.flips(f.range, f.sensor.elevation, f.sensor.az_step, f.delta, f.skip)
            pairs += p
            flips += n
            dev = max(dev, d)
            _, n2, far2, d2 = oracle.flips_paper_form(f.range, f.sensor.elevation,
                                                      f.sensor.az_step, f.delta, f.skip)
            lit_flips += n2
            lit_far += far2
            lit_dev = max(lit_dev, d2)
        assert flips == 0 or dev < 1e-5, (name, flips, dev)
        out[name] = {"frames": len(fr), "pairs": pairs, "flips": flips,
                     "max_abs_d_minus_delta_m": dev,
                     "literal_eq3_form": {"flips": lit_flips, "flips_beyond_bound": lit_far,
                                          "max_abs_d_minus_delta_m": lit_dev}}
    out["bound_m"] = 1e-5
    out["note"] = ("oracle.flips in the CPU-baseline leg, outside the timed region; the GPU "
                   "edge bits equal the oracle's bit for bit, so the counts hold for both. "
                   "literal_eq3_form: the same pairs decided by Eq. 3 as printed, "
                   "d1*d1 + d2*d2 - (2 cos alpha)*d1*d2 in fp32 (a diagnostic; not used)")
    return out


def host_ahead(torch, stream, us: float = 1000.0) -> None:
    """Occupy the stream with a spin kernel of about `us` microseconds so that the launches
    enqueued after it are all queued on the device before the first timing event runs:
    events then time device work back to back, not the host's launch rate."""
    with torch.cuda.stream(stream):
        torch.cuda._sleep(int(us * 2000))


def edges_section(flic, synth, torch, dev, stream, peak, peak_kind):
    """flic_edges alone on the largest frame the API takes (512 x 4096 = 2^21 pixels: the
    c3 range image tiled 4 x 2), 16 frame copies in rotation (201 MB > L2), for S = 3 and
    5.  Algorithmic bytes: 4 B of range read and 2 B of mask written per pixel."""
    f3 = synth.config_c3(with_xyz=False)
    R, C = 512, 4096
    rimg = np.tile(f3.range, (4, 2))
    s = synth.make_sensor(R, C, -22.5, 22.5)
    ncopy, reps = 16, 4
    rs = [torch.from_numpy(rimg.reshape(-1)).to(dev) for _ in range(ncopy)]
    ms = [torch.empty(R * C, dtype=torch.int16, device=dev) for _ in range(ncopy)]
    out = {"workload": f"{R}x{C} (the c3 range image tiled 4 x 2), {ncopy} copies in "
                       f"rotation ({ncopy * 6 * R * C / 1e6:.0f} MB > L2)",
           "algorithmic_bytes_per_launch": 6 * R * C}
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    for S in (3, 5):
        h = flic.flic_create(R, C, s.elevation, s.az_step, 0.4, S)
        for i in range(3 * ncopy):
            flic.flic_edges(h, rs[i % ncopy], ms[i % ncopy], stream)
        torch.cuda.synchronize()
        host_ahead(torch, stream, 3000.0)
        ev[0].record(stream)
        for i in range(reps * ncopy):
            flic.flic_edges(h, rs[i % ncopy], ms[i % ncopy], stream)
        ev[1].record(stream)
        torch.cuda.synchronize()
        ok = flic.flic_device_status(h) == flic.FLIC_OK
        h.close()
        us = ev[0].elapsed_time(ev[1]) * 1e3 / (reps * ncopy)
        gbs = 6 * R * C / (us * 1e-6) / 1e9
        out[f"S{S}"] = {"us_per_launch": round(us, 3),
                        "roofline": {"bound": "hbm", "achieved": round(gbs, 1), "peak": peak,
                                     "unit": "GB/s", "frac": round(gbs / peak, 4),
                                     "traffic": None,
                                     "peak_source": f"of {peak_kind} (hbm_gbs, burst copy)"},
                        "status_ok": ok}
    out["timing"] = (f"{reps * ncopy} back-to-back launches between two CUDA events on the "
                     "launching stream, all queued behind a spin kernel before the first event "
                     "(device time, inter-launch gaps included), after 48 warm-up launches")
    return out


def projection_batch_section(flic, synth, torch, dev, stream, peak, peak_kind):
    """A c5 batch of 96 clouds (24 per serving sensor, 30k-260k points each: 16 distinct
    clouds, each in 6 separate device buffers) projected by flic_project_batch, labelled
    by flic_label_batch and scattered by flic_scatter_batch; two such batches in rotation
    (> L2).  Algorithmic bytes: projection 12 B xyz read + 4 B pixel index written per
    point and 4 B of range written per pixel; scatter 4 B pixel index + 4 B label read and
    4 B written per point."""
    sens = synth.c5_sensors()
    distinct = [synth.c5_frame(sens[i % 4], 9000 + i, as_cloud=True) for i in range(16)]
    nb, per = 2, 96
    batches = []
    for _ in range(nb):
        fr = [distinct[i % 16] for i in range(per)]
        hs = [flic.flic_create(f.sensor.rows, f.sensor.cols, f.sensor.elevation,
                               f.sensor.az_step, f.delta, f.skip) for f in fr]
        xyz = [torch.from_numpy(np.ascontiguousarray(f.xyz).reshape(-1)).to(dev) for f in fr]
        pix = [torch.empty(f.xyz.shape[0], dtype=torch.int32, device=dev) for f in fr]
        rng = [torch.empty(f.range.size, dtype=torch.float32, device=dev) for f in fr]
        lab = [torch.empty(f.range.size, dtype=torch.int32, device=dev) for f in fr]
        plab = [torch.empty_like(p) for p in pix]
        ca = flic.CloudArgs(hs, xyz, pix, range_out=rng, labels=lab, point_labels=plab)
        b = flic.flic_batch_create(per)
        batches.append((hs, ca, b, flic.BatchArgs(hs, rng, lab), xyz, pix, rng, lab, plab))
    npts = sum(distinct[i % 16].xyz.shape[0] for i in range(per))
    npx = sum(distinct[i % 16].range.size for i in range(per))
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    t = []
    for rep in range(23):
        hs, ca, b, ba = batches[rep % nb][:4]
        host_ahead(torch, stream, 1000.0)
        ev[0].record(stream)
        flic.flic_project_batch(ca, stream)
        ev[1].record(stream)
        flic.flic_label_batch(b, ba, stream)
        ev[2].record(stream)
        flic.flic_scatter_batch(ca, stream)
        ev[3].record(stream)
        torch.cuda.synchronize()
        if rep >= 3:
            t.append([ev[0].elapsed_time(ev[1]), ev[1].elapsed_time(ev[2]),
                      ev[2].elapsed_time(ev[3]), ev[0].elapsed_time(ev[3])])
    ok = all(flic.flic_device_status(h) == flic.FLIC_OK for bt in batches for h in bt[0])
    for bt in batches:
        bt[2].close()
        for h in bt[0]:
            h.close()
    t = np.array(t)
    med = [float(np.median(t[:, i])) for i in range(4)]
    pb = 16 * npts + 4 * npx
    sb = 12 * npts

    def roof(nbytes, ms):
        gbs = nbytes / (ms * 1e-3) / 1e9
        return {"bound": "hbm", "achieved": round(gbs, 1), "peak": peak, "unit": "GB/s",
                "frac": round(gbs / peak, 4), "traffic": None,
                "algorithmic_bytes_per_call": nbytes,
                "peak_source": f"of {peak_kind} (hbm_gbs, burst copy)"}

    return {"workload": f"c5 batch: {per} clouds on the 4 serving sensors, {npts:,} points, "
                        f"{npx:,} pixels, {nb} batches in rotation",
            "ms_project_batch": round(med[0], 4), "ms_label_batch": round(med[1], 4),
            "ms_scatter_batch": round(med[2], 4), "ms_total": round(med[3], 4),
            "clouds_per_s": round(per / (med[3] * 1e-3), 1),
            "mpoints_per_s": round(npts / (med[3] * 1e-3) / 1e6, 1),
            "roofline_project": roof(pb, med[0]), "roofline_scatter": roof(sb, med[2]),
            "launches": "project: 3 (keys cleared, points projected, ranges decoded); "
                        "label: 1; scatter: 1 (at most 96 clouds per launch)",
            "timing": "CUDA events between the calls on the launching stream, the three "
                      "calls queued behind a spin kernel before the first event (device "
                      "time); median of 20 after 3 warm-up batches",
            "status_ok": ok}


def main():
    args = parse_args()
    world, rank, local = dist_env()
    if args.impl == "reference":
        run_reference(args, world, rank)
        return

    import torch
    from paper_2003_00575_gb300 import flic, synth

    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    # ---- inputs: each rank labels its own 256 frames (weak scaling, no data collective)
    frames = synth.config_c4(args.frames, first_seed=rank_first_seed(rank, args.frames))
    sizes = [f.range.size for f in frames]
    offs = np.concatenate([[0], np.cumsum(sizes)])
    total_px = int(offs[-1])
    handles = [flic.flic_create(f.sensor.rows, f.sensor.cols, f.sensor.elevation,
                                f.sensor.az_step, f.delta, f.skip) for f in frames]
    host_range = torch.from_numpy(np.concatenate([f.range.reshape(-1) for f in frames]))
    rng_dev = torch.empty((NCOPIES, total_px), dtype=torch.float32, device=dev)
    lab_dev = torch.empty((NCOPIES, total_px), dtype=torch.int32, device=dev)
    for k in range(NCOPIES):
        rng_dev[k].copy_(host_range)
    tun = [int(x) for x in args.tuning.split(",")] if args.tuning else None
    batches, bargs = [], []
    for k in range(NCOPIES):
        b = flic.flic_batch_create(len(frames))
        if tun:
            flic.flic_batch_set_tuning(b, *tun)
        batches.append(b)
        bargs.append(flic.BatchArgs(
            handles, [rng_dev[k, offs[i]:offs[i + 1]] for i in range(len(frames))],
            [lab_dev[k, offs[i]:offs[i + 1]] for i in range(len(frames))]))
    stream = torch.cuda.current_stream()

    # ---- launch shape: autotuned on these frames (cached as JSON), or given
    tuned = None
    if not tun and not args.no_autotune:
        from paper_2003_00575_gb300 import autotune
        shapes = [(f.sensor.rows, f.sensor.cols, f.skip) for f in frames]
        tuned = autotune.tune_batch(flic, batches[0], bargs[0], shapes, stream)
        for b in batches[1:]:
            autotune.apply(flic, b, tuned["config"])

    # ---- warm-up
    for i in range(max(3, args.warmup)):
        flic.flic_label_batch(batches[i % NCOPIES], bargs[i % NCOPIES], stream)
    barrier()
    plan = flic.flic_batch_last_plan(batches[0])

    # ---- timed: K steps, events on the launching stream, clocks sampled meanwhile
    bus = None
    try:
        props = torch.cuda.get_device_properties(dev)
        bus = f"{props.pci_domain_id:08x}:{props.pci_bus_id:02x}:{props.pci_device_id:02x}.0"
    except Exception:
        bus = None
    sampler = ClockSampler(bus)
    sampler.start()
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    barrier()
    t_wall0 = time.perf_counter()
    evs[0].record(stream)
    for i in range(args.steps):
        flic.flic_label_batch(batches[i % NCOPIES], bargs[i % NCOPIES], stream)
        evs[i + 1].record(stream)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    t_wall1 = time.perf_counter()
    clocks = sampler.stop()
    step_ms = [evs[i].elapsed_time(evs[i + 1]) for i in range(args.steps)]
    total_ms = reduce_max(dist, evs[0].elapsed_time(evs[args.steps]), dev)
    ms_per_step = total_ms / args.steps
    value = total_px * world / (ms_per_step / 1e3) / 1e6
    frames_per_s = len(frames) * world / (ms_per_step / 1e3)

    # check the last outputs once (cheap invariant: every label is -1 or a valid index
    # whose own label is itself); parity proper lives in tests/
    lab0 = lab_dev[(args.steps - 1) % NCOPIES]
    sane = True
    for i in (0, len(frames) // 2, len(frames) - 1):
        l = lab0[offs[i]:offs[i + 1]].long()
        v = l[l >= 0]
        sane &= bool(((v >= 0) & (v < sizes[i])).all().item())
        if v.numel():
            sane &= bool((l[v] == v).all().item())

    # ---- roofline of flic_label_kernel (the only kernel in a step)
    peak, peak_kind = load_peak()
    mean_launch_s = statistics.mean(step_ms) / 1e3
    achieved = BYTES_PER_PX * total_px / mean_launch_s / 1e9
    traffic = committed_traffic()
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "traffic": traffic,
                "peak_source": f"of {peak_kind} (MEASURED_PEAKS.json hbm_gbs, burst copy)",
                "kernel": "flic_label_kernel",
                "algorithmic_bytes_per_launch": BYTES_PER_PX * total_px}
    # the ALU roof beside it: the edge test's 2S predicates per measurement, 6 fp32 ops each
    # (sub, mul, mul, mul, add, compare), against one fp32 op per lane per cycle
    # (128 lanes per SM, no FMA in the predicate) at the sampled maximum SM clock
    ops = sum(int((f.range > 0).sum()) * 2 * f.skip * 6 for f in frames)
    nsm = torch.cuda.get_device_properties(dev).multi_processor_count
    alu_peak = nsm * 128 * clocks["sm_max_mhz"] * 1e6 / 1e9 if clocks["sm_max_mhz"] else None
    alu_achieved = ops / mean_launch_s / 1e9
    roofline["alu"] = {"bound": "alu", "achieved": round(alu_achieved, 1),
                       "peak": round(alu_peak, 1) if alu_peak else None, "unit": "Gop/s",
                       "frac": round(alu_achieved / alu_peak, 4) if alu_peak else None,
                       "ops_per_launch": ops,
                       "peak_source": f"derived: {nsm} SMs x 128 fp32 lanes x max SM clock"}
    # the roof that binds this kernel: instruction issue, one warp instruction per cycle per
    # scheduler (4 per SM) at the sampled maximum SM clock, against the warp instructions
    # ncu counted for one launch of the same sources (null once the sources have changed)
    inst = committed_counter("warp_instructions_per_launch_full_batch")
    issue_peak = nsm * 4 * clocks["sm_max_mhz"] * 1e6 / 1e9 if clocks["sm_max_mhz"] else None
    issue_achieved = inst / mean_launch_s / 1e9 if inst else None
    roofline["issue"] = {"bound": "issue",
                         "achieved": round(issue_achieved, 1) if issue_achieved else None,
                         "peak": round(issue_peak, 1) if issue_peak else None,
                         "unit": "G warp-instructions/s",
                         "frac": round(issue_achieved / issue_peak, 4)
                         if issue_achieved and issue_peak else None,
                         "warp_instructions_per_launch": inst,
                         "peak_source": f"derived: {nsm} SMs x 4 schedulers x max SM clock"}

    # ---- cluster candidates (§III-B, the paper's minimum of 100 points) over the batch's
    # fresh labels: flic_filter_relabel_batch alone is timed
    rl_ms = []
    rl_num = torch.empty(len(frames), dtype=torch.int32, device=dev)
    rl_ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    for rep in range(23):
        k = rep % NCOPIES
        flic.flic_label_batch(batches[k], bargs[k], stream)
        rl_ev[0].record(stream)
        flic.flic_filter_relabel_batch(batches[k], bargs[k], 100, rl_num, stream)
        rl_ev[1].record(stream)
        torch.cuda.synchronize()
        if rep >= 3:
            rl_ms.append(rl_ev[0].elapsed_time(rl_ev[1]))
    cluster_filter = {
        "min_size": 100, "ms_per_batch": round(statistics.median(rl_ms), 4),
        "mpixel_per_s": round(total_px / (statistics.median(rl_ms) / 1e3) / 1e6, 1),
        "kept_clusters_per_frame": round(float(rl_num.float().mean().item()), 2),
        "launches": 6,
        "note": "relabel of the c4 batch's labels: components under 100 px dropped, the rest "
                "numbered 0..N-1 by minimum index; timed alone, after a fresh labelling"}

    # ---- labelling and the filter in one call (flic_label_filter_batch: sizes counted
    # inside the labelling kernel, no size histogram), against the two calls back to back
    # and the labelling alone; each queued behind a spin kernel so that the events time
    # the device
    modes = ("label", "separate", "fused")
    pair_ms = {m: [] for m in modes}
    pair_ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    for rep in range(69):
        k = rep % NCOPIES
        mode = modes[rep % 3]
        host_ahead(torch, stream, 1000.0)
        pair_ev[0].record(stream)
        if mode == "fused":
            flic.flic_label_filter_batch(batches[k], bargs[k], 100, rl_num, stream)
        else:
            flic.flic_label_batch(batches[k], bargs[k], stream)
            if mode == "separate":
                flic.flic_filter_relabel_batch(batches[k], bargs[k], 100, rl_num, stream)
        pair_ev[1].record(stream)
        torch.cuda.synchronize()
        if rep >= 9:
            pair_ms[mode].append(pair_ev[0].elapsed_time(pair_ev[1]))
    lab_ms = statistics.median(pair_ms["label"])
    sep_ms = statistics.median(pair_ms["separate"])
    fused_ms = statistics.median(pair_ms["fused"])
    label_filter = {
        "min_size": 100,
        "label_ms_per_batch": round(lab_ms, 4),
        "separate_ms_per_batch": round(sep_ms, 4),
        "fused_ms_per_batch": round(fused_ms, 4),
        "filter_share_separate_ms": round(sep_ms - lab_ms, 4),
        "filter_share_fused_ms": round(fused_ms - lab_ms, 4),
        "fused_mpixel_per_s": round(total_px / (fused_ms / 1e3) / 1e6, 1),
        "launches_separate": 7, "launches_fused": 5,
        "note": "label + cluster filter of the c4 batch: flic_label_batch then "
                "flic_filter_relabel_batch, against flic_label_filter_batch (component sizes "
                "counted in the labelling kernel; the zeroing and histogram launches go); the "
                "filter shares subtract the labelling alone, timed the same way"}

    # ---- ground extraction (§III-A, 10 degrees, height line 1.7 m) fused into the same
    # batched labelling: the batch timed again with the ground removed first
    for h in handles:
        flic.flic_set_ground(h, math.radians(10.0), 1.7)
    gd_ms = []
    gd_ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    for rep in range(33):
        k = rep % NCOPIES
        gd_ev[0].record(stream)
        flic.flic_label_batch(batches[k], bargs[k], stream)
        gd_ev[1].record(stream)
        torch.cuda.synchronize()
        if rep >= 3:
            gd_ms.append(gd_ev[0].elapsed_time(gd_ev[1]))
    lab_g = lab_dev[(33 - 1) % NCOPIES]
    removed = float(((lab_g < 0).sum() - (rng_dev[(33 - 1) % NCOPIES] <= 0).sum()).item())
    for h in handles:
        flic.flic_set_ground(h, 0.0, 0.0)
    ground_extraction = {
        "theta_deg": 10.0, "mount_height_m": 1.7,
        "ms_per_batch": round(statistics.median(gd_ms), 4),
        "mpixel_per_s": round(total_px / (statistics.median(gd_ms) / 1e3) / 1e6, 1),
        "ground_fraction_of_pixels": round(removed / total_px, 4),
        "note": "c4 batch labelled with ground extraction in the same persistent launch"}

    # ---- segmentation quality (§IV metrics) of the GPU labels on the ray-cast scenes,
    # whose per-pixel object ids are the ground truth: IoU_mu and P_x over the instances of
    # at least 100 px, with the ground removed by the ground truth or by §III-A's
    # extraction, for the direct neighbourhood (S = 1) and with skip connections
    from paper_2003_00575_gb300 import quality
    seg = {}
    for cname, fr in (("c2", synth.config_c2()), ("c3", synth.config_c3(with_xyz=False))):
        R, C = fr.sensor.rows, fr.sensor.cols
        gt = fr.object_id
        for S in sorted({1, fr.skip}):
            for mode in ("gt_ground_removed", "ground_extraction"):
                hq = flic.flic_create(R, C, fr.sensor.elevation, fr.sensor.az_step, fr.delta, S)
                rng_q = fr.range
                if mode == "gt_ground_removed":
                    rng_q = np.where(gt == 0, np.float32(0), fr.range).astype(np.float32)
                else:
                    flic.flic_set_ground(hq, math.radians(10.0), 1.7)
                lab_q = torch.empty(R * C, dtype=torch.int32, device=dev)
                flic.flic_label(hq, torch.from_numpy(np.ascontiguousarray(rng_q).reshape(-1)).to(dev),
                                lab_q, stream)
                torch.cuda.synchronize()
                seg[f"{cname}_S{S}_{mode}"] = quality.scores(lab_q.cpu().numpy(), gt)
                hq.close()
        # the paper's one Map Connection (every second point, §III-B-2) against offsets 1..2
        rng_q = np.where(gt == 0, np.float32(0), fr.range).astype(np.float32)
        for key, lat in (("S2", False), ("1MC_every_2nd_point", True)):
            hq = flic.flic_create(R, C, fr.sensor.elevation, fr.sensor.az_step, fr.delta, 2,
                                  lattice=lat)
            lab_q = torch.empty(R * C, dtype=torch.int32, device=dev)
            flic.flic_label(hq, torch.from_numpy(np.ascontiguousarray(rng_q).reshape(-1)).to(dev),
                            lab_q, stream)
            torch.cuda.synchronize()
            seg[f"{cname}_{key}_gt_ground_removed"] = quality.scores(lab_q.cpu().numpy(), gt)
            hq.close()
        # the distance-threshold study (§IV, parameter study of delta): IoU_mu over delta
        rng_t = torch.from_numpy(np.ascontiguousarray(rng_q).reshape(-1)).to(dev)
        for S in sorted({1, fr.skip}):
            sweep = {}
            for dl in (0.1, 0.2, 0.3, 0.4, 0.5, 0.6, 0.8, 1.0, 1.5, 2.0):
                hq = flic.flic_create(R, C, fr.sensor.elevation, fr.sensor.az_step, dl, S)
                lab_q = torch.empty(R * C, dtype=torch.int32, device=dev)
                flic.flic_label(hq, rng_t, lab_q, stream)
                torch.cuda.synchronize()
                sweep[str(dl)] = quality.scores(lab_q.cpu().numpy(), gt).get("iou_mu")
                hq.close()
            seg[f"{cname}_S{S}_iou_mu_by_delta_m"] = sweep
    seg["note"] = ("§IV metrics against the ray caster's object ids (instances >= 100 px); "
                   "the paper's own numbers are on SemanticKITTI, not comparable")

    # ---- per-frame launches: the same frames, one flic_label call each
    single_lat = []
    pf_total = []
    pf_evs = [torch.cuda.Event(enable_timing=True) for _ in range(len(frames) + 1)]
    for rep in range(args.per_frame_reps + 2):
        k = rep % NCOPIES
        pf_evs[0].record(stream)
        for i, h in enumerate(handles):
            flic.flic_label(h, rng_dev[k, offs[i]:offs[i + 1]], lab_dev[k, offs[i]:offs[i + 1]],
                            stream)
            pf_evs[i + 1].record(stream)
        torch.cuda.synchronize()
        if rep >= 2:
            pf_total.append(pf_evs[0].elapsed_time(pf_evs[-1]))
            single_lat += [pf_evs[i].elapsed_time(pf_evs[i + 1]) for i in range(len(frames))]
    pf_ms = statistics.mean(pf_total)
    per_frame = {
        "frames_per_s": round(len(frames) / (pf_ms / 1e3), 1),
        "mpixel_per_s": round(total_px / (pf_ms / 1e3) / 1e6, 1),
        "ms_per_256_frames": round(pf_ms, 4),
        "latency_ms_p50": round(pct(single_lat, 50), 4),
        "latency_ms_p99": round(pct(single_lat, 99), 4),
    }

    # ---- e2e: the host-buffer batch call (flic_label_batch_host) on pinned packed
    # buffers: per step every range image goes up and every label comes back, inside the
    # timed region; groups of frames overlap their copies with the labelling of others
    host_in = host_range.pin_memory()
    host_out = torch.empty(total_px, dtype=torch.int32).pin_memory()
    e2e_steps = max(3, args.e2e_steps)
    hb = flic.flic_batch_create(len(frames))
    if tun:
        flic.flic_batch_set_tuning(hb, *tun)
    elif tuned:
        autotune.apply(flic, hb, tuned["config"])

    def e2e_time(groups, steps, ready=True):
        for _ in range(3):
            flic.flic_label_batch_host(hb, handles, host_in, host_out, groups, ready, stream)
        torch.cuda.synchronize()
        barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            flic.flic_label_batch_host(hb, handles, host_in, host_out, groups, ready, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        return reduce_max(dist, e0.elapsed_time(e1) / steps, dev)

    e2e_groups = {g: round(e2e_time(g, max(3, e2e_steps // 4)), 4) for g in (1, 2, 3, 6, 8)}
    e2e_ordered = round(e2e_time(0, max(3, e2e_steps // 4), ready=False), 4)
    e2e_ms = e2e_time(0, e2e_steps)
    e2e_groups[4] = round(e2e_ms, 4)
    flic.flic_label_batch(batches[0], bargs[0], stream)  # the device path on the same frames
    torch.cuda.synchronize()
    e2e_ok = bool(np.array_equal(host_out.numpy(), lab_dev[0].cpu().numpy()))
    # the link's limit for this step: one step's upload and download at once, on two
    # streams, nothing else running (best of 8)
    up_s, dn_s = torch.cuda.Stream(), torch.cuda.Stream()
    link_ms = {"both": [], "h2d": [], "d2h": []}
    for rep in range(8):
        for kind in link_ms:
            c0 = torch.cuda.Event(enable_timing=True)
            c1 = torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            # a short sleep on the stream first, so that the copies are queued by the time
            # the start event is reached (the host's enqueue time is not the link's)
            torch.cuda._sleep(200_000)
            c0.record(stream)
            up_s.wait_event(c0)
            dn_s.wait_event(c0)
            if kind != "d2h":
                with torch.cuda.stream(up_s):
                    rng_dev[1].copy_(host_in, non_blocking=True)
            if kind != "h2d":
                with torch.cuda.stream(dn_s):
                    host_out.copy_(lab_dev[1], non_blocking=True)
            stream.wait_stream(up_s)
            stream.wait_stream(dn_s)
            c1.record(stream)
            torch.cuda.synchronize()
            link_ms[kind].append(c0.elapsed_time(c1))
    link = {k: round(min(v[2:]), 4) for k, v in link_ms.items()}
    hb.close()
    e2e = {"value": round(total_px * world / (e2e_ms / 1e3) / 1e6, 1), "unit": UNIT,
           "h2d_bytes_per_step": 4 * total_px, "d2h_bytes_per_step": 4 * total_px,
           "ms_per_step": round(e2e_ms, 4),
           "api": "flic_label_batch_host, 4 groups, FLIC_HOST_INPUT_READY (a step's uploads "
                  "run under the previous step's downloads)",
           "ms_per_step_by_groups": {str(k): v for k, v in sorted(e2e_groups.items())},
           "ms_per_step_each_call_ordered_on_stream": e2e_ordered,
           "copy_floor": {"ms_h2d_and_d2h_at_once": link["both"], "ms_h2d_alone": link["h2d"],
                          "ms_d2h_alone": link["d2h"],
                          "frac": round(link["both"] / e2e_ms, 4),
                          "note": "one step's 4 B/px upload and 4 B/px download as plain "
                                  "copies on two streams: the link's limit for e2e"},
           "labels_match_device_path": e2e_ok}
    sane &= e2e_ok

    # ---- projection path on the occlusion-heavy 128x2048 frame (262,144 points)
    f3 = synth.config_c3()
    s3 = f3.sensor
    h3 = flic.flic_create(s3.rows, s3.cols, s3.elevation, s3.az_step, f3.delta, f3.skip)
    cloud = np.tile(f3.xyz, (max(1, args.proj_scale), 1))  # copies tie; the lowest index wins
    xyz = torch.from_numpy(cloud).to(dev)
    rimg = torch.empty(s3.rows * s3.cols, dtype=torch.float32, device=dev)
    pix = torch.empty(cloud.shape[0], dtype=torch.int32, device=dev)
    lab3 = torch.empty(s3.rows * s3.cols, dtype=torch.int32, device=dev)
    plab = torch.empty_like(pix)
    pe = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    lat_proj = []
    for rep in range(53):
        pe[0].record(stream)
        flic.flic_project(h3, xyz, rimg, pix, stream)
        pe[1].record(stream)
        flic.flic_label(h3, rimg, lab3, stream)
        pe[2].record(stream)
        flic.flic_scatter(h3, lab3, pix, plab, stream)
        pe[3].record(stream)
        torch.cuda.synchronize()
        if rep >= 3:
            lat_proj.append([pe[0].elapsed_time(pe[1]), pe[1].elapsed_time(pe[2]),
                             pe[2].elapsed_time(pe[3]), pe[0].elapsed_time(pe[3])])
    lp = np.array(lat_proj)
    projection = {
        "workload": f"c3 128x2048 S5 delta 0.4, {cloud.shape[0]:,} xyz points"
                    + (f" (the c3 cloud {args.proj_scale} times)" if args.proj_scale > 1 else ""),
        "ms_project": round(float(np.median(lp[:, 0])), 4),
        "ms_label": round(float(np.median(lp[:, 1])), 4),
        "ms_scatter": round(float(np.median(lp[:, 2])), 4),
        "latency_ms_p50": round(pct(lp[:, 3], 50), 4),
        "latency_ms_p99": round(pct(lp[:, 3], 99), 4),
        "mpoints_per_s": round(cloud.shape[0] / (float(np.median(lp[:, 3])) / 1e3) / 1e6, 1),
    }
    h3.close()
    edges = edges_section(flic, synth, torch, dev, stream, peak, peak_kind)
    sane &= edges["S3"]["status_ok"] and edges["S5"]["status_ok"]
    projection_batch = projection_batch_section(flic, synth, torch, dev, stream, peak, peak_kind)
    sane &= projection_batch["status_ok"]

    # ---- short serving sweep: four Poisson sensors, half clouds (the full one: serve.py)
    serving = None
    if args.serve_seconds > 0 and world == 1:
        from paper_2003_00575_gb300 import serve
        sens = synth.c5_sensors()
        sh = [flic.flic_create(x.rows, x.cols, x.elevation, x.az_step, 0.5, 3) for x in sens]
        pool = serve.FramePool(sens, per_kind=2, outputs=128)
        srv = flic.flic_server_create(sh, pool.max_points, nstreams=2, max_batch=256,
                                      mem_budget=2 << 30)
        serve.run_step(flic, srv, pool, 500.0, 0.3, 999)  # first launches capture graphs
        serving = [serve.run_step(flic, srv, pool, rate, args.serve_seconds / 3, 1000 + i)
                   for i, rate in enumerate((1000.0, 5000.0, 20000.0))]
        srv.close()
        for x in sh:
            x.close()

    # ---- CPU baseline: the oracle as it stands, 1 thread, all frames once (rank 0, N=1)
    cpu = None
    fp64_flips = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle  # CPU baseline leg only
        oracle.build()
        t0 = time.perf_counter()
        for f in frames:
            oracle.label(f.range, f.sensor.elevation, f.sensor.az_step, f.delta, f.skip)
        dt = time.perf_counter() - t0
        ncores = os.cpu_count() or 1
        cpu = {"value": round(total_px / dt / 1e6, 3), "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"all {len(frames)} c4 frames once ({total_px} px, {dt:.2f} s), "
                         f"sequential C BFS labeller, 1 thread of {ncores} host cores",
               "frames_per_s": round(len(frames) / dt, 2), "host_cpu": host_cpu()}
        # the same frames spread over every host core (threads: the C labeller runs
        # outside the interpreter lock)
        from concurrent.futures import ThreadPoolExecutor
        t0 = time.perf_counter()
        with ThreadPoolExecutor(ncores) as ex:
            list(ex.map(lambda f: oracle.label(f.range, f.sensor.elevation, f.sensor.az_step,
                                               f.delta, f.skip), frames))
        dt_all = time.perf_counter() - t0
        cpu["all_cores"] = {"value": round(total_px / dt_all / 1e6, 3), "unit": UNIT,
                            "cores": ncores, "frames_per_s": round(len(frames) / dt_all, 2)}
        fp64_flips = fp64_flip_count(oracle, synth, frames)

    for h in handles:
        st = flic.flic_device_status(h)
        sane &= st == flic.FLIC_OK

    if rank == 0:
        line = {
            "metric": METRIC, "value": round(value, 1), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_per_step, 5),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "frames_per_gpu": len(frames),
                       "pixels_per_gpu": total_px,
                       "l2": f"inputs larger than L2: {NCOPIES} buffer copies in rotation "
                             f"({NCOPIES * 8 * total_px / 1e6:.0f} MB)",
                       "parallelism": f"frames sharded, {world} rank(s)",
                       "launch": plan,
                       "tuning": tuned if tuned else (args.tuning or "built-in")},
            "frames_per_s": round(frames_per_s, 1),
            "latency_ms_p50": round(pct(step_ms, 50), 4),
            "latency_ms_p99": round(pct(step_ms, 99), 4),
            "per_frame": per_frame,
            "batched_vs_per_frame": round(frames_per_s / world / per_frame["frames_per_s"], 2),
            "e2e": e2e,
            "roofline": roofline,
            "projection": projection,
            "projection_batch": projection_batch,
            "edges": edges,
            "cluster_filter": cluster_filter,
            "label_filter": label_filter,
            "ground_extraction": ground_extraction,
            "segmentation_quality": seg,
            "serving": serving,
            "cpu_baseline": cpu,
            "fp64_flips": fp64_flips,
            "clocks": {k: clocks[k] for k in ("sm_mhz", "sm_max_mhz", "reasons")},
            "clock_samples": clocks["samples"],
            "clock_note": (None if clocks["samples"] >= 10 else
                           f"only {clocks['samples']} clock samples under load: the timed region "
                           "was short; the clock record is weak evidence"),
            "gpu_launches": args.steps,
            "wall_s_timed": round(t_wall1 - t_wall0, 3),
            "outputs_sane": bool(sane),
            "paper_context": "paper: up to 165 Hz, Python, one i7-6820HQ core (not comparable)",
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
