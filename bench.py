#!/usr/bin/env python
"""Benchmark of the GS-NFS per-frame codec on GB300.

Workload: dynamic 3DGS frames of 1,000,000 Gaussians (56 float32 attributes,
octree depth 16, 5 quantisation groups), seeded synthetic frames shaped like
the paper's dynamic-scene workloads.  One step = the whole hot path on a
batch of F = 16 frames: batched encode (voxelise, sort, merge, occupancy,
rANS, RAHT prelude + forward, quantise + RLGR, container) followed by
decoding every stream (rANS, octree, RLGR, inverse RAHT).  `value` = frames
encoded AND decoded per second over all ranks, inputs resident in HBM.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gsnfs|reference]

Beside the headline the line carries the batched-vs-plain legs: the
bandwidth ladder (16 frames spanning 50k-2M Gaussians at depths 16-18, 5
rungs; batched call against one plain call per frame and rung) and the
dynamic sequence (30 frames of ~250k Gaussians; plain per-frame p50/p99
latency and batched throughput).

Under torchrun (N > 1) each rank codes its own frames (weak scaling, no
data-path collective).  `--impl reference` times the FP64 CPU oracle on the
host cores (the comparison arm): the same frames, one whole frame per
process, every frame of a step coded in parallel.  Prints one JSON line on
rank 0.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "encode/decode frames/s at 1M Gaussians, batched vs plain; % HBM roofline"
UNIT = "frames/s"
N_GAUSS = 1_000_000
C = 56
J = 16
N_FRAMES = 16  # frames per rank per step
RANS_CHUNK = 4096
LADDER_FRAMES = 16  # of the 64-frame ladder, spanning its sizes
SEQ_FRAMES = 30  # of the 300-frame sequence, every 10th
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per frame of this
# workload from one ncu capture of each kernel (2 frames, scaled per frame;
# summaries under profiles/), with the SHA-1 of the kernel's source file at
# capture time: reported only while that file is unchanged.
TRAFFIC = {
    "raht_forward_pass0": (521.32e6, "csrc/raht.cu", "e71b430b053aea96af59c126e5d948bacc8bcb50"),
    "raht_inverse_pass0": (441.58e6, "csrc/raht.cu", "e71b430b053aea96af59c126e5d948bacc8bcb50"),
    "rlgr_encode": (277.95e6, "csrc/rlgr.cu", "4e2e1fc2ff5a6d4b5b09d83a4d1bd52db792c215"),
    "rlgr_decode": (253.00e6, "csrc/rlgr.cu", "4e2e1fc2ff5a6d4b5b09d83a4d1bd52db792c215"),
}
# warp instructions executed per frame (ncu smsp__inst_executed.sum on 2 frames of 1M Gaussians, halved) and the
# source they were counted on: the RLGR coders are bound by instruction issue, not by DRAM
INSTR = {
    "rlgr_encode": (112873533, "csrc/rlgr.cu", "4e2e1fc2ff5a6d4b5b09d83a4d1bd52db792c215"),
    "rlgr_decode": (116638655, "csrc/rlgr.cu", "4e2e1fc2ff5a6d4b5b09d83a4d1bd52db792c215"),
}
# timed steps of the oracle arm (each one is the whole headline workload on the host cores)
REF_MAX_STEPS = 24
# largest share of serialised GPU time in the ncu launch list of the headline workload (16.0% of the timed steps)
DOMINANT = "raht_forward_pass0"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=80)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gsnfs", choices=["gsnfs", "reference"])
    ap.add_argument("--frames", type=int, default=N_FRAMES, help="frames per rank per step")
    ap.add_argument("--block", type=int, default=512, help="RLGR block size")
    ap.add_argument("--no-extras", action="store_true", help="skip plain-path, e2e and CPU-baseline legs")
    ap.add_argument("--no-tune", action="store_true", help="built-in launch shapes instead of autotuning them "
                                                            "(short profiling runs)")
    ap.add_argument("--graphs", type=int, default=1, choices=[0, 1],
                    help="replay the headline encoder's device work as a CUDA graph (captured once per request "
                         "shape during the warm-up steps)")
    ap.add_argument("--workload", default="headline", choices=["headline", "ladder", "sequence", "pointcloud",
                                                                 "blocksweep"],
                    help="other workloads, each printing its own JSON line: ladder (64 frames of 50k-2M Gaussians x "
                         "5 rungs, batched vs plain), sequence (300 frames of ~250k Gaussians, 3 steps), pointcloud "
                         "(150 frames of ~1M points, depth 10, YCbCr, 5 steps), blocksweep (RLGR block size)")
    ap.add_argument("--seq-frames", type=int, default=0, help="frames of the sequence / point-cloud workloads "
                                                              "(default: 300 / 150)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons, power = [], None, set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
                power.append(float(f[3]))
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if f[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm),
                "power_w_max": max(power) if power else None}


def _headline_frame(seed_t_n):
    from paper_2606_05650_gb300 import synthetic as syn
    seed, t, n = seed_t_n if len(seed_t_n) == 3 else (*seed_t_n, N_GAUSS)
    return syn.DynamicScene(seed).frame(t, n=n)


def _ladder_frame(f_n):
    from paper_2606_05650_gb300 import synthetic as syn
    f, n = f_n
    return syn.DynamicScene(3000).frame(f, n=int(n))


def _seq_frame(t):
    from paper_2606_05650_gb300 import synthetic as syn
    return syn.DynamicScene(2000).frame(t)


def _pool_map(fn, items):
    """Host frames generated by a spawned pool on the host cores (spawned, so it is safe beside CUDA)."""
    import multiprocessing as mp
    if not items:
        return []
    with mp.get_context("spawn").Pool(max(1, min(os.cpu_count() or 1, 16, len(items)))) as pool:
        return pool.map(fn, items, chunksize=1)


def make_frames(rank, F, n=N_GAUSS):
    """The frames rank `rank` codes: its own dynamic scene (frames are independent units, so ranks share
    no data and need no collective on the data path)."""
    items = [(1000 + rank, t, n) for t in range(F)]
    if F * n <= 2_000_000:  # small: not worth a pool
        return [_headline_frame(it) for it in items]
    return _pool_map(_headline_frame, items)


def ladder_subset():
    """LADDER_FRAMES of the 64 ladder frames (Gaussian counts log-uniform in [50k, 2M], depths 16/17/18):
    the frames at evenly spaced ranks of the sorted sizes, smallest and largest included."""
    import numpy as np
    from paper_2606_05650_gb300 import synthetic as syn
    sizes, depths = syn.ladder_sizes(3000)
    pick = np.argsort(sizes, kind="stable")[np.linspace(0, len(sizes) - 1, LADDER_FRAMES).round().astype(int)]
    return [int(f) for f in pick], [int(sizes[f]) for f in pick], [int(depths[f]) for f in pick]


def max_over_ranks(elapsed_ms, world, dist, device=None):
    """The job's time: the slowest rank's timed region (all_reduce MAX; no-op at one rank)."""
    if world <= 1:
        return float(elapsed_ms)
    import torch
    t = torch.tensor([float(elapsed_ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# Stage-minimum bytes per Gaussian of one encode + decode round trip at C = 56 (each stage reading and writing its
# compulsory bytes once, stages unfused): encode 1,244 (voxelise 36, sort 24, merge 468, occupancy 15, rANS 5,
# prelude 24, forward 448, quantise + RLGR 224), decode 758 (geometry 30: occupancy decode, codes, centres;
# prelude 24; RLGR 256: stream read, coefficients written; inverse 448).
PIPELINE_BYTES_PER_GAUSSIAN = 1244 + 758


def pipeline_fraction(frames_per_s, gaussians_per_frame, peak_gbs):
    """End-to-end roofline fraction: frames/s x stage-minimum bytes per frame / peak HBM bandwidth."""
    return frames_per_s * gaussians_per_frame * PIPELINE_BYTES_PER_GAUSSIAN / (peak_gbs * 1e9)


def job_throughput(world, frames_per_rank, steps, elapsed_ms):
    """Frames encoded and decoded per second by the whole job (weak scaling: every rank codes its own frames)."""
    return world * frames_per_rank * steps / (elapsed_ms / 1e3)


def headline_config(F, block, world):
    """The workload of the headline line, the same for the GPU arm and the reference arm."""
    return {"workload": f"dynamic 3DGS frames, {N_GAUSS} Gaussians x {C} float32 attributes, depth {J}, "
                        f"{F} frames per GPU per step, encode + decode of every frame",
            "frames_per_step_per_gpu": F, "gaussians_per_frame": N_GAUSS, "channels": C, "depth": J,
            "rlgr_block": block, "rans_chunk": RANS_CHUNK, "parallelism": f"frames x {world}",
            "l2": f"inputs {F * N_GAUSS * (3 + C) * 4 / 1e9:.1f} GB per step > 129 MB L2 (no flush needed)"}


# ------------------------------------------------------------------ GPU arm
def run_gpu(args):
    import numpy as np

    rank, world, local = dist_env()
    F = args.frames
    # host frames first, on the host cores, before any CUDA work
    frames = make_frames(rank, F)
    lad_idx, lad_n, lad_J = ladder_subset()
    extra_frames = {}
    if not args.no_extras and rank == 0:
        extra_frames["ladder"] = _pool_map(_ladder_frame, list(zip(lad_idx, lad_n)))
        extra_frames["sequence"] = _pool_map(_seq_frame, list(range(0, 10 * SEQ_FRAMES, 10)))

    import torch
    import torch.distributed as dist
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)
    import __graft_entry__
    if rank == 0:
        __graft_entry__.build()
    if world > 1:
        dist.barrier()
    __graft_entry__.build()
    from paper_2606_05650_gb300 import gsnfs as G, synthetic as syn

    P = [torch.from_numpy(p).to(dev) for p, _ in frames]
    A = [torch.from_numpy(a).to(dev) for _, a in frames]
    qp = G.QuantParams(syn.gs_channel_groups(), syn.GS_BASE_STEPS, rlgr_block=args.block, rans_chunk=RANS_CHUNK)
    Js = [J] * F
    out = None
    # decoded frames and per-step decode statuses (the decoder is asynchronous: it takes the header records the
    # encoder returns, so the step's only host wait is the encoder's read-back of its offsets)
    pos_o = torch.empty((F * N_GAUSS, 3), dtype=torch.float32, device=dev)
    att_o = torch.empty((F * N_GAUSS, C), dtype=torch.float32, device=dev)
    status = torch.full((64,), -1, dtype=torch.int32, device=dev)
    nstep = [0]

    def step():
        nonlocal out
        out, offs, hdr = G.encode_batch(P, A, Js, [1.0], qp, out=out, headers=True)
        k = nstep[0] % status.numel()
        nstep[0] += 1
        rows = G.decode_batch_async(out, offs, hdr, C, F * N_GAUSS, pos_o, att_o, status[k:k + 1])
        return offs, rows

    # launch shapes tuned on this workload (outputs checked identical for every candidate)
    from paper_2606_05650_gb300 import autotune
    tuning = ({"params": "built-in", "ms": None, "default_ms": None} if args.no_tune else
              autotune.tune_round_trip(P, A, Js, qp, use_cache=False))
    G.set_graphs(bool(args.graphs))
    for _ in range(max(args.warmup, 1)):
        offs, rows = step()
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream(dev)

    def barrier():
        if world > 1:
            dist.barrier()

    # ---- timed region (device-resident inputs; inputs 1.9 GB per step >> 129 MB L2)
    G.profile_enable(True)
    G.profile_read()
    clocks = ClockSampler(local)
    clocks.start()
    l0 = G.launch_count()
    barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        offs, rows = step()
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    launches = G.launch_count() - l0
    ck = clocks.stop()
    st_seen = status[:min(nstep[0], status.numel())].cpu().tolist()
    if any(v != 0 for v in st_seen):
        raise RuntimeError(f"asynchronous decode reported status {st_seen}")
    elapsed_ms = e0.elapsed_time(e1)
    stages = G.profile_read()
    G.profile_enable(False)
    elapsed_ms = max_over_ranks(elapsed_ms, world, dist, dev)
    value = job_throughput(world, F, args.steps, elapsed_ms)
    nv_frames = np.diff(rows).astype(np.int64)
    stream_bytes = np.diff(offs).astype(np.int64)

    extras = {}
    if not args.no_extras:
        extras = gpu_extras(args, G, torch, P, A, frames, qp, out, offs, dev, stream)
        if rank == 0:
            extras["ladder"] = ladder_leg(G, torch, dev, stream, extra_frames.pop("ladder"), lad_J, args.block,
                                          lad_idx)
            extras["sequence"] = sequence_leg(G, torch, dev, stream, extra_frames.pop("sequence"), args.block)

    if rank == 0:
        peaks, src = measured_peaks()
        hbm = float(peaks["hbm_gbs"])
        smax = ck.get("sm_max_mhz") or 2070.0
        issue_peak = torch.cuda.get_device_properties(dev).multi_processor_count * 4 * float(smax) * 1e6
        roof = roofline(stages, frames, nv_frames, stream_bytes, args.steps, F, hbm, src, issue_peak)
        res = {
            "metric": METRIC, "value": round(value, 2), "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(elapsed_ms / args.steps, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": headline_config(F, args.block, world),
            "path": "batched: one encode call (returning the streams' header records) and one asynchronous decode "
                    "call per step for all frames of the rank"
                    + ("; encoder replayed as a CUDA graph" if args.graphs else ""),
            "tuning": {"params": tuning["params"], "tuned_ms": tuning["ms"], "default_ms": tuning["default_ms"]},
            "encode_decode_fps": round(value, 2),
            "voxels_per_frame": int(nv_frames.mean()), "bytes_per_frame": int(stream_bytes.mean()),
            "bits_per_gaussian": round(8 * float(stream_bytes.mean()) / N_GAUSS, 3),
            "roofline": roof,
            "pipeline_fraction": round(pipeline_fraction(value, N_GAUSS, roof["peak"]), 4) if roof else None,
            "stages_ms_per_step": {k: round(v[0] / args.steps, 4) for k, v in stages.items() if v[1]},
            "stages_roofline": stage_roofline(stages, sum(p.shape[0] for p, _ in frames), args.steps, hbm, C, J),
            "gpu_launches": int(launches),
            "clocks": ck,
        }
        res.update(extras)
        if not args.no_extras:
            res["cpu_baseline"] = cpu_baseline()
        print(json.dumps(res), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


def measured_traffic(kernel, frames_per_launch, table=None):
    """Per-launch DRAM traffic (or warp instructions, from INSTR) from the ncu capture, or None once the kernel's
    source changed."""
    import hashlib
    ent = (TRAFFIC if table is None else table).get(kernel)
    if ent is None:
        return None
    per_frame, rel, sha = ent
    path = os.path.join(ROOT, "paper_2606_05650_gb300", rel)
    try:
        with open(path, "rb") as f:
            if hashlib.sha1(f.read()).hexdigest() != sha:
                return None
    except OSError:
        return None
    return int(per_frame * frames_per_launch)


def roofline(stages, frames, nv_frames, stream_bytes, steps, F, hbm, src, issue_peak=None):
    """Dominant kernel of the step with its algorithmic bytes per launch; issue_peak (warp instructions per
    second: SMs x 4 schedulers x maximum SM clock) adds the issue-rate fraction of the kernels in INSTR."""
    n_in = sum(p.shape[0] for p, _ in frames)
    nv = int(nv_frames.sum())
    comp = int(stream_bytes.sum())
    # algorithmic bytes per launch (all F frames of one step are one launch)
    alg = {
        # cluster average gathered from the N x C input, N_v x C coefficients written
        "raht_forward_pass0": 4 * C * (n_in + nv),
        # dequantised coefficients read, attributes written
        "raht_inverse_pass0": 4 * C * (nv + nv),
        # coefficients read, compressed attribute payload written
        "rlgr_encode": 4 * C * nv + comp,
        # compressed payload read, dequantised coefficients written (per frame launch)
        "rlgr_decode": comp + 4 * C * nv,
    }
    # The dominant kernel is the one with the largest share of serialised GPU time in the ncu launch list of
    # this workload: event times of the stages on the two concurrent branches include the other branch's use of
    # the SMs, so the largest event time need not be the largest kernel.
    best = DOMINANT if stages.get(DOMINANT, (0.0, 0))[1] else None
    if best is None:
        best_ms = -1.0
        for k in alg:
            ms, cnt = stages.get(k, (0.0, 0))
            if cnt and ms > best_ms:
                best, best_ms = k, ms
    if best is None:
        return None
    ms, cnt = stages[best]
    launches_per_step = cnt / steps
    bytes_per_launch = alg[best] / launches_per_step
    avg_ms = ms / cnt
    ach = bytes_per_launch / (avg_ms / 1e3) / 1e9
    return {"kernel": best, "selected_by": "largest share of serialised GPU time (ncu launch list)",
            "bound": "hbm", "achieved": round(ach, 1), "peak": hbm, "unit": "GB/s",
            "frac": round(ach / hbm, 4), "peak_source": f"{src} hbm_gbs (MEASURED_PEAKS.json)",
            "traffic": measured_traffic(best, F / launches_per_step), "bytes_per_launch": int(bytes_per_launch),
            "avg_launch_ms": round(avg_ms, 4),
            "all": {k: per_kernel(k, stages, alg, steps, F, hbm, issue_peak) for k in alg if stages.get(k, (0, 0))[1]}}


# Algorithmic bytes per Gaussian of each timed stage (the compulsory reads and writes of the stage at C channels
# of 4 bytes), and whether the stage runs on one of the two concurrent branches of a call, where its event time
# includes the other branch's use of the SMs (a lower bound on the stage's own rate).
def stage_bytes(C, J):
    passes = (3 * J + 7) // 8
    return {
        "voxelize": (36, False),             # positions read twice (box, codes), codes and indices written
        "sort": (24 * passes, False),        # per 8-bit digit pass: 12-byte pairs read and written
        "dedup": (29, False),                # sorted codes read; voxel codes, first rows, segments written
        "occupancy": (16, True),             # codes and gap levels read, occupancy bytes written
        "rans": (9.5, True),                 # occupancy bytes read, compressed occupancy written
        "raht_prelude": (48, True),          # encoder and decoder schedules, 24 bytes each
        "raht_forward": (8 * C, True),       # rows gathered and coefficient rows written
        "rlgr_encode": (4 * C + 32, True),   # coefficients read, attribute payload written
        "container": (66, False),            # both sections read and written once
        "occupancy_decode": (9.5, True),     # compressed occupancy read, occupancy bytes written
        "octree_decode": (131, True),        # levels of nodes and the voxel centres
        "rlgr_decode": (32 + 4 * C, True),   # payload read, dequantised coefficients written
        "raht_inverse": (8 * C, True),       # coefficient rows read, attribute rows written
    }


def stage_roofline(stages, n_gauss, steps, hbm, C, J):
    """Per-stage algorithmic GB/s and fraction of the HBM peak from the stages' event times."""
    out = {}
    for k, (per, conc) in stage_bytes(C, J).items():
        ms, cnt = stages.get(k, (0.0, 0))
        if not cnt or ms <= 0:
            continue
        b = per * n_gauss
        gbs = b / (ms / steps / 1e3) / 1e9
        out[k] = {"ms_per_step": round(ms / steps, 4), "bytes_per_step": int(b), "GBs": round(gbs, 1),
                  "frac": round(gbs / hbm, 4), "branch": "concurrent" if conc else "serial"}
    return out


def per_kernel(k, stages, alg, steps, F, hbm, issue_peak):
    ms = stages[k][0] / stages[k][1]
    per_step = stages[k][1] / steps
    gbs = alg[k] / per_step / (ms / 1e3) / 1e9
    ent = {"ms_per_launch": round(ms, 4), "GBs": round(gbs, 1), "frac": round(gbs / hbm, 4)}
    inst = measured_traffic(k, F / per_step, INSTR)
    if inst is not None and issue_peak:
        ent["issue"] = {"warp_inst_per_launch": inst, "warp_inst_per_s": round(inst / (ms / 1e3) / 1e12, 4),
                        "unit": "T/s", "peak": round(issue_peak / 1e12, 4), "frac": round(inst / (ms / 1e3) / issue_peak, 4)}
    return ent


def gpu_extras(args, G, torch, P, A, frames, qp, out, offs, dev, stream):
    """Plain one-frame-at-a-time path (fps, p50/p99), batched encode-only and
    decode-only rates, and the end-to-end rate through host buffers."""
    import numpy as np
    F = len(P)
    res = {}
    # batched encode only / decode only
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    K = max(2, min(args.steps, 5))
    ev[0].record(stream)
    for _ in range(K):
        out, offs = G.encode_batch(P, A, [J] * F, [1.0], qp, out=out)
    ev[1].record(stream)
    for _ in range(K):
        G.decode_batch(out, offs, C, F * N_GAUSS)
    ev[2].record(stream)
    torch.cuda.synchronize()
    res["batched"] = {"encode_fps": round(F * K / (ev[0].elapsed_time(ev[1]) / 1e3), 2),
                      "decode_fps": round(F * K / (ev[1].elapsed_time(ev[2]) / 1e3), 2)}
    # plain path, one frame per call
    enc_ms, dec_ms = [], []
    buf = torch.empty(G.max_bitstream_bytes(N_GAUSS, J, qp), dtype=torch.uint8, device=dev)
    with _no_gc():
        for rep in range(2):
            for f in range(F):
                a, b, c = (torch.cuda.Event(enable_timing=True) for _ in range(3))
                a.record(stream)
                bs, nv, _, _ = G.encode_frame(P[f], A[f], J, qp, out=buf)
                b.record(stream)
                G.decode_frame(bs)
                c.record(stream)
                torch.cuda.synchronize()
                if rep:
                    enc_ms.append(a.elapsed_time(b))
                    dec_ms.append(b.elapsed_time(c))
    q = lambda v, p: float(np.percentile(v, p))
    res["plain"] = {"encode_fps": round(1e3 / statistics.mean(enc_ms), 2),
                    "decode_fps": round(1e3 / statistics.mean(dec_ms), 2),
                    "encode_decode_fps": round(1e3 / (statistics.mean(enc_ms) + statistics.mean(dec_ms)), 2),
                    "encode_ms_p50": round(q(enc_ms, 50), 3), "encode_ms_p99": round(q(enc_ms, 99), 3),
                    "decode_ms_p50": round(q(dec_ms, 50), 3), "decode_ms_p99": round(q(dec_ms, 99), 3)}
    # encoder reconstruction (the decoded frame returned by the encode call itself): plain encode with it
    trec = _timed_calls(torch, stream, lambda k=0: G.encode_frame(P[k % F], A[k % F], J, qp, out=buf, recon=True), F)
    res["plain"]["encode_with_reconstruction_ms_p50"] = round(q(trec, 50), 3)
    # differentiable codec layer: 500,000 Gaussians at depth 16, forward
    # A_hat = T^T(step q(T A)) and its straight-through backward T^T T g
    from paper_2606_05650_gb300 import synthetic as syn
    p5, _ = syn.DynamicScene(4000).frame(0, n=500_000)
    codes5, _, _ = G.voxelize(torch.from_numpy(p5).to(dev), J)
    plan5 = G.RahtPlan(codes5, J, C)
    a5 = torch.randn(codes5.shape[0], C, device=dev, requires_grad=True)
    g5 = torch.randn_like(a5)
    fwd, bwd = [], []
    for it in range(8):
        x, y, z = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        x.record(stream)
        rec = G.AttrCodecFn.apply(a5, plan5, qp)
        y.record(stream)
        rec.backward(g5)
        z.record(stream)
        torch.cuda.synchronize()
        a5.grad = None
        if it >= 3:
            fwd.append(x.elapsed_time(y))
            bwd.append(y.elapsed_time(z))
    nv5 = int(codes5.shape[0])
    res["codec_layer"] = {"gaussians": 500_000, "voxels": nv5, "depth": J, "channels": C,
                          "forward_ms": round(statistics.median(fwd), 3),
                          "backward_ms": round(statistics.median(bwd), 3),
                          "backward_over_forward": round(statistics.median(bwd) / statistics.median(fwd), 3),
                          "forward_GBs": round(16 * C * nv5 / (statistics.median(fwd) / 1e3) / 1e9, 1)}
    del plan5
    # colour decorrelation (Sec. 4) on a 1M-Gaussian frame with correlated SH colours: size and RGB PSNR
    from oracle import oracle as orc
    from paper_2606_05650_gb300 import synthetic as syn
    pc, _ = frames[0]
    ac = syn.gs_attributes_correlated_sh(np.random.default_rng(77), pc.shape[0])
    _, merged, *_ = orc.voxelize(pc, ac, J)
    dpc, dac = torch.from_numpy(pc).to(dev), torch.from_numpy(ac).to(dev)
    colour = {}
    for name, col, sc in (("rgb", False, 1.0), ("yuv_klt", True, 1.0), ("yuv_klt_steps_x0.66", True, 0.66)):
        qcol = G.QuantParams(syn.gs_channel_groups(), np.array(syn.GS_BASE_STEPS) * sc, color=col)
        t = _timed_calls(torch, stream, lambda _=0: G.encode_frame(dpc, dac, J, qcol), 3)
        bsc, *_ = G.encode_frame(dpc, dac, J, qcol)
        td = _timed_calls(torch, stream, lambda _=0: G.decode_frame(bsc), 3)
        _, dec = G.decode_frame(bsc)
        err = (dec.cpu().numpy().astype(np.float64) - merged) ** 2
        sh = err[:, 8:].mean()
        colour[name] = {"bytes": int(bsc.numel()), "bits_per_gaussian": round(8 * bsc.numel() / pc.shape[0], 2),
                        "sh_rgb_psnr_db": round(float(10 * np.log10(1.0 / sh)), 2),
                        "encode_ms": round(statistics.median(t), 3), "decode_ms": round(statistics.median(td), 3)}
    colour["size_ratio_rgb_over_klt"] = round(colour["rgb"]["bytes"] / colour["yuv_klt"]["bytes"], 3)
    colour["size_ratio_rgb_over_klt_x0.66"] = round(colour["rgb"]["bytes"] / colour["yuv_klt_steps_x0.66"]["bytes"], 3)
    res["colour_decorrelation"] = colour
    # level of detail: one 1M-Gaussian stream decoded to depths 16, 12, 8
    s0 = out[int(offs[0]):int(offs[1])].clone()
    lod = {}
    for depth in (J, 12, 8):
        t = _timed_calls(torch, stream, lambda _=0: G.decode_frame_lod(s0, depth), 10)
        n_nodes = G.decode_frame_lod(s0, depth)[0].shape[0]
        lod[str(depth)] = {"ms": round(statistics.median(t), 3), "nodes": int(n_nodes)}
    res["lod_decode"] = lod
    # rendered-view quality (Sec. 5.1): PSNR of renders of the decoded frame against renders of the
    # original Gaussians, 960 x 540 from 3 orbit views, per quantisation rung; and the rasteriser's own time
    views = syn.orbit_views(3, radius=1.2)
    Wr, Hr, fr = 960, 540, 1000.0
    p0, a0 = P[0], A[0]
    ref_imgs = [G.render(p0, a0, v, fr, fr, Wr / 2, Hr / 2, Wr, Hr).clamp_(0, 1) for v in views]
    img_buf = torch.empty((Hr, Wr, 3), dtype=torch.float32, device=dev)
    tr = _timed_calls(torch, stream, lambda _=0: G.render(p0, a0, views[0], fr, fr, Wr / 2, Hr / 2, Wr, Hr,
                                                          out=img_buf), 5)
    rq = {"gaussians": int(p0.shape[0]), "views": len(views), "image": [Wr, Hr],
          "render_ms": round(statistics.median(tr), 3), "rungs": []}
    for sc in (0.5, 1.0, 2.0, 4.0):
        qr = G.QuantParams(syn.gs_channel_groups(), np.array(syn.GS_BASE_STEPS) * sc)
        bsr, *_ = G.encode_frame(p0, a0, J, qr)
        dpos, datt = G.decode_frame(bsr)
        ps = []
        for v, ref in zip(views, ref_imgs):
            img = G.render(dpos, datt.contiguous(), v, fr, fr, Wr / 2, Hr / 2, Wr, Hr).clamp_(0, 1)
            mse = float(((img - ref) ** 2).mean())
            ps.append(10 * np.log10(1.0 / max(mse, 1e-20)))
        rq["rungs"].append({"step_scale": sc, "bits_per_gaussian": round(8 * bsr.numel() / p0.shape[0], 2),
                            "psnr_db": round(float(np.mean(ps)), 2)})
    res["rendered_quality"] = rq
    # end to end: pinned host inputs -> H2D -> encode -> D2H streams -> decode -> D2H frames
    hp = [torch.from_numpy(p).pin_memory() for p, _ in frames]
    ha = [torch.from_numpy(a).pin_memory() for _, a in frames]
    dp = [torch.empty_like(x, device=dev) for x in hp]
    da = [torch.empty_like(x, device=dev) for x in ha]
    total = int(offs[-1])
    hout = torch.empty(out.numel(), dtype=torch.uint8).pin_memory()
    hpos = torch.empty((F * N_GAUSS, 3), dtype=torch.float32).pin_memory()
    hatt = torch.empty((F * N_GAUSS, C), dtype=torch.float32).pin_memory()

    pos1 = torch.empty((F * N_GAUSS, 3), dtype=torch.float32, device=dev)
    att1 = torch.empty((F * N_GAUSS, C), dtype=torch.float32, device=dev)

    def e2e_step():
        for x, y in zip(hp + ha, dp + da):
            y.copy_(x, non_blocking=True)
        o, off = G.encode_batch(dp, da, [J] * F, [1.0], qp, out=out)
        n = int(off[-1])
        hout[:n].copy_(o[:n], non_blocking=True)
        pos, attr, rows = G.decode_batch(o, off, C, F * N_GAUSS, pos_out=pos1, attr_out=att1)
        m = int(rows[-1])
        hpos[:m].copy_(pos, non_blocking=True)
        hatt[:m].copy_(attr, non_blocking=True)
        torch.cuda.synchronize()
        return n, m

    e2e_step()
    t0 = time.perf_counter()
    K2 = max(2, min(args.steps, 5))
    for _ in range(K2):
        n, m = e2e_step()
    dt_serial = (time.perf_counter() - t0) / K2
    K3 = max(6, min(args.steps, 96))  # as many steps as the headline loop: filling and draining the pipeline
    # (about two steps) is then a small part
    dt, n, m, timeline = e2e_streamed(G, torch, dev, qp, F, hp, ha, dp, da, out, pos1, att1, hout, hpos, hatt, K3)
    h2d = sum(x.numel() * 4 for x in hp + ha)
    d2h = n + m * (3 + C) * 4
    res["e2e"] = {"value": round(F / dt, 2), "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                  "d2h_bytes_per_step": int(d2h), "ms_per_step": round(dt * 1e3, 3), "steps": K3,
                  "mode": "streamed: uploads, coding and downloads of consecutive steps overlap (3 buffer sets; "
                          "encoder returns header records, decoder asynchronous)",
                  "timeline": timeline,
                  "serial": {"value": round(F / dt_serial, 2), "ms_per_step": round(dt_serial * 1e3, 3)}}
    return res


def e2e_streamed(G, torch, dev, qp, F, hp, ha, dp, da, out, pos1, att1, hout, hpos, hatt, steps, chunk=1 << 24, NB=3):
    """End-to-end streamed loop through the public API: pinned host inputs -> H2D -> batched encode -> batched
    decode -> D2H of the streams and the decoded frames, every step.  The encoder hands back the streams' header
    records with its offsets (gsnfs_encode_batch_headers), so the decoder (gsnfs_decode_batch_async) reads nothing
    back and does not block; the only host read of a step is the encoder's own, at its end.  A step's results go
    down right after the next step's encoder has read back (a small device-to-host read queues behind a bulk
    download on the link, so no bulk download is in flight while the encoder reads back, except the one being
    overtaken); the upload of step k+1 overlaps everything.  NB sets of device buffers: step k reuses those of step
    k-NB.  Copies are issued in pieces of `chunk` elements.  Returns (seconds per step, stream bytes, voxel rows,
    timeline of the steady steps); decode statuses are checked after the loop."""
    import time
    s_in, s_cmp, s_out = torch.cuda.Stream(dev), torch.cuda.Stream(dev), torch.cuda.Stream(dev)
    dpN = [dp] + [[torch.empty_like(x) for x in dp] for _ in range(NB - 1)]
    daN = [da] + [[torch.empty_like(x) for x in da] for _ in range(NB - 1)]
    outN = [out] + [torch.empty_like(out) for _ in range(NB - 1)]
    posN = [pos1] + [torch.empty((F * N_GAUSS, 3), dtype=torch.float32, device=dev) for _ in range(NB - 1)]
    attN = [att1] + [torch.empty((F * N_GAUSS, C), dtype=torch.float32, device=dev) for _ in range(NB - 1)]
    ev_in = [torch.cuda.Event() for _ in range(NB)]
    ev_cmp = [torch.cuda.Event() for _ in range(NB)]
    ev_out = [torch.cuda.Event() for _ in range(NB)]
    status = torch.full((steps + 8,), -1, dtype=torch.int32, device=dev)
    tl = []  # per step: timing events of the three streams and host seconds spent in the coding calls

    def chunked(dst, src):
        d, s_ = dst.view(-1), src.view(-1)
        for i in range(0, d.numel(), chunk):
            d[i:i + chunk].copy_(s_[i:i + chunk], non_blocking=True)

    def tev():
        return torch.cuda.Event(enable_timing=True)

    def upload(k, rec):
        b = k % NB
        with torch.cuda.stream(s_in):
            s_in.wait_event(ev_cmp[b])  # step k-NB has finished reading these inputs
            rec["up"] = (tev(), tev())
            rec["up"][0].record(s_in)
            for x, y in zip(hp + ha, dpN[b] + daN[b]):
                chunked(y, x)
            rec["up"][1].record(s_in)
            ev_in[b].record(s_in)

    def download(k, rec, n, m):
        b = k % NB
        with torch.cuda.stream(s_out):
            s_out.wait_event(ev_cmp[b])
            rec["down"] = (tev(), tev())
            rec["down"][0].record(s_out)
            chunked(hout[:n], outN[b][:n])
            chunked(hpos[:m], posN[b][:m])
            chunked(hatt[:m], attN[b][:m])
            rec["down"][1].record(s_out)
            ev_out[b].record(s_out)

    def streamed(K, base):
        recs = [dict() for _ in range(K)]
        upload(0, recs[0])
        prev = None
        n = m = 0
        for k in range(K):
            if k + 1 < K:
                upload(k + 1, recs[k + 1])
            b = k % NB
            h0 = time.perf_counter()
            with torch.cuda.stream(s_cmp):
                s_cmp.wait_event(ev_in[b])
                s_cmp.wait_event(ev_out[b])  # step k-NB's results have left these buffers
                recs[k]["code"] = (tev(), tev())
                recs[k]["code"][0].record(s_cmp)
                o, off, hdr = G.encode_batch(dpN[b], daN[b], [J] * F, [1.0], qp, out=outN[b], headers=True)
            if prev is not None:
                download(*prev)
            with torch.cuda.stream(s_cmp):
                rows = G.decode_batch_async(o, off, hdr, C, F * N_GAUSS, posN[b], attN[b],
                                            status[base + k:base + k + 1])
                recs[k]["code"][1].record(s_cmp)
                ev_cmp[b].record(s_cmp)
            recs[k]["host_in_calls_s"] = time.perf_counter() - h0
            n, m = int(off[-1]), int(rows[-1])
            prev = (k, recs[k], n, m)
        download(*prev)
        torch.cuda.synchronize()
        tl[:] = recs
        return n, m

    streamed(3, 0)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    n, m = streamed(steps, 3)
    dt = (time.perf_counter() - t0) / steps
    st = status[:3 + steps].cpu().tolist()
    if any(v != 0 for v in st):
        raise RuntimeError(f"asynchronous decode reported status {st}")
    # timeline of the timed steps (skipping the first two, which fill the pipeline)
    zero = tl[0]["up"][0]
    span = lambda ev: (zero.elapsed_time(ev[0]), zero.elapsed_time(ev[1]))
    steady = tl[2:]
    mean = lambda xs: round(float(sum(xs) / max(len(xs), 1)), 3)
    timeline = {"steps_summarised": len(steady),
                "upload_ms": mean([span(r["up"])[1] - span(r["up"])[0] for r in steady]),
                "coding_ms": mean([span(r["code"])[1] - span(r["code"])[0] for r in steady]),
                "download_ms": mean([span(r["down"])[1] - span(r["down"])[0] for r in steady]),
                "coding_start_interval_ms": mean([span(b_["code"])[0] - span(a_["code"])[0]
                                                  for a_, b_ in zip(steady, steady[1:])]),
                "host_ms_in_coding_calls": mean([1e3 * r["host_in_calls_s"] for r in steady]),
                "link_floor_ms": round((sum(x.numel() * 4 for x in hp + ha) + n + m * (3 + C) * 4) / 340e9 * 1e3, 3),
                "note": "link_floor_ms: the step's bytes at the 340 GB/s measured for uploads and downloads at once"}
    return dt, n, m, timeline


def ladder_leg(G, torch, dev, stream, frames, Js, block, idx):
    """Batched against plain on the bandwidth ladder: the given frames (a spread of the 64-frame ladder's sizes
    and depths) each at 5 quantisation rungs (steps x 1, 2, 4, 8, 16).  Encode: one batched call for all frames
    and rungs (with and without CUDA-graph replay) against one plain call per frame and rung.  Decode: batched
    calls over all streams (at most 64 per call) against one plain call per stream.  The two paths write
    byte-identical streams (checked by total size here and byte by byte in the tests)."""
    import numpy as np
    from paper_2606_05650_gb300 import synthetic as syn
    scales = [float(x) for x in syn.LADDER_RUNG_SCALES]
    P = [torch.from_numpy(p).to(dev) for p, _ in frames]
    A = [torch.from_numpy(a).to(dev) for _, a in frames]
    F, R = len(P), len(scales)
    total_n = sum(int(p.shape[0]) for p in P)
    qp = G.QuantParams(syn.gs_channel_groups(), syn.GS_BASE_STEPS, rlgr_block=block, rans_chunk=RANS_CHUNK)
    st = {"out": torch.empty(int(total_n * C * 2 * R), dtype=torch.uint8, device=dev)}

    def batched(_=0):
        st["out"], st["offs"] = G.encode_batch(P, A, Js, scales, qp, out=st["out"])

    res = {"frames": F, "rungs": R, "ladder_frame_ids": idx, "gaussians": total_n,
           "gaussians_min_max": [min(int(p.shape[0]) for p in P), max(int(p.shape[0]) for p in P)],
           "depths": sorted(set(int(j) for j in Js))}
    for graphs in (False, True):
        G.set_graphs(graphs)
        ms = float(np.median(_timed_calls(torch, stream, batched, 5)))
        res["batched_graphs_encode_ms" if graphs else "batched_encode_ms"] = round(ms, 3)
    G.set_graphs(False)
    out, offs = st["out"], st["offs"]
    qps = [G.QuantParams(syn.gs_channel_groups(), np.array(syn.GS_BASE_STEPS) * sc, rlgr_block=block,
                         rans_chunk=RANS_CHUNK) for sc in scales]
    buf = torch.empty(max(G.max_bitstream_bytes(int(p.shape[0]), j, qp) for p, j in zip(P, Js)), dtype=torch.uint8,
                      device=dev)
    plain_bytes = [0]

    def plain(_=0):
        tot = 0
        for f in range(F):
            for r in range(R):
                bs, *_ = G.encode_frame(P[f], A[f], Js[f], qps[r], out=buf)
                tot += int(bs.numel())
        plain_bytes[0] = tot

    plain_enc = float(np.median(_timed_calls(torch, stream, plain, 2)))
    # decode: batched over contiguous runs of at most 64 streams, against one call per stream
    nstreams = F * R
    rows_cap = total_n * R
    pos_o = torch.empty((rows_cap, 3), dtype=torch.float32, device=dev)
    att_o = torch.empty((rows_cap, C), dtype=torch.float32, device=dev)

    def batched_dec(_=0):
        for k0 in range(0, nstreams, 64):
            sub = offs[k0:min(k0 + 64, nstreams) + 1]
            G.decode_batch(out, sub, C, rows_cap, pos_out=pos_o, attr_out=att_o)

    streams = [out[int(offs[k]):int(offs[k + 1])] for k in range(nstreams)]

    def plain_dec(_=0):
        for b in streams:
            G.decode_frame(b)

    bdec = float(np.median(_timed_calls(torch, stream, batched_dec, 3)))
    pdec = float(np.median(_timed_calls(torch, stream, plain_dec, 2)))
    benc = res["batched_graphs_encode_ms"]
    res.update({
        "plain_per_rung_encode_ms": round(plain_enc, 3),
        "batched_decode_ms": round(bdec, 3), "plain_per_stream_decode_ms": round(pdec, 3),
        # frames/s with each frame at all 5 rungs
        "batched_fps": round(F / (benc / 1e3), 2), "plain_per_rung_fps": round(F / (plain_enc / 1e3), 2),
        "batched_encode_decode_fps": round(F / ((benc + bdec) / 1e3), 2),
        "plain_encode_decode_fps": round(F / ((plain_enc + pdec) / 1e3), 2),
        "batched_over_plain_encode": round(plain_enc / benc, 3),
        "batched_over_plain_encode_decode": round((plain_enc + pdec) / (benc + bdec), 3),
        "bytes_all_rungs": int(offs[-1]), "plain_bytes_all_rungs": plain_bytes[0],
        "bytes_equal": int(offs[-1]) == plain_bytes[0],
        "sample": f"{F} of the 64 ladder frames (evenly spaced ranks of the sorted sizes), all {R} rungs"})
    return res


def sequence_leg(G, torch, dev, stream, frames, block):
    """The dynamic 3DGS sequence (every 10th of 300 frames of ~250k Gaussians, depth 16, base steps): plain
    one-frame encode and decode latency (p50/p99 over the frames) and frames/s, against one batched encode
    call and one batched decode call for all frames."""
    import numpy as np
    from paper_2606_05650_gb300 import synthetic as syn
    P = [torch.from_numpy(p).to(dev) for p, _ in frames]
    A = [torch.from_numpy(a).to(dev) for _, a in frames]
    F = len(P)
    qp = G.QuantParams(syn.gs_channel_groups(), syn.GS_BASE_STEPS, rlgr_block=block, rans_chunk=RANS_CHUNK)
    nmax = max(int(p.shape[0]) for p in P)
    buf = torch.empty(G.max_bitstream_bytes(nmax, J, qp), dtype=torch.uint8, device=dev)
    enc, dec = [], []
    with _no_gc():
        for rep in range(2):
            for f in range(F):
                a, b, c = (torch.cuda.Event(enable_timing=True) for _ in range(3))
                a.record(stream)
                bs, nv, _, _ = G.encode_frame(P[f], A[f], J, qp, out=buf)
                b.record(stream)
                G.decode_frame(bs)
                c.record(stream)
                torch.cuda.synchronize()
                if rep:
                    enc.append(a.elapsed_time(b))
                    dec.append(b.elapsed_time(c))
    n_tot = sum(int(p.shape[0]) for p in P)
    st = {"out": None}

    def batched(_=0):
        st["out"], offs = G.encode_batch(P, A, [J] * F, [1.0], qp, out=st["out"])
        G.decode_batch(st["out"], offs, C, n_tot)

    bt = float(np.median(_timed_calls(torch, stream, batched, 3)))
    pct = lambda v, q: round(float(np.percentile(v, q)), 3)
    return {"frames": F, "gaussians_per_frame_mean": round(n_tot / F), "depth": J,
            "encode_ms_p50": pct(enc, 50), "encode_ms_p99": pct(enc, 99),
            "decode_ms_p50": pct(dec, 50), "decode_ms_p99": pct(dec, 99),
            "plain_encode_decode_fps": round(1e3 / (float(np.mean(enc)) + float(np.mean(dec))), 2),
            "batched_encode_decode_fps": round(F / (bt / 1e3), 2),
            "batched_over_plain": round((float(np.mean(enc)) + float(np.mean(dec))) * F / bt, 3),
            "sample": f"frames 0, 10, ..., {10 * (F - 1)} of the 300-frame sequence"}


# ------------------------------------------------------------ CPU oracle
def _oracle_code(pos, attr):
    """Encode + decode of one frame by the FP64 oracle (one core); seconds."""
    from oracle import oracle as orc
    from paper_2606_05650_gb300 import synthetic as syn
    t0 = time.perf_counter()
    r = orc.encode_frame(pos, attr, J, syn.gs_channel_groups(), syn.GS_BASE_STEPS, block=512, chunk_syms=RANS_CHUNK)
    orc.decode_frame(r["bitstream"])
    return time.perf_counter() - t0


def _oracle_worker(seed_ts, q_in, q_out):
    """Reference-arm process: generates its frames once, then codes all of them on each request."""
    sys.path.insert(0, ROOT)
    frames = [_headline_frame(st) for st in seed_ts]
    q_out.put(("ready", 0.0))
    while q_in.get() is not None:
        q_out.put(("done", sum(_oracle_code(p, a) for p, a in frames)))


def host_cpu():
    """Host CPU description for the baseline: logical cores and the model line of /proc/cpuinfo (or the
    implementer / part ids on Arm hosts that print no model name)."""
    info = {"nproc": os.cpu_count()}
    try:
        with open("/proc/cpuinfo") as f:
            lines = f.read().splitlines()
    except OSError:
        return info
    kv = {}
    for ln in lines:
        if ":" in ln:
            k, v = ln.split(":", 1)
            kv.setdefault(k.strip(), v.strip())
    for k in ("model name", "Model", "Hardware"):
        if kv.get(k):
            info["model"] = kv[k]
            return info
    if kv.get("CPU implementer"):
        info["model"] = f"implementer {kv['CPU implementer']} part {kv.get('CPU part', '?')}"
    return info


def cpu_baseline():
    """The oracle as it stands, one 1M-Gaussian frame of the headline scene on one host core."""
    from oracle import oracle as orc
    orc.build()
    pos, attr = _headline_frame((1000, 0))
    dt = _oracle_code(pos, attr)
    return {"value": round(1.0 / dt, 4), "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"1 frame of {N_GAUSS} Gaussians (encode + decode, FP64 C oracle, single thread), {dt:.1f} s",
            "host": host_cpu()}


def run_reference(args):
    """Comparison arm: the FP64 oracle on the host cores, the headline workload itself.  Each step encodes and
    decodes the same F frames the GPU arm codes, one whole frame per process and all of them in parallel
    (processes = min(F, host cores); with fewer cores than frames a process codes several)."""
    rank, world, local = dist_env()
    if rank != 0:
        return
    import multiprocessing as mp
    from oracle import oracle as orc
    orc.build()
    F = args.frames
    workers = max(1, min(F, os.cpu_count() or 1))
    ctx = mp.get_context("spawn")
    q_out = ctx.Queue()
    qs, procs = [], []
    for w in range(workers):
        q = ctx.Queue()
        pr = ctx.Process(target=_oracle_worker, args=([(1000, t) for t in range(w, F, workers)], q, q_out),
                         daemon=True)
        pr.start()
        qs.append(q)
        procs.append(pr)
    for _ in range(workers):
        q_out.get()  # frames generated (not timed)

    def step():
        for q in qs:
            q.put(1)
        return sum(q_out.get()[1] for _ in range(workers))

    # every step codes the whole headline workload (about 3 s on 16 cores), so the timed steps are capped to keep
    # the arm within a few minutes; the line reports the counts it ran
    K, W = min(args.steps, REF_MAX_STEPS), min(args.warmup, 3)
    for _ in range(W):
        step()
    t0 = time.perf_counter()
    busy = 0.0
    for _ in range(K):
        busy += step()
    dt = time.perf_counter() - t0
    for q in qs:
        q.put(None)
    for pr in procs:
        pr.join(timeout=30)
    value = F * K / dt
    sample = (f"the headline workload itself: each step encodes + decodes all {F} frames of {N_GAUSS} Gaussians "
              f"(FP64 C oracle), one whole frame per process, {workers} processes in parallel; "
              f"{busy / (F * K):.2f} s of one core per frame; {K} timed steps of the {args.steps} requested")
    res = {"metric": METRIC, "value": round(value, 4), "unit": UNIT, "n_gpus": args.gpus, "steps": K,
           "warmup": W, "ms_per_step": round(dt / K * 1e3, 1), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
           "config": headline_config(F, args.block, 1),
           "cpu_baseline": {"value": round(value, 4), "unit": UNIT, "cores": workers, "kind": "oracle",
                            "sample": sample, "host": host_cpu()},
           "e2e": {"value": round(value, 4), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(res), flush=True)


def run_ladder(args):
    """64 frames with log-uniform sizes in [50k, 2M] and depths 16/17/18, each
    encoded at 5 rungs (steps x 1, 2, 4, 8, 16): one batched call (frames x
    rungs, with and without CUDA graphs) against the plain path (one call per
    frame and rung, and one multi-rung call per frame)."""
    import numpy as np
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2606_05650_gb300 import gsnfs as G, synthetic as syn
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    sizes, depths = syn.ladder_sizes(3000)
    scales = [float(x) for x in syn.LADDER_RUNG_SCALES]
    scene = syn.DynamicScene(3000)
    P, A = [], []
    for f, n in enumerate(sizes):
        p, a = scene.frame(f, n=int(n))
        P.append(torch.from_numpy(p).to(dev))
        A.append(torch.from_numpy(a).to(dev))
    F, R = len(P), len(scales)
    qp = G.QuantParams(syn.gs_channel_groups(), syn.GS_BASE_STEPS, rlgr_block=args.block)
    Js = [int(j) for j in depths]
    stream = torch.cuda.current_stream(dev)
    total_n = int(sizes.sum())
    # capacity: a generous estimate, grown by the binding if a call needs more
    out = torch.empty(int(total_n * C * 2 * R), dtype=torch.uint8, device=dev)

    def timed(fn, reps):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    res = {}
    sizes_out = {}

    def batched():
        nonlocal out
        out, offs = G.encode_batch(P, A, Js, scales, qp, out=out)
        sizes_out["batched"] = int(offs[-1])

    for graphs in (False, True):
        G.set_graphs(graphs)
        ms = timed(batched, max(2, min(args.steps, 5)))
        res["batched_graphs" if graphs else "batched"] = {"ms": round(ms, 2), "frames_per_s": round(F / (ms / 1e3), 1),
                                                          "gaussians_per_s": round(total_n / (ms / 1e3), 0)}
    buf = torch.empty(max(G.max_bitstream_bytes(int(n), int(j), qp) for n, j in zip(sizes, depths)),
                      dtype=torch.uint8, device=dev)
    qps = [G.QuantParams(syn.gs_channel_groups(), np.array(syn.GS_BASE_STEPS) * sc, rlgr_block=args.block)
           for sc in scales]
    plain_bytes = [0]

    def plain():
        tot = 0
        for f in range(F):
            for r in range(R):
                bs, *_ = G.encode_frame(P[f], A[f], Js[f], qps[r], out=buf)
                tot += bs.numel()
        plain_bytes[0] = tot

    for graphs in (False, True):
        G.set_graphs(graphs)
        ms = timed(plain, 1)
        res["plain_per_rung_graphs" if graphs else "plain_per_rung"] = {
            "ms": round(ms, 2), "frames_per_s": round(F / (ms / 1e3), 1),
            "gaussians_per_s": round(total_n / (ms / 1e3), 0)}
    G.set_graphs(False)
    o1 = torch.empty(int(sizes.max()) * C * 2 * R, dtype=torch.uint8, device=dev)

    def plain_multi():
        nonlocal o1
        for f in range(F):
            o1, _ = G.encode_batch([P[f]], [A[f]], [Js[f]], scales, qp, out=o1)

    ms = timed(plain_multi, 1)
    res["plain_multirung"] = {"ms": round(ms, 2), "frames_per_s": round(F / (ms / 1e3), 1),
                              "gaussians_per_s": round(total_n / (ms / 1e3), 0)}
    # rate-distortion: the same batched call returning per-stream distortion, hull and budgeted choice
    from paper_2606_05650_gb300 import rd
    G.set_graphs(False)
    st_rd = {}

    def batched_rd():
        st_rd["r"] = G.encode_batch(P, A, Js, scales, qp, out=out, distortion=True)

    res["batched_with_distortion"] = {"ms": round(timed(batched_rd, 2), 2)}
    o_rd, offs_rd, dist = st_rd["r"]
    rate = np.diff(offs_rd.astype(np.int64)).reshape(F, R)
    nvox = np.array([G.peek_frame(o_rd[int(offs_rd[f * R]):int(offs_rd[f * R]) + 96].cpu().numpy())[0]
                     for f in range(F)])
    psnr = rd.psnr(dist, nvox)
    budget = rate[:, 2]  # e.g. the x4 rung's size
    sel = rd.select(rate, psnr, budget)
    res["rd"] = {"psnr_db_mean_per_rung": [round(float(x), 2) for x in psnr.mean(0)],
                 "bits_per_gaussian_per_rung": [round(float(x), 2) for x in 8 * rate.sum(0) / total_n],
                 "hull_points_mean": round(float(np.mean([len(rd.upper_hull(rate[f], psnr[f])) for f in range(F)])), 2),
                 "selected_rung_histogram_at_x4_budget": np.bincount(sel, minlength=R).tolist()}
    # rendered-view PSNR (Sec. 5.1's measure) for the first frames: decoded streams rendered by the GPU
    # rasteriser from 2 orbit views (480 x 270) against the same views of the original Gaussians
    from paper_2606_05650_gb300 import synthetic as syn
    Fr = min(4, F)
    views = syn.orbit_views(2, radius=1.2)

    def render(p, a, v):
        return G.render(p, a.contiguous(), v, 500.0, 500.0, 240, 135, 480, 270)
    rq = np.zeros((Fr, R))
    for f in range(Fr):
        for r in range(R):
            i = f * R + r
            dp, da = G.decode_frame(o_rd[int(offs_rd[i]):int(offs_rd[i + 1])])
            rq[f, r] = rd.rendered_psnr(render, (P[f], A[f]), (dp, da), views)
    rsel = rd.select(rate[:Fr], rq, budget[:Fr])
    res["rd"]["rendered"] = {"frames": Fr, "views": len(views), "image": [480, 270],
                             "psnr_db_mean_per_rung": [round(float(x), 2) for x in rq.mean(0)],
                             "selected_rung_histogram_at_x4_budget": np.bincount(rsel, minlength=R).tolist()}
    line = {"metric": "ladder encode frames/s (each frame at 5 rungs)", "unit": "frames/s", "higher_is_better": True,
            "value": res["batched_graphs"]["frames_per_s"], "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"{F} dynamic 3DGS frames, Gaussians log-uniform in [50k, 2M] (total {total_n}), "
                                   f"depths 16/17/18, {C} channels, {R} rungs x{scales}",
                       "rlgr_block": args.block, "graph_stats": G.graph_stats()},
            "bytes_all_rungs": sizes_out["batched"], "plain_bytes_all_rungs": plain_bytes[0], "legs": res}
    print(json.dumps(line), flush=True)


class _no_gc:
    """Per-call latency legs run with Python's garbage collector collected beforehand and paused: a collection
    inside a timed call (the events bracket the host's enqueue and its wait) would be charged to the codec."""

    def __enter__(self):
        import gc
        gc.collect()
        self.was = gc.isenabled()
        gc.disable()

    def __exit__(self, *exc):
        import gc
        if self.was:
            gc.enable()
        return False


def _timed_calls(torch, stream, fn, reps):
    """Per-call device times (ms) of fn() on the stream, after one warm-up call."""
    fn()
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(reps + 1)]
    ev[0].record(stream)
    for k in range(reps):
        fn(k)
        ev[k + 1].record(stream)
    torch.cuda.synchronize()
    return [ev[k].elapsed_time(ev[k + 1]) for k in range(reps)]


def _gen_pc_frame(t):
    from paper_2606_05650_gb300 import synthetic as syn
    return syn.capsule_humanoids_frame(11, t, 1_000_000)


def _gen_seq_frame(t):
    from paper_2606_05650_gb300 import synthetic as syn
    return syn.DynamicScene(2000).frame(t)


def _gen_frames(fn, count):
    """Frames generated on the host cores by a spawned pool (before any GPU work)."""
    import multiprocessing as mp
    with mp.get_context("spawn").Pool(max(1, min(os.cpu_count() or 1, 16))) as pool:
        return pool.map(fn, range(count), chunksize=1)


def run_sequence(args, pointcloud=False):
    """A dynamic sequence coded frame by frame (intra only).  3DGS: 300 frames
    of ~250k Gaussians (+-10%), depth 16, 56 channels, steps x {1, 2, 4};
    point cloud: 150 frames of ~1M points on two capsule humanoids, depth 10,
    YCbCr, steps {0.025 ... 0.4}.  Reports per-frame encode and decode latency
    (p50/p99) of the plain path, the batched throughput over all frames, and
    for the point cloud the attribute PSNR per step."""
    import numpy as np
    Fn = args.seq_frames or (150 if pointcloud else 300)
    host_frames = _gen_frames(_gen_pc_frame if pointcloud else _gen_seq_frame, Fn)
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2606_05650_gb300 import gsnfs as G, synthetic as syn
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    if pointcloud:
        Jd, C = 10, 3
        qps = [G.QuantParams(np.zeros(3, np.uint8), [s]) for s in (0.025, 0.05, 0.1, 0.2, 0.4)]
    else:
        Jd, C = 16, 56
        qps = [G.QuantParams(syn.gs_channel_groups(), np.array(syn.GS_BASE_STEPS) * m) for m in (1.0, 2.0, 4.0)]
    P, A, n_tot = [], [], 0
    for p, a in host_frames:
        P.append(torch.from_numpy(p).to(dev))
        A.append(torch.from_numpy(a).to(dev))
        n_tot += p.shape[0]
    del host_frames
    nmax = max(int(p.shape[0]) for p in P)
    buf = torch.empty(G.max_bitstream_bytes(nmax, Jd, qps[0]), dtype=torch.uint8, device=dev)
    legs = []
    for qi, qp in enumerate(qps):
        enc, dec, sizes = [], [], []
        with _no_gc():
            for t in range(Fn):
                def e(_=0):
                    return G.encode_frame(P[t], A[t], Jd, qp, out=buf)
                enc += _timed_calls(torch, stream, e, 1)
                bs, nv, _, _ = e()
                sizes.append(int(bs.numel()))
                dec += _timed_calls(torch, stream, lambda _=0: G.decode_frame(bs), 1)
        leg = {"step_set": qi, "encode_ms_p50": round(float(np.percentile(enc, 50)), 3),
               "encode_ms_p99": round(float(np.percentile(enc, 99)), 3),
               "decode_ms_p50": round(float(np.percentile(dec, 50)), 3),
               "decode_ms_p99": round(float(np.percentile(dec, 99)), 3),
               "plain_encode_fps": round(1e3 / float(np.mean(enc)), 1),
               "plain_decode_fps": round(1e3 / float(np.mean(dec)), 1),
               "bytes_per_frame": int(np.mean(sizes)), "bits_per_point": round(8 * sum(sizes) / n_tot, 3)}
        if pointcloud:  # attribute PSNR of the decoded frames against the voxel means (peak 1)
            from oracle import oracle as orc
            psnr = []
            for t in range(min(Fn, 3)):
                bs, nv, _, _ = G.encode_frame(P[t], A[t], Jd, qp, out=buf)
                gp, ga = G.decode_frame(bs)
                _, merged, *_ = orc.voxelize(P[t].cpu().numpy(), A[t].cpu().numpy(), Jd)
                mse = ((ga.cpu().numpy().astype(np.float64) - merged) ** 2).mean(0)
                psnr.append(10 * np.log10(1.0 / mse))
            leg["psnr_ycbcr_db"] = [round(float(x), 2) for x in np.mean(psnr, 0)]
            leg["step"] = float(qp.steps[0])
        legs.append(leg)
    # batched: all frames of the sequence, every step set as a rung, 64 frames per call
    scales = [float(q.steps[0] / qps[0].steps[0]) for q in qps]
    out = None
    def batched(_=0):
        nonlocal out
        for f0 in range(0, Fn, 64):
            out, offs = G.encode_batch(P[f0:f0 + 64], A[f0:f0 + 64], [Jd] * len(P[f0:f0 + 64]), scales, qps[0],
                                       out=out)
    ms = _timed_calls(torch, stream, batched, 2)
    line = {"metric": ("point-cloud" if pointcloud else "3DGS sequence") + " per-frame codec (plain latency, batched "
            "throughput)", "unit": "frames/s", "higher_is_better": True,
            "value": round(Fn / (float(np.mean(ms)) / 1e3), 1), "dtype": "f32", "data": "synthetic",
            "config": {"workload": (f"{Fn} frames of ~1M points on two capsule humanoids, depth 10, YCbCr" if pointcloud
                                    else f"{Fn} dynamic 3DGS frames of ~250k Gaussians (+-10%), depth 16, 56 channels"),
                       "points_total": n_tot, "step_sets": len(qps)},
            "batched_all_steps_fps": round(Fn / (float(np.mean(ms)) / 1e3), 1),
            "batched_gaussians_per_s": round(n_tot / (float(np.mean(ms)) / 1e3), 0), "plain": legs}
    print(json.dumps(line), flush=True)


def run_blocksweep(args):
    """RLGR block size B against stream size and codec time (8 frames of 1M
    Gaussians, batched encode + decode)."""
    import numpy as np
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2606_05650_gb300 import gsnfs as G, synthetic as syn
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    frames = make_frames(0, args.frames)
    P = [torch.from_numpy(p).to(dev) for p, _ in frames]
    A = [torch.from_numpy(a).to(dev) for _, a in frames]
    F = len(P)
    res = []
    for B in (256, 512, 1024, 2048, 4096, 8192):
        qp = G.QuantParams(syn.gs_channel_groups(), syn.GS_BASE_STEPS, rlgr_block=B)
        st = {"out": None}
        G.profile_enable(True)
        G.profile_read()

        def rt(_=0):
            st["out"], offs = G.encode_batch(P, A, [J] * F, [1.0], qp, out=st["out"])
            st["offs"] = offs
            G.decode_batch(st["out"], offs, C, F * N_GAUSS)
        ms = _timed_calls(torch, stream, rt, 3)
        stg = G.profile_read()
        G.profile_enable(False)
        per = lambda k: round(stg[k][0] / max(stg[k][1], 1), 4) if k in stg else None
        res.append({"B": B, "round_trip_ms": round(float(np.mean(ms)), 3),
                    "bytes_per_frame": int(st["offs"][-1]) // F,
                    "rlgr_encode_ms": per("rlgr_encode"), "rlgr_decode_ms": per("rlgr_decode")})
    print(json.dumps({"metric": "RLGR block size sweep", "unit": "ms per 8-frame round trip", "data": "synthetic",
                      "config": {"workload": f"{F} dynamic 3DGS frames of {N_GAUSS} Gaussians, depth {J}, C = {C}"},
                      "sweep": res}), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "ladder":
        run_ladder(args)
    elif args.workload in ("sequence", "pointcloud"):
        run_sequence(args, pointcloud=args.workload == "pointcloud")
    elif args.workload == "blocksweep":
        run_blocksweep(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
