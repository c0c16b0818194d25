#!/usr/bin/env python
"""Benchmark of full handle/tunnel loop detection (faces/s) on the tube-chain workload.

One step = one complete detection of the batch -- operator build, initial pass (every
event, loop and Reeb node), tunnel passes and result download -- for 4 seed vertices on
the tube-chain mesh (8 smooth-unioned tori R = 1, r = 0.35, spacing 1.6, blend 0.15,
marching tetrahedra, ~512k faces, genus 8, normal jitter 0.1 of the mean edge), all four
problems in one batch (one launch per kernel per step, step loops as device-driven graphs).

value  = faces per step / device time per step (CUDA events on the library's stream,
         inputs already in HBM, L2 flushed by a 256 MiB write before each timed step), in
         the FP32 form (FP32 values, rows deciding near a threshold redone in FP64) unless
         --precision fp64;
e2e    = the same metric through the C ABI with host (pinned) buffers, host wall time,
         host->device input copies and result download inside the call;
plain_fp64 = the same problems one per call, FP64, kernels launched from the host (no
         batching, no graph); speedup_vs_plain_fp64 = value / plain_fp64.value;
roofline = the initial-pass frontier update kernel (the diffusion SpMV): algorithmic
         bytes per launch / mean launch time from CUDA events recorded around each launch
         inside the library, against the measured HBM copy bandwidth;
cpu_baseline = the plain CPU oracle on a bounded sample of the same workload;
check_vs_oracle = those sampled problems' GPU results against the oracle's: integer
         results identical, max |phi - phi_oracle|, rows redone in FP64, and the largest
         residual of the FP64 mass check of the diffusion step over the batch.

--impl reference times the CPU oracle itself (the only reference implementation of this
method available here) with the same metric and JSON layout.
Multi-GPU (torchrun, N ranks): the job is the tube chain with 4 N seed vertices; its problems are
partitioned over the ranks by greedy LPT on face counts (each rank's share is the single-GPU
batch's size: weak scaling), with no collective on the data path; value = every problem's faces /
the slowest rank's step time; per-problem statuses are gathered on rank 0.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "faces/s full loop detection (batched FP32 vs plain FP64 GPU); SpMV HBM GB/s vs peak"
UNIT = "faces/s"
L2_FLUSH_BYTES = 256 << 20
MIDRUN_STEPS = (100, 400, 1000)


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--scale", type=float, default=1.0, help="workload grid scale (1.0 = full size)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-sample", type=int, default=3, help="problems timed for the CPU baseline (about 13 s of one core)")
    ap.add_argument("--profile-case", action="store_true",
                    help="one detection of the workload bounded to --max-steps initial steps (for profilers)")
    ap.add_argument("--shape", default="",
                    help="profile case: fixed launch shape 'threads,blocks_per_sm,hook_variant,rows_per_warp' "
                         "instead of the autotuner (keeps tuning runs out of a profiler's launch list)")
    ap.add_argument("--max-steps", type=int, default=400)
    ap.add_argument("--max-pass-steps", type=int, default=200)
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64", "bf16"],
                    help="form of the timed batched path (fp32: FP32 values with FP64 near-threshold recheck)")
    ap.add_argument("--no-plain", action="store_true", help="skip the plain FP64 comparison arm")
    ap.add_argument("--plain-steps", type=int, default=5, help="timed steps of the plain FP64 arm")
    ap.add_argument("--fp64-steps", type=int, default=3, help="timed steps of the batched FP64 arm")
    ap.add_argument("--no-batch", action="store_true",
                    help="skip the 1024-problem batch workload measured beside the headline")
    return ap.parse_args()


def workload_desc(probs):
    m = probs[0][0]
    nprob = sum(len(s) for _, s in probs)
    faces = sum(mm.nf * len(s) for mm, s in probs)
    return {"workload": f"tube chain, 8 smooth-unioned tori, {m.nf} faces, genus {m.genus()}, {nprob} seeds",
            "mesh_faces": m.nf, "mesh_vertices": m.nv, "genus": m.genus(), "problems": nprob,
            "faces_per_step": faces}, faces


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def max_over_ranks(x: float, dist=None, device=None) -> float:
    """The largest x over all ranks (the slowest rank's time); x itself without a process group."""
    if dist is None:
        return x
    import torch

    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_value(faces_all_ranks: float, ms_max: float) -> float:
    """Whole-job faces/s: the faces of every problem of the job, over all ranks, in the time of the
    slowest rank."""
    return faces_all_ranks / (ms_max / 1e3)


def job_problems(world: int, scale: float):
    """The job at N GPUs: the tube-chain mesh with 4 N seed vertices (seed streams 0 .. 4N-1), so that
    every rank's share is the single-GPU batch's size (weak scaling); N = 1 is the 4-seed batch."""
    import meshgen

    (m, seeds), = meshgen.workload(2, scale)
    if world > 1:
        seeds = [meshgen.seed_vertex(s, m.nv) for s in range(4 * world)]
    return [(m, seeds)]


def run_ranks(args, world: int, rank: int, local: int) -> int:
    """N > 1: the job's problems partitioned over the ranks by greedy LPT on their face counts (no
    collective on the data path); each rank times its own share; the job takes the slowest rank's
    time; per-problem statuses are gathered on rank 0, which prints the line."""
    import torch
    import torch.distributed as dist

    import paper_2105_13168_gb300 as vls
    from paper_2105_13168_gb300 import partition

    torch.cuda.set_device(local)
    dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    probs = job_problems(world, args.scale)
    cfg, faces = workload_desc(probs)
    sub, mine = partition.shard(probs, rank, world)
    stream = torch.cuda.current_stream()
    ctx = vls.vls_create(vls.vls_default_options(precision=args.precision), stream.cuda_stream)
    meshes_dev = [(torch.from_numpy(m.X).to(dev), torch.from_numpy(m.F).to(dev)) for m, _ in sub]
    pinned = [(torch.from_numpy(m.X).pin_memory(), torch.from_numpy(m.F).pin_memory()) for m, _ in sub]
    meshes_host = [(x.numpy(), f.numpy()) for x, f in pinned]
    seeds = [s for _, s in sub]
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)

    def one(host=False):
        if not sub:
            return []
        res = vls.vls_detect_batch(ctx, meshes_host if host else meshes_dev, seeds, device=not host)
        out = vls.read_result(res)
        vls.vls_result_free(res)
        return out

    for _ in range(args.warmup):
        one()
    sampler = ClockSampler(local) if rank == 0 else None
    dist.barrier()
    torch.cuda.synchronize()
    if sampler:
        sampler.start()
    step_ms, launches, out = [], 0, []
    for _ in range(args.steps):
        flush.fill_(1)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        out = one()
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        launches += out[0].stats["kernel_launches"] if out else 0
    torch.cuda.synchronize()
    clocks = sampler.stop() if sampler else None
    dist.barrier()
    ms_max = max_over_ranks(sum(step_ms) / len(step_ms), dist, dev)
    e2e_s, h2d, d2h = [], 0, 0
    for _ in range(args.steps):
        flush.fill_(1)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        o2 = one(host=True)
        e2e_s.append(time.perf_counter() - t0)
        if o2:
            h2d, d2h = o2[0].stats["h2d_bytes"], o2[0].stats["d2h_bytes"]
    e2e_max = max_over_ranks(1e3 * sum(e2e_s) / len(e2e_s), dist, dev)
    launches_all = max_over_ranks(float(launches), dist, dev)
    status = partition.gather([p.status for p in out], mine, len(partition.flatten(probs)), dist)
    if rank == 0:
        assert all(st == 0 for st in status), status
        cfg = dict(cfg, precision=args.precision, inputs="resident in HBM (device pointers) for value; pinned host for e2e",
                   l2="flushed by a 256 MiB write before every timed step",
                   parallelism=f"{world} GPUs, problems partitioned by greedy LPT on face counts")
        line = {"metric": METRIC, "value": whole_job_value(faces, ms_max), "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None,
                "dtype": {"fp32": "f32", "bf16": "bf16", "fp64": "f64"}[args.precision], "data": "synthetic",
                "config": cfg, "clocks": clocks,
                "e2e": {"value": faces / (e2e_max / 1e3), "unit": UNIT, "h2d_bytes_per_step": h2d,
                        "d2h_bytes_per_step": d2h},
                "gpu_launches": int(launches_all) * world}
        print(json.dumps(line), flush=True)
    dist.destroy_process_group()
    return 0


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def update_kernel_traffic(rows_per_launch: float, prec: str):
    """DRAM bytes per launch of the update kernel: bytes per row from a committed ncu capture
    scaled by the mean rows per launch, if the kernel source is unchanged since (else None)."""
    p = os.path.join(ROOT, "profiles", "k_update_traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f)
    src = os.path.join(ROOT, "paper_2105_13168_gb300", "csrc", "initial.cu")
    h = hashlib.sha256(open(src, "rb").read()).hexdigest()
    if d.get("source_sha256") != h or d.get("precision", "fp64") != prec or not d.get("dram_bytes_per_row"):
        return None
    return float(d["dram_bytes_per_row"]) * rows_per_launch


def host_cpu() -> dict:
    """The host's core count and CPU model (the CPU baseline runs on these cores)."""
    model = None
    try:
        with open("/proc/cpuinfo") as f:
            for ln in f:
                key = ln.split(":")[0].strip().lower()
                if key in ("model name", "cpu model", "hardware"):
                    model = ln.split(":", 1)[1].strip()
                    break
                if key == "cpu part" and model is None:
                    part = ln.split(":", 1)[1].strip()
                    model = {"0xd4f": "Arm Neoverse-V2", "0xd40": "Arm Neoverse-V1", "0xd0c": "Arm Neoverse-N1",
                             "0xd8e": "Arm Neoverse-N2"}.get(part.lower(), "Arm cpu part " + part)
    except OSError:
        pass
    import platform

    return {"nproc": os.cpu_count(), "cpu_model": model or platform.processor() or platform.machine(),
            "arch": platform.machine()}


def cpu_baseline(probs, nsample: int) -> dict:
    import oracle

    flat = [(m, s) for m, seeds in probs for s in seeds][:max(1, nsample)]
    t0 = time.perf_counter()
    faces = 0
    results = []
    for m, s in flat:
        r = oracle.detect(m, s, record_steps=1)
        assert r.status == 0, r.status_name
        faces += m.nf
        results.append(r)
    dt = time.perf_counter() - t0
    # untimed: the same problems stopped mid-run (front in flight), for the value check
    midrun = {k: [oracle.detect(m, s, max_steps=k, tunnels=0) for m, s in flat] for k in MIDRUN_STEPS}
    return dict({"value": faces / dt, "unit": UNIT, "cores": 1, "kind": "oracle", "seconds": round(dt, 2),
                 "sample": f"{len(flat)} of {sum(len(s) for _, s in probs)} problems of the same workload, full "
                           "detection (initial pass, tunnel passes, refinement passes), single-threaded FP64 oracle"},
                **host_cpu()), results, midrun


def compare_with_oracle(g, o) -> dict:
    """The FP32-form contract against the oracle for one problem: status, events, layer table and
    handle loops identical; counted (FP32 drift can move a decision taken within ~1e-6 of its
    threshold): steps whose band records differ, vertices whose cover step or final layer
    differs, tunnel loops that differ."""
    import numpy as np

    same = (g.status == o.status and g.genus == o.genus and g.events() == o.events()
            and np.array_equal(g.layers, o.layers) and len(g.handles) == len(o.handles)
            and len(g.tunnels) == len(o.tunnels) and len(g.refined) == len(o.refined))
    if same:
        for hg, ho in zip(g.handles, o.handles):
            same &= (hg.step, hg.layer) == (ho.step, ho.layer) and np.array_equal(hg.edges, ho.edges) \
                and np.array_equal(hg.verts, ho.verts)
    tun = sum((tg.status, tg.stop_step, tg.bstar) != (to.status, to.stop_step, to.bstar)
              or not np.array_equal(tg.verts, to.verts) for tg, to in zip(g.tunnels, o.tunnels))
    ref = sum((tg.status, tg.stop_step, tg.bstar) != (to.status, to.stop_step, to.bstar)
              or not np.array_equal(tg.verts, to.verts) for tg, to in zip(g.refined, o.refined))
    rec = int((g.records != o.records).any(axis=1).sum()) if len(g.records) == len(o.records) else -1
    bad = np.nonzero((g.records != o.records).any(axis=1))[0] if rec > 0 else []
    first = int(bad[0]) if len(bad) else None
    # PL streamlines (Sec. 3.2): status agreement, and the length difference where the pass's vertex
    # loop is the oracle's (the FP32 arrival times drift, so the points move slightly)
    sl_n = sl_same = 0
    sl_rel = 0.0
    for tg, to in list(zip(g.tunnels, o.tunnels)) + list(zip(g.refined, o.refined)):
        if tg.stream_status < 0 and to.stream_status < 0:
            continue
        sl_n += 1
        sl_same += tg.stream_status == to.stream_status
        if tg.stream_status == to.stream_status == 0 and np.array_equal(tg.verts, to.verts):
            sl_rel = max(sl_rel, abs(tg.stream_length - to.stream_length) / to.stream_length)
    # loop classification (Sec. 3.5): offset length change > 0 reads as a handle, < 0 as a tunnel
    dl = np.asarray(g.offset_change)
    return {"identical": bool(same), "record_steps_differing": rec,
            "first_differing_step": None if first is None else first + 1,
            "uncertified_at_first_differing_step": None if first is None else int(g.step_uncertified[first]),
            "uncertified": [int(g.stats["uncertified"]), int(g.stats["pass_uncertified"]),
                            int(g.stats["refine_uncertified"])],
            "cover_steps_differing": int((g.cover != o.cover).sum()),
            "final_layers_differing": int((g.layer != o.layer).sum()), "tunnel_loops_differing": int(tun),
            "refined_loops_differing": int(ref),
            "streamlines": [sl_n, sl_same, sl_rel],
            "classified_as_handle": [int((dl[:, 0] > 0).sum()), int((dl[:, 2] > 0).sum())] if dl.size else [0, 0],
            "classified_as_tunnel": int((dl[:, 1] < 0).sum()) if dl.size else 0, "loops": int(len(dl))}


def measure_batch_workload(vls, torch, stream, flush, prec: str, steps: int = 2) -> dict:
    """The 1024-problem batch workload (256 tori / tube chains of genus 1-20, 2k-200k faces, 4
    seeds each) in one call per step: faces/s with device-resident inputs, and the frontier
    update kernel's bandwidth at this scale (one host-launched kernel-timing pass)."""
    import meshgen

    dev = torch.device("cuda", torch.cuda.current_device())
    probs = meshgen.workload(4)
    faces = sum(m.nf * len(s) for m, s in probs)
    meshes = [(torch.from_numpy(m.X).to(dev), torch.from_numpy(m.F).to(dev)) for m, _ in probs]
    seeds = [s for _, s in probs]
    ctx = vls.vls_create(vls.vls_default_options(precision=prec), stream.cuda_stream)
    vls.vls_result_free(vls.vls_detect_batch(ctx, meshes, seeds, device=True))  # warm-up (and tuning)
    ms, ok = [], 0
    for _ in range(steps):
        flush.fill_(1)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        res = vls.vls_detect_batch(ctx, meshes, seeds, device=True)
        e1.record(stream)
        e1.synchronize()
        out = vls.read_result(res)
        vls.vls_result_free(res)
        ms.append(e0.elapsed_time(e1))
        ok = sum(p.status == 0 for p in out)
    vls.vls_destroy(ctx)
    pctx = vls.vls_create(vls.vls_default_options(precision=prec, profile=1), stream.cuda_stream)
    res = vls.vls_detect_batch(pctx, meshes, seeds, device=True)
    pout = vls.read_result(res)
    vls.vls_result_free(res)
    vls.vls_destroy(pctx)
    n_upd, ms_upd = pout[0].stats["n_update"], pout[0].stats["ms_update"]
    rows = sum(p.stats["row_updates"] for p in pout)
    deg = sum(3 * m.nf * len(s) for m, s in probs) / sum(m.nv * len(s) for m, s in probs)
    bpr = {"fp64": 44, "fp32": 40, "bf16": 38}[prec] + 4 * deg
    gbs = (rows / n_upd * bpr) / (ms_upd / n_upd * 1e-3) / 1e9 if n_upd else None
    peak, _ = measured_peaks()
    mean = sum(ms) / len(ms)
    return {"workload": f"256 tori / tube chains (genus 1-20), 1024 problems, {faces} faces", "value": faces / (mean / 1e3),
            "unit": UNIT, "ms_per_step": mean, "steps": len(ms), "problems_ok": ok,
            "k_update": {"rows_per_launch": round(rows / n_upd, 1) if n_upd else None, "bytes_per_row": round(bpr, 2),
                         "launch_us": 1e3 * ms_upd / n_upd if n_upd else None, "achieved_gbs": gbs,
                         "frac": gbs / peak if gbs else None}}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import meshgen
    import oracle

    probs = meshgen.workload(2, args.scale)
    cfg, _ = workload_desc(probs)
    m, seeds = probs[0]
    times = []
    for it in range(args.warmup + args.steps):
        s = seeds[it % len(seeds)]
        t0 = time.perf_counter()
        r = oracle.detect(m, s)
        dt = time.perf_counter() - t0
        assert r.status == 0
        if it >= args.warmup:
            times.append(dt)
    mean = sum(times) / len(times)
    value = m.nf / mean
    cfg = dict(cfg, sample="each step: one problem (one seed) of the workload, full detection")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": mean * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": cfg,
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": "one problem (one seed) per step of the tube-chain workload"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_profile_case(args):
    """One detection of the workload with bounded step counts, device inputs, no extra runs."""
    import torch

    import meshgen
    import paper_2105_13168_gb300 as vls

    torch.cuda.set_device(0)
    probs = meshgen.workload(2, args.scale)
    cfg, faces = workload_desc(probs)
    dev = torch.device("cuda", 0)
    meshes_dev = [(torch.from_numpy(m.X).to(dev), torch.from_numpy(m.F).to(dev)) for m, _ in probs]
    shape = {}
    if args.shape:
        t, bps, hv, rpw = (int(x) for x in args.shape.split(","))
        shape = dict(threads=t, blocks_per_sm=bps, hook_variant=hv, rows_per_warp=rpw)
    opts = vls.vls_default_options(max_steps=args.max_steps, max_pass_steps=args.max_pass_steps,
                                   precision=args.precision, **shape)
    ctx = vls.vls_create(opts, torch.cuda.current_stream().cuda_stream)
    res = vls.vls_detect_batch(ctx, meshes_dev, [s for _, s in probs], device=True)
    out = vls.read_result(res)
    vls.vls_result_free(res)
    vls.vls_destroy(ctx)
    torch.cuda.synchronize()
    print(json.dumps({"profile_case": cfg, "max_steps": args.max_steps,
                      "status": [p.status_name for p in out], "launches": out[0].stats["kernel_launches"],
                      "rows": sum(p.stats["row_updates"] for p in out)}), flush=True)
    return 0


def main():
    args = parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.profile_case:
        return run_profile_case(args)
    import numpy as np
    import torch

    import meshgen
    import paper_2105_13168_gb300 as vls

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        return run_ranks(args, world, rank, local)
    dist = None
    torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())

    probs = meshgen.workload(2, args.scale)
    cfg, faces = workload_desc(probs)
    # CPU baseline (rank 0, one GPU): timed before any GPU work of this process
    cpu, orc_results, orc_midrun = None, [], []
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu, orc_results, orc_midrun = cpu_baseline(probs, args.cpu_sample)

    stream = torch.cuda.current_stream()
    prec = args.precision
    ctx = vls.vls_create(vls.vls_default_options(precision=prec), stream.cuda_stream)
    meshes_dev = [(torch.from_numpy(m.X).to(dev), torch.from_numpy(m.F).to(dev)) for m, _ in probs]
    seeds = [s for _, s in probs]
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)

    def one(device_inputs=True):
        if device_inputs:
            res = vls.vls_detect_batch(ctx, meshes_dev, seeds, device=True)
        else:
            res = vls.vls_detect_batch(ctx, meshes_host, seeds, device=False)
        out = vls.read_result(res)
        vls.vls_result_free(res)
        return out

    for _ in range(args.warmup):
        out = one()
        assert all(p.status == 0 for p in out), [p.status_name for p in out]
    # ---- timed region: device-resident inputs
    sampler = ClockSampler(torch.cuda.current_device()) if rank == 0 else None
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    if sampler:
        sampler.start()
    step_ms, launches = [], 0
    for _ in range(args.steps):
        flush.fill_(1)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        out = one()
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        launches += out[0].stats["kernel_launches"]
        assert all(p.status == 0 for p in out), [p.status_name for p in out]
    torch.cuda.synchronize()
    clocks = sampler.stop() if sampler else None
    if dist is not None:
        dist.barrier()
    ms = sum(step_ms) / len(step_ms)
    ms_max = max_over_ranks(ms, dist, dev)
    value = whole_job_value(faces, ms_max)
    # ---- e2e: host buffers through the C ABI (pinned), copies inside the call
    pinned = [(torch.from_numpy(m.X).pin_memory(), torch.from_numpy(m.F).pin_memory()) for m, _ in probs]
    meshes_host = [(x.numpy(), f.numpy()) for x, f in pinned]
    one(device_inputs=False)
    e2e_s, h2d, d2h = [], 0, 0
    for _ in range(args.steps):
        flush.fill_(1)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        out = one(device_inputs=False)
        e2e_s.append(time.perf_counter() - t0)
        h2d, d2h = out[0].stats["h2d_bytes"], out[0].stats["d2h_bytes"]
    e2e_v = faces / (sum(e2e_s) / len(e2e_s))
    vls.vls_destroy(ctx)
    # ---- kernel timing pass: the same workload with CUDA events around every launch of the
    # frontier update kernel (host-driven launches so that each launch can be bracketed)
    pctx = vls.vls_create(vls.vls_default_options(profile=1, precision=prec), stream.cuda_stream)
    flush.fill_(1)
    res = vls.vls_detect_batch(pctx, meshes_dev, seeds, device=True)
    pout = vls.read_result(res)
    vls.vls_result_free(res)
    vls.vls_destroy(pctx)
    upd_ms, upd_n = pout[0].stats["ms_update"], pout[0].stats["n_update"]
    rows = sum(p.stats["row_updates"] for p in pout)
    # ---- the same batch once more with the final state kept: rechecks, and the check of the
    # problems the CPU baseline ran against the oracle (integer results, max value error)
    cctx = vls.vls_create(vls.vls_default_options(precision=prec, keep_state=1, record_steps=1), stream.cuda_stream)
    res = vls.vls_detect_batch(cctx, meshes_dev, seeds, device=True)
    cout = vls.read_result(res)
    vls.vls_result_free(res)
    vls.vls_destroy(cctx)
    # loop classification (Sec. 3.5) of every problem's loops: offset length change > 0 reads as a handle
    dls = [np.asarray(p.offset_change) for p in cout if len(p.handles)]
    nloops = sum(len(x) for x in dls)
    classes = {"loops": nloops,
               "handle_loops_read_as_handles": sum(int((x[:, 0] > 0).sum()) for x in dls),
               "refined_loops_read_as_handles": sum(int((x[:, 2] > 0).sum()) for x in dls),
               "tunnel_loops_read_as_tunnels": sum(int((x[:, 1] < 0).sum()) for x in dls)}
    check = {"problems_checked": len(orc_results), "classification": classes,
             "phase_ms": {k: round(cout[0].stats[k], 2) for k in ("ms_operator", "ms_initial", "ms_tunnel",
                                                                  "ms_refine", "ms_download")},
             "uncertified_decisions": [[int(p.stats["uncertified"]), int(p.stats["pass_uncertified"]),
                                        int(p.stats["refine_uncertified"])] for p in cout],
             "mass_check_max_resid": max(p.stats["mass_resid"] for p in cout),
             "rechecks": cout[0].stats["rechecks"],
             "pass_rechecks": cout[0].stats["pass_rechecks"], "row_updates": rows,
             "pass_updates": sum(p.stats["pass_updates"] for p in cout)}
    if orc_results:
        cmp = [compare_with_oracle(g, o) for g, o in zip(cout, orc_results)]
        check["events_and_handle_loops_identical"] = all(c["identical"] for c in cmp)
        for key in ("record_steps_differing", "first_differing_step", "uncertified_at_first_differing_step",
                    "cover_steps_differing", "final_layers_differing", "tunnel_loops_differing",
                    "refined_loops_differing"):
            check[key] = [c[key] for c in cmp]
        check["streamlines"] = {"traced": sum(c["streamlines"][0] for c in cmp),
                                "status_as_oracle": sum(c["streamlines"][1] for c in cmp),
                                "max_rel_length_diff_same_vertex_loop": max(c["streamlines"][2] for c in cmp)}
        # values mid-run (front in flight; at the end every value is 0 or 1): the max error against
        # the FP64 oracle at a few steps
        nchk = len(orc_results)
        flat = [(x, f, s) for (x, f), ss in zip(meshes_dev, seeds) for s in ss][:nchk]
        check["max_abs_err_phi_vs_oracle"] = {}
        for k, oms in orc_midrun.items():
            mctx = vls.vls_create(vls.vls_default_options(precision=prec, keep_state=1, max_steps=k, tunnels=0),
                                  stream.cuda_stream)
            errs = []
            for (x, f, s), om in zip(flat, oms):
                r = vls.vls_detect(mctx, x, f, s, device=True)
                gm = vls.read_result(r)[0]
                vls.vls_result_free(r)
                errs.append(float(np.abs(gm.phi - om.phi).max()))
            vls.vls_destroy(mctx)
            check["max_abs_err_phi_vs_oracle"][f"step_{k}"] = max(errs)
    # ---- plain FP64 arm: the same problems one at a time (no batching), FP64, kernels launched
    # from the host (no graph)
    plain = None
    if not args.no_plain:
        qctx = vls.vls_create(vls.vls_default_options(precision="fp64", host_loop=1), stream.cuda_stream)
        flat = [(x, f, s) for (x, f), ss in zip(meshes_dev, seeds) for s in ss]

        def plain_step():
            outs = []
            for x, f, s in flat:
                r = vls.vls_detect(qctx, x, f, s, device=True)
                outs.extend(vls.read_result(r))
                vls.vls_result_free(r)
            return outs

        x0, f0, s0 = flat[0]
        vls.vls_result_free(vls.vls_detect(qctx, x0, f0, s0, device=True))  # warm-up
        pms = []
        for _ in range(max(1, args.plain_steps)):
            flush.fill_(1)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            pouts = plain_step()
            e1.record(stream)
            e1.synchronize()
            pms.append(e0.elapsed_time(e1))
            assert all(p.status == 0 for p in pouts)
        vls.vls_destroy(qctx)
        pm = sum(pms) / len(pms)
        plain = {"value": faces / (pm / 1e3), "unit": UNIT, "ms_per_step": pm, "steps": len(pms),
                 "form": "FP64, one problem per call (no batching), step kernels launched from the host (no graph)"}
    # ---- batched FP64 arm: the headline's batch and graphs in the FP64 form (what the FP32 form
    # itself buys, with batching and graphs held equal)
    fp64b = None
    if not args.no_plain and prec != "fp64":
        bctx = vls.vls_create(vls.vls_default_options(precision="fp64"), stream.cuda_stream)
        res = vls.vls_detect_batch(bctx, meshes_dev, seeds, device=True)  # warm-up (and tuning)
        vls.vls_result_free(res)
        bms = []
        for _ in range(max(1, args.fp64_steps)):
            flush.fill_(1)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            res = vls.vls_detect_batch(bctx, meshes_dev, seeds, device=True)
            e1.record(stream)
            e1.synchronize()
            bouts = vls.read_result(res)
            vls.vls_result_free(res)
            bms.append(e0.elapsed_time(e1))
            assert all(p.status == 0 for p in bouts)
        vls.vls_destroy(bctx)
        bm = sum(bms) / len(bms)
        fp64b = {"value": faces / (bm / 1e3), "unit": UNIT, "ms_per_step": bm, "steps": len(bms),
                 "form": "FP64, the same batch in one call per step, step loops as device-driven graphs"}
    batch = None
    if not args.no_batch and rank == 0:
        batch = measure_batch_workload(vls, torch, stream, flush, prec)
    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return 0
    # ---- roofline of the frontier update kernel
    peak, peak_kind = measured_peaks()
    deg = sum(3 * m.nf * len(s) for m, s in probs) / sum(m.nv * len(s) for m, s in probs)
    # frontier entry 8, row bounds 8, columns 4d, own state (layer 4 + value 8, 4 or 2), output 16
    bytes_per_row = {"fp64": 44, "fp32": 40, "bf16": 38}[prec] + 4 * deg
    launch_s = (upd_ms / upd_n) / 1e3 if upd_n else None
    rows_per_launch = rows / upd_n if upd_n else 0
    achieved = (rows_per_launch * bytes_per_row / launch_s) / 1e9 if launch_s else None
    roof = {"kernel": f"k_update (initial-pass frontier update, {prec.upper()})", "bound": "hbm", "achieved": achieved,
            "peak": peak, "peak_kind": peak_kind, "unit": "GB/s", "frac": (achieved / peak) if achieved else None,
            "traffic": update_kernel_traffic(rows_per_launch, prec), "bytes_per_row": round(bytes_per_row, 2),
            "rows_per_launch": round(rows_per_launch, 1), "launch_us": launch_s * 1e6 if launch_s else None,
            "launches": upd_n, "share_of_timed_step": (upd_ms / ms) if ms else None,
            "method": "CUDA events around each launch in a kernel-timing pass of the same workload "
                      "(host-driven launches); the timed steps run the device-driven graph"}
    cfg = dict(cfg, precision={"fp32": "fp32 values, fp64 near-threshold recheck",
                               "bf16": "bf16 values, fp32 arithmetic, fp64 near-threshold recheck",
                               "fp64": "fp64"}[prec], inputs="resident in HBM (device pointers) for value; pinned host for e2e",
               l2="flushed by a 256 MiB write before every timed step",
               parallelism=f"{world} GPU(s), each its own copy of the batch" if world > 1 else "1 GPU")
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": {"fp32": "f32", "bf16": "bf16", "fp64": "f64"}[prec], "data": "synthetic",
            "config": cfg,
            "e2e": {"value": e2e_v, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "gpu_launches": launches, "roofline": roof, "clocks": clocks, "check_vs_oracle": check}
    if batch is not None:
        line["batch_workload"] = batch
    if plain is not None:
        line["plain_fp64"] = plain
        line["speedup_vs_plain_fp64"] = value / world / plain["value"]
    if fp64b is not None:
        line["batched_fp64"] = fp64b
        line["speedup_vs_batched_fp64"] = value / world / fp64b["value"]
    if cpu is not None:
        line["cpu_baseline"] = cpu
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
