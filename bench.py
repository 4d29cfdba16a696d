"""Benchmark: TRS partition decisions per second at 2160p.

Workload: the 64-frame 3840x2160 10-bit moving-blob sequence, n = 16 slices,
lambda = 0.1 (k = 3).  One step = one batched decision of all 64 frames
(texture map, region tables, both search steps, decoding) replayed from a
CUDA graph, inputs resident in HBM (1.06 GB of luma per step, larger than
the 126 MB L2, so no flush is needed).  The JSON line also carries:
  plain     the same 64 frames decided one frame per launch chain
  e2e       the same metric through trs_batch_decide_host from pinned host
            buffers, host<->device copies inside the timed region
  roofline  the dominant kernel against its bound, and the texture kernel
            against HBM
  cpu_baseline  the oracle on this host, on a bounded sample of frames

--impl reference times the oracle as the reference arm.
Multi-GPU (torchrun): every rank decides its own copy of the workload
(replicas, weak scaling); rank 0 prints max-over-ranks timing.
"""

from __future__ import annotations

import argparse
import json
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "TRS partition decisions/sec at 2160p (batched vs plain); p50/p99 latency; % HBM peak"
UNIT = "decisions/s"
NFRAMES = 64
N_REGIONS = 16
LAMBDA = 0.1
WORKLOAD = "3840x2160p10 moving-blob sequence, 64 frames, n=16, lambda=0.1, k=3"


def _gen(f):
    import synth
    return synth.sequence_2160p_frame(f)


def make_inputs(nframes: int):
    ctx = mp.get_context("spawn")
    with ctx.Pool(min(16, os.cpu_count() or 1)) as pool:
        return pool.map(_gen, range(nframes))


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), float(d.get("sm_max_mhz", 2070.0)), "measured"
    except Exception:
        return 6800.0, 2070.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "20"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.p = None
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.p:
            self.p.terminate()
            try:
                self.out, _ = self.p.communicate(timeout=5)
            except Exception:
                self.p.kill()

    def summary(self):
        rows = []
        for line in (self.out or "").strip().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 7:
                continue
            try:
                rows.append((float(parts[0]), float(parts[1]), parts[3:7]))
            except ValueError:
                continue
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, r in rows for i, v in enumerate(r) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


def cpu_baseline(frames, budget_s: float = 12.0):
    """The oracle (O2, one core) on a bounded sample of the same frames."""
    from oracle import oracle as O
    O.build()
    t0 = time.perf_counter()
    done = 0
    for plane, times in frames:
        O.decide(plane, times, 10, N_REGIONS, LAMBDA)
        done += 1
        if time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    return {"value": done / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{done} of the {NFRAMES} workload frames, oracle texture + Q16 + exact DP search, 1 thread"}


def run_reference(args, rank, world):
    """Reference arm: the oracle timed on this host's cores, same metric."""
    if rank != 0:
        return
    frames = make_inputs(min(NFRAMES, 8))
    from oracle import oracle as O
    O.build()
    per_step = 2  # frames per step: a bounded sample, ~0.4 s of CPU work

    def step(i):
        for j in range(per_step):
            plane, times = frames[(i * per_step + j) % len(frames)]
            O.decide(plane, times, 10, N_REGIONS, LAMBDA)

    for i in range(args.warmup):
        step(i)
    t0 = time.perf_counter()
    for i in range(args.steps):
        step(i)
    dt = time.perf_counter() - t0
    value = per_step * args.steps / dt
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "frames_per_step": per_step},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"{per_step} frames per step of the workload, oracle on 1 thread"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--frames", type=int, default=NFRAMES,
                    help="frames per step (a smaller case for profiling; the metric uses 64)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    nfr = args.frames
    frames = make_inputs(nfr)  # spawn pool, before any CUDA call

    import torch
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    import __graft_entry__
    if rank == 0:
        __graft_entry__.build()
    if dist:
        dist.barrier()
    __graft_entry__.build()
    from paper_2012_14792_gb300 import runtime, trs

    dev = torch.device("cuda", local)
    dec = runtime.Decider(max_width=3840, max_height=2160, max_regions=N_REGIONS, max_batch=nfr,
                          device=local)
    lumas, tts, ins = [], [], []
    for plane, times in frames:
        raw = np.ascontiguousarray(plane).view(np.uint8)
        l = torch.from_numpy(raw).to(dev)
        t = torch.from_numpy(times).to(dev)
        lumas.append(l)
        tts.append(t)
        ins.append((l, raw.strides[0], plane.shape[1], plane.shape[0], 10, t, N_REGIONS, LAMBDA))
    out = torch.zeros(nfr * trs.PARTITION_BYTES, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)

    def sync_all():
        torch.cuda.synchronize(dev)
        if dist:
            dist.barrier()

    # --- batched, timed --------------------------------------------------
    for _ in range(args.warmup):
        dec.batch_decide(ins, out)
    sync_all()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        ev0.record(stream)
        for _ in range(args.steps):
            dec.batch_decide(ins, out)
        ev1.record(stream)
        sync_all()
    ms = ev0.elapsed_time(ev1)
    stage = trs.trs_batch_stage_ms(dec.ctx)  # CUDA events inside the graph, last timed step
    if dist:
        t = torch.tensor([ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    value = world * nfr * args.steps / (ms / 1e3)
    parts = dec.partitions(out, nfr)
    assert all(p.status == 0 for p in parts), [p.status for p in parts]

    # --- plain: one frame per launch chain ------------------------------
    one = torch.zeros(trs.PARTITION_BYTES, dtype=torch.uint8, device=dev)
    for (l, pitch, W, H, bd, t, n, lam) in ins[:4]:
        dec.decide(l, pitch, W, H, bd, t, n, lam, one)
    sync_all()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = max(1, args.steps // 4)
    e0.record(stream)
    for _ in range(reps):
        for (l, pitch, W, H, bd, t, n, lam) in ins:
            dec.decide(l, pitch, W, H, bd, t, n, lam, one)
    e1.record(stream)
    sync_all()
    plain_value = nfr * reps / (e0.elapsed_time(e1) / 1e3)

    # --- end to end through the host-buffer C call ------------------------
    pinned = [torch.from_numpy(np.ascontiguousarray(p).view(np.uint8)).pin_memory() for p, _ in frames]
    pinned_t = [torch.from_numpy(t).pin_memory() for _, t in frames]
    hdescs = [trs.frame_desc(pinned[i], pinned_t[i], 3840, 2160, 7680, 10, N_REGIONS, LAMBDA)
              for i in range(nfr)]
    for _ in range(2):
        trs.trs_batch_decide_host(dec.ctx, hdescs)
    sync_all()
    e_steps = max(3, args.steps // 4)
    t0 = time.perf_counter()
    for _ in range(e_steps):
        hp = trs.trs_batch_decide_host(dec.ctx, hdescs)
    sync_all()
    e2e_dt = time.perf_counter() - t0
    if dist:
        t = torch.tensor([e2e_dt], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_dt = float(t.item())
    assert bytes(hp[0]) == bytes(parts[0])
    e2e = {"value": world * nfr * e_steps / e2e_dt, "unit": UNIT,
           "h2d_bytes_per_step": int(sum(p.numel() for p in pinned) + sum(t.numel() * 4 for t in pinned_t)),
           "d2h_bytes_per_step": nfr * trs.PARTITION_BYTES}

    # --- roofline -----------------------------------------------------------
    hbm, sm_max, src = peaks()
    tex_bytes = sum(p.numel() for p in pinned)  # each luma sample read once
    tex_ms = stage.get("texture", 0.0)
    tex_gbs = tex_bytes / (tex_ms / 1e3) / 1e9 if tex_ms > 0 else 0.0
    row_relax, col_relax = trs.trs_plan_work(3840, 2160, N_REGIONS)
    # INT32 issue peak: 152 SMs x 128 lanes x max SM clock; a relaxation is a
    # 64-bit combine + a 64-bit minimum, at least 6 INT32 lane operations
    alu_peak = 152 * 128 * sm_max * 1e6 / 6.0 / 1e12  # T relaxations / s
    kinds = {"step1_rows": row_relax, "step2_rows": row_relax, "step1_columns": col_relax,
             "step2_columns": col_relax}
    dominant = max(stage, key=stage.get) if stage else "texture"
    if dominant == "texture":
        roof = {"kernel": "texture_kernel", "bound": "hbm", "achieved": tex_gbs, "peak": hbm, "unit": "GB/s",
                "frac": tex_gbs / hbm, "traffic": None, "peak_source": src}
    else:
        work = kinds.get(dominant, row_relax + col_relax) * nfr
        ach = work / (stage[dominant] / 1e3) / 1e12
        roof = {"kernel": dominant, "bound": "alu", "achieved": ach, "peak": alu_peak,
                "unit": "T relaxations/s", "frac": ach / alu_peak, "traffic": None,
                "peak_source": "derived: 152 SMs x 128 INT32 lanes x %.0f MHz / 6 ops" % sm_max}
    tex_roof = {"kernel": "texture_kernel", "bound": "hbm", "achieved": tex_gbs, "peak": hbm, "unit": "GB/s",
                "frac": tex_gbs / hbm, "peak_source": src}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(frames)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
                "config": {"workload": WORKLOAD if nfr == NFRAMES else f"{WORKLOAD} (first {nfr} frames)",
                           "frames_per_step": nfr, "form": "batched, CUDA graph",
                           "l2": f"inputs {tex_bytes / 1e9:.2f} GB per step > L2, no flush"},
                "plain": {"value": plain_value, "unit": UNIT, "form": "one frame per launch chain"},
                "stage_ms": stage, "clocks": clk.summary(), "e2e": e2e,
                "gpu_launches": 8 * args.steps, "roofline": roof, "roofline_texture": tex_roof,
                "cpu_baseline": cpu}
        print(json.dumps(line), flush=True)
    dec.close()
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
