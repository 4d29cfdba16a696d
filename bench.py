"""Benchmark: TRS partition decisions per second at 2160p.

Workload: the 64-frame 3840x2160 10-bit moving-blob sequence, n = 16 slices,
lambda = 0.1 (k = 3).  One step = one batched decision of all 64 frames
(texture map, region tables, both search steps, decoding) replayed from a
CUDA graph, inputs resident in HBM (1.06 GB of luma per step, larger than
the 126 MB L2, so no flush is needed).  The JSON line also carries:
  plain     the same 64 frames decided one frame per launch chain
  e2e       the same metric through trs_batch_decide_host from pinned host
            buffers, host<->device copies inside the timed region
  roofline  one fixed kernel (the step-1 row DP) against its bound;
            rooflines: every kernel of the step with its share of the
            one-chunk stage sum; roofline_texture: the texture kernel
  config_480p8_n4, config_1080p10_n8  the two single-frame configurations,
            batched and one frame per launch chain, beside the oracle
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
# Batches in flight in the timed stream of steps, and the chunks each
# captured batch is pipelined in (trs_set_batch_parts).  Measured at 2160p,
# n = 16 (decisions/s): 2 in flight 125.6 k (1 chunk), 127.2 k (2), 109.4 k (3);
# 3 in flight 132.1 k (1 chunk), 126.9 k (2), 123.1 k (3).
PARTS = 1
IN_FLIGHT = 3
E2E_THREADS = 2  # host threads of the end-to-end form (at most IN_FLIGHT)
N_REGIONS = 16
LAMBDA = 0.1
WORKLOAD = "3840x2160p10 moving-blob sequence, 64 frames, n=16, lambda=0.1, k=3"
# the kernel the headline roofline reports, fixed by name: the step-1 row DP.
# The two row DPs are the search's largest stages in every measurement, and
# step 1's work count is exact (step 2 skips the items of windows that break
# Eq. 4, so its count over-states its work)
ROOFLINE_KERNEL = "band_kernel<1>"


def _gen(f):
    import synth
    return synth.sequence_2160p_frame(f)


def _gen_mixed(i):
    import synth
    return synth.mixed_batch_frame(i)


def _gen_config(a):
    import synth
    name, seed = a
    return synth.make_frame(getattr(synth, name), seed)


# the single-frame configurations beside the headline one: (spec, n)
CONFIGS = {"config_480p8_n4": ("SPEC_480P8", 4), "config_1080p10_n8": ("SPEC_1080P10", 8)}
CONFIG_FRAMES = 64


def make_inputs(nframes: int, mixed: bool = False, configs: bool = False):
    """Draws the workload frames in a spawn pool (before any CUDA call)."""
    ctx = mp.get_context("spawn")
    with ctx.Pool(min(16, os.cpu_count() or 1)) as pool:
        seq = pool.map(_gen, range(nframes))
        mix = pool.map(_gen_mixed, range(256)) if mixed else None
        cfg = {k: pool.map(_gen_config, [(name, s) for s in range(CONFIG_FRAMES)])
               for k, (name, _) in CONFIGS.items()} if configs else None
    return seq, mix, cfg


def run_config(runtime, trs, spec, n, frames, device: int, steps: int, warmup: int, in_flight: int):
    """One single-frame configuration (832x480 8-bit n = 4, 1920x1080 10-bit
    n = 8) at full rate: its seeded frames decided as one batch per step
    (graph replays, `in_flight` contexts on their own streams), and one frame
    per launch chain."""
    import torch
    dev = torch.device("cuda", device)
    nf = len(frames)
    decs = [runtime.Decider(max_width=spec.width, max_height=spec.height, max_regions=n, max_batch=nf,
                            device=device) for _ in range(in_flight)]
    try:
        ins, keep = [], []
        for plane, times in frames:
            raw = np.ascontiguousarray(plane).view(np.uint8)
            l = torch.from_numpy(raw).to(dev)
            t = torch.from_numpy(times).to(dev)
            keep += [l, t]
            ins.append((l, raw.strides[0], spec.width, spec.height, spec.bit_depth, t, n, LAMBDA))
        outs = [torch.zeros(nf * trs.PARTITION_BYTES, dtype=torch.uint8, device=dev) for _ in decs]
        streams = [torch.cuda.Stream(dev) for _ in decs]
        cur = torch.cuda.current_stream(dev)

        def run(count):
            for k in range(count):
                i = k % in_flight
                with torch.cuda.stream(streams[i]):
                    decs[i].batch_decide(ins, outs[i])

        run(max(warmup, in_flight))
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(cur)
        for st in streams:
            st.wait_event(e0)
        run(steps)
        for st in streams:
            e = torch.cuda.Event()
            e.record(st)
            cur.wait_event(e)
        e1.record(cur)
        torch.cuda.synchronize(dev)
        ms = e0.elapsed_time(e1)
        ps = decs[0].partitions(outs[0], nf)
        assert all(p.status == 0 for p in ps)
        # one frame per launch chain
        one = torch.zeros(trs.PARTITION_BYTES, dtype=torch.uint8, device=dev)
        for (l, pitch, W, H, bd, t, nn, lam) in ins[:4]:
            decs[0].decide(l, pitch, W, H, bd, t, nn, lam, one)
        torch.cuda.synchronize(dev)
        reps = max(1, steps // 4)
        e0.record(cur)
        for _ in range(reps):
            for (l, pitch, W, H, bd, t, nn, lam) in ins:
                decs[0].decide(l, pitch, W, H, bd, t, nn, lam, one)
        e1.record(cur)
        torch.cuda.synchronize(dev)
        plain_ms = e0.elapsed_time(e1)
        assert bytes(decs[0].partitions(one)[0]) == bytes(ps[-1])  # the same decision alone and in the batch
    finally:
        for d in decs:
            d.close()
    return {"workload": f"{spec.width}x{spec.height}p{spec.bit_depth}, n={n}, lambda={LAMBDA}, k=3, "
                        f"{nf} seeded frames",
            "batched": {"value": nf * steps / (ms / 1e3), "unit": UNIT, "ms_per_step": ms / steps,
                        "frames_per_step": nf, "in_flight": in_flight,
                        "form": "batched, CUDA graph, default launch shapes"},
            "plain": {"value": nf * reps / (plain_ms / 1e3), "unit": UNIT, "form": "one frame per launch chain"}}


def run_mixed(runtime, trs, items, device: int, steps: int, warmup: int, n_parts: int, in_flight: int):
    """The 256-frame mixed batch (146 x 480p8, 73 x 1080p10, 37 x 2160p10,
    n from {4, 8, 16}, lambda 0.1), one graph launch per step, the steps
    spread over `in_flight` contexts on their own streams."""
    import torch
    dev = torch.device("cuda", device)
    decs = [runtime.Decider(max_width=3840, max_height=2160, max_regions=16, max_batch=len(items), device=device)
            for _ in range(in_flight)]
    ins, keep = [], []
    for it in items:
        raw = np.ascontiguousarray(it.plane).view(np.uint8)
        l = torch.from_numpy(raw).to(dev)
        t = torch.from_numpy(it.times).to(dev)
        keep += [l, t]
        ins.append((l, raw.strides[0], it.spec.width, it.spec.height, it.spec.bit_depth, t, it.n_regions, it.lam))
    tune = decs[0].autotune(ins)
    for d in decs:
        trs.trs_set_tune(d.ctx, tune["band_warps"], tune["col_warps"], tune["col_batch"])
        trs.trs_set_batch_parts(d.ctx, n_parts)
    outs = [torch.zeros(len(items) * trs.PARTITION_BYTES, dtype=torch.uint8, device=dev) for _ in decs]
    streams = [torch.cuda.Stream(dev) for _ in decs]
    cur = torch.cuda.current_stream(dev)

    def run(count):
        for s in range(count):
            i = s % in_flight
            with torch.cuda.stream(streams[i]):
                decs[i].batch_decide(ins, outs[i])

    run(max(warmup, in_flight))
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(cur)
    for st in streams:
        st.wait_event(e0)
    run(steps)
    for st in streams:
        e = torch.cuda.Event()
        e.record(st)
        cur.wait_event(e)
    e1.record(cur)
    torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1)
    parts = decs[0].partitions(outs[0], len(items))
    assert all(p.status == 0 for p in parts)
    stage = trs.trs_batch_stage_ms(decs[0].ctx)
    sf = trs.trs_batch_stage_frames(decs[0].ctx)
    for d in decs:
        d.close()
    luma_bytes = sum(it.spec.frame_bytes for it in items)
    half_bytes = sum(it.spec.frame_bytes for it in items[:sf])
    return {"value": len(items) * steps / (ms / 1e3), "unit": UNIT, "frames_per_step": len(items),
            "ms_per_step": ms / steps, "luma_gb_per_step": luma_bytes / 1e9, "in_flight": in_flight,
            "stage_ms": stage, "parts": n_parts, "stage_frames": sf,
            "texture_gbs": half_bytes / (stage["texture"] / 1e3) / 1e9, "autotune": tune}

def max_over_ranks(x: float, dist, device=None) -> float:
    """The slowest rank's time (every rank calls this with its own)."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank: float, world: int, seconds: float) -> float:
    """Whole-job throughput: every rank processed units_per_rank in the
    slowest rank's time (weak scaling, replicas)."""
    return world * units_per_rank / seconds


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), float(d.get("sm_max_mhz", 2070.0)), "measured"
    except Exception:
        return 6800.0, 2070.0, "fallback"


def ncu_traffic(stage: str, frames: int):
    """DRAM bytes per launch of a stage's kernel from the committed ncu
    capture (profiles/ncu_traffic.json), scaled to `frames`; None when there
    is none or the kernel's source changed since it was taken."""
    import hashlib
    try:
        with open(os.path.join(ROOT, "profiles", "ncu_traffic.json")) as f:
            k = json.load(f)["kernels"][stage]
        h = hashlib.sha256()
        for src in k["sources"]:  # the kernel's file and the headers it compiles with
            with open(os.path.join(ROOT, src), "rb") as f:
                h.update(f.read())
        if h.hexdigest()[:16] != k["sources_sha256_16"]:
            return None
        return (k["dram_read_bytes"] + k["dram_write_bytes"]) * frames / k["frames"]
    except Exception:
        return None


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


def cpu_baseline(frames, budget_s: float = 12.0, bd: int = 10, n: int = N_REGIONS, lam: float = LAMBDA,
                 what: str = "workload"):
    """The oracle (O2, one core) on a bounded sample of the same frames."""
    from oracle import oracle as O
    O.build()
    t0 = time.perf_counter()
    done = 0
    for plane, times in frames:
        O.decide(plane, times, bd, n, lam)
        done += 1
        if time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    return {"value": done / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{done} of the {len(frames)} {what} frames, oracle texture + Q16 + exact DP search, 1 thread"}


def _oracle_worker_init(shm_name, shape_p, shape_t, bd, n, lam):
    global _W
    from multiprocessing import shared_memory
    from oracle import oracle as O
    shm = shared_memory.SharedMemory(name=shm_name)
    n_p = int(np.prod(shape_p)) * 2
    planes = np.ndarray(shape_p, dtype=np.uint16, buffer=shm.buf[:n_p])
    times = np.ndarray(shape_t, dtype=np.float32, buffer=shm.buf[n_p:n_p + int(np.prod(shape_t)) * 4])
    _W = (shm, planes, times, O, bd, n, lam)


def _oracle_worker_decide(i: int) -> int:
    shm, planes, times, O, bd, n, lam = _W
    if i >= 0:
        plane = planes[i] if bd > 8 else planes[i].astype(np.uint8)
        O.decide(plane, times[i], bd, n, lam)
    return i


def _oracle_worker_decide_many(idx) -> int:
    for i in idx:
        _oracle_worker_decide(i)
    return len(idx)


def cpu_baseline_all_cores(frames, bd: int = 10, n: int = N_REGIONS, lam: float = LAMBDA, what: str = "workload",
                           min_s: float = 1.5):
    """The oracle as it stands, one process per host core (spawned), each
    deciding whole frames read from shared memory; wall-clock over all of
    them.  Each pass over the frames hands every process one task (frames
    i, i + cores, ...), so that small frames are not timed as inter-process
    messages; passes repeat until min_s of wall time has gone by."""
    import multiprocessing as mp
    from multiprocessing import shared_memory
    planes = np.stack([np.ascontiguousarray(p) for p, _ in frames]).astype(np.uint16)
    times = np.stack([t for _, t in frames]).astype(np.float32)
    shm = shared_memory.SharedMemory(create=True, size=planes.nbytes + times.nbytes)
    try:
        shm.buf[:planes.nbytes] = planes.tobytes()
        shm.buf[planes.nbytes:planes.nbytes + times.nbytes] = times.tobytes()
        cores = os.cpu_count() or 1
        ctx = mp.get_context("spawn")
        # bounded waits: a worker that cannot start is replaced by the pool
        # over and over, so an unbounded map would never return
        with ctx.Pool(cores, initializer=_oracle_worker_init,
                      initargs=(shm.name, planes.shape, times.shape, bd, n, lam)) as pool:
            try:
                pool.map_async(_oracle_worker_decide, [-1] * cores).get(timeout=180)  # workers up, oracle loaded
                tasks = [list(range(i, len(frames), cores)) for i in range(min(cores, len(frames)))]
                t0 = time.perf_counter()
                done = 0
                while True:
                    done += sum(pool.map_async(_oracle_worker_decide_many, tasks, chunksize=1).get(timeout=600))
                    dt = time.perf_counter() - t0
                    if dt >= min_s:
                        break
            except mp.TimeoutError:
                return {"value": None, "unavailable": "oracle worker processes did not finish in time"}
    finally:
        shm.close()
        shm.unlink()
    return {"value": done / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"all {len(frames)} {what} frames, {done // len(frames)} pass(es), oracle texture + Q16 + "
                      f"exact DP search, {cores} spawned processes"}


def run_serving(trs, device: int, duration_s: float = 7.0, saturate_s: float = 1.0,
                sweep_fracs=(0.1, 0.5, 0.9), sweep_s: float = 2.0):
    """32 concurrent streams (half 1080p10 n=8, half 2160p10 n=16) with
    Poisson arrivals at U[30, 60] fps each, through the continuous-batching
    server.  Latency = wait before the server accepted the frame (both of the
    stream's slots busy) + the server's submit-to-ready time.  Then the
    saturated rate (every stream keeps both slots busy) and the latency at
    offered loads of 10, 50 and 90 % of it (all stream rates scaled alike)."""
    import collections
    import gc

    import synth
    import torch

    streams = synth.serving_streams(32)
    arrivals = synth.poisson_arrivals(streams, duration_s)
    pool = {}
    for spec in (synth.SPEC_1080P10, synth.SPEC_2160P10):
        pool[spec.name] = [torch.from_numpy(np.ascontiguousarray(synth.make_frame(spec, seed=900 + k,
                                                                                   workload="serve")[0])
                                            .view(np.uint8)).pin_memory() for k in range(4)]
    srv = trs.trs_server_create(3840, 2160, max_regions=16, max_streams=32, max_batch=32, max_inflight=3,
                                device=device)
    try:
        sids = []
        for st in streams:
            sid = trs.trs_server_open_stream(srv, st.spec.width, st.spec.height, st.spec.bit_depth, st.n_regions,
                                             0.1)
            _, times = synth.make_frame(st.spec, seed=7, stream=st.stream, workload="serve")
            trs.trs_server_update_times(srv, sid, np.ascontiguousarray(times))
            sids.append(sid)

        def frame(i, f):
            buf = pool[streams[i].spec.name][f % 4]
            return buf, streams[i].spec.width * 2

        # warm-up: one frame per stream
        for i, sid in enumerate(sids):
            b, pitch = frame(i, 0)
            trs.trs_server_submit(srv, sid, b, pitch)
        got = 0
        while got < len(sids):
            got += len(trs.trs_server_poll(srv, 64, 100_000))

        def poisson_run(arr):
            """Submits each arrival at its time; latency from arrival to ready (ms)."""
            lat = []
            waiting = collections.deque()
            accepted = {}
            t0 = time.perf_counter()
            k = 0
            while k < len(arr) or waiting or accepted:
                now = time.perf_counter() - t0
                while k < len(arr) and arr[k][0] <= now:
                    waiting.append(arr[k])
                    k += 1
                still = collections.deque()
                for (ta, i, f) in waiting:
                    b, pitch = frame(i, f)
                    try:
                        tk = trs.trs_server_submit(srv, sids[i], b, pitch)
                        accepted[tk] = (time.perf_counter() - t0) - ta
                    except trs.TrsError as e:
                        if e.status != trs.EBUSY:
                            raise
                        still.append((ta, i, f))
                waiting = still
                nxt = arr[k][0] - (time.perf_counter() - t0) if k < len(arr) else 0.0
                for d in trs.trs_server_poll(srv, 64, int(max(50, min(2000, nxt * 1e6)))):
                    assert d.status == 0
                    lat.append(accepted.pop(d.ticket) * 1e3 + d.latency_us / 1e3)
            return np.array(lat), time.perf_counter() - t0

        # Poisson arrivals at the workload's rates.  The objects alive now
        # (torch, numpy, the frames) are moved out of the cyclic collector's
        # reach first, so that no full collection over them runs inside the
        # submitting loop, where its time would be counted as latency
        gc.collect()
        gc.freeze()
        lat, elapsed = poisson_run(arrivals)

        # saturation: every stream keeps both request slots busy
        done = 0
        f = 0
        t1 = time.perf_counter()
        while time.perf_counter() - t1 < saturate_s:
            for i, sid in enumerate(sids):
                b, pitch = frame(i, f)
                try:
                    trs.trs_server_submit(srv, sid, b, pitch)
                except trs.TrsError as e:
                    if e.status != trs.EBUSY:
                        raise
            f += 1
            done += len(trs.trs_server_poll(srv, 64, 200))
        while trs.trs_server_info(srv).inflight:
            done += len(trs.trs_server_poll(srv, 64, 10_000))
        sat_dt = time.perf_counter() - t1
        saturated = done / sat_dt
        # latency under load: the same streams, every rate scaled so that the
        # offered load is a fraction of the saturated rate
        natural = sum(st.fps for st in streams)
        sweep = []
        for frac in sweep_fracs:
            scale = frac * saturated / natural
            scaled = [synth.StreamSpec(st.stream, st.spec, st.n_regions, st.fps * scale) for st in streams]
            arr = synth.poisson_arrivals(scaled, sweep_s, seed=60 + int(frac * 100))
            sl, sdt = poisson_run(arr)
            sweep.append({"offered_frac_of_saturated": frac, "offered_per_s": len(arr) / sweep_s,
                          "achieved_per_s": len(sl) / sdt, "decisions": int(len(sl)),
                          "p50_ms": float(np.percentile(sl, 50)), "p99_ms": float(np.percentile(sl, 99)),
                          "max_ms": float(sl.max())})
        info = trs.trs_server_info(srv)
        return {"streams": len(sids), "offered_per_s": len(arrivals) / duration_s,
                "decisions": int(len(lat)), "achieved_per_s": len(lat) / elapsed,
                "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                "max_ms": float(lat.max()), "saturated_per_s": saturated, "load_sweep": sweep,
                "mean_batch": info.frames / max(1, info.batches), "device_bytes": int(info.mem_used_bytes),
                "form": "continuous batching, 3 batches in flight on separate CUDA streams"}
    finally:
        gc.unfreeze()
        trs.trs_server_destroy(srv)


def run_multi_tile(runtime, trs, device: int, reps: int = 50, ns=(6, 7, 8)):
    """Multi-tile rectangular slices (trs_search_mt) on one 1920x1080 frame:
    the slice-set list is built on the host once per shape (timed apart), then
    the device search (one graph: two passes over the list, one decode warp)
    is timed alone with CUDA events on its stream."""
    import torch
    import synth
    spec = synth.SPEC_1080P10
    W, H = spec.width, spec.height
    plane, times = synth.make_frame(spec, seed=7)
    dev = f"cuda:{device}"
    dec = runtime.Decider(max_width=W, max_height=H, max_regions=8, max_batch=1, device=device)
    res = []
    try:
        luma, pitch = runtime.luma_to_device(plane, dev)
        st = dec.stats_buffers(W, H)
        dec.texture_map(luma, W, H, pitch, spec.bit_depth, st)
        tab = dec.tables_buffer(W, H)
        dec.region_tables(st, torch.from_numpy(times).to(dev), W, H, tab)
        out = torch.zeros(trs.MT_PARTITION_BYTES, dtype=torch.uint8, device=dev)
        s = torch.cuda.current_stream(device)
        for n in ns:
            t0 = time.perf_counter()
            trs.trs_search_mt(dec.ctx, tab, W, H, n, 0.1, out)
            torch.cuda.synchronize(device)
            build_s = time.perf_counter() - t0
            for _ in range(3):
                trs.trs_search_mt(dec.ctx, tab, W, H, n, 0.1, out)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize(device)
            e0.record(s)
            for _ in range(reps):
                trs.trs_search_mt(dec.ctx, tab, W, H, n, 0.1, out)
            e1.record(s)
            torch.cuda.synchronize(device)
            ms = e0.elapsed_time(e1) / reps
            rec = trs.trs_mt_partition.from_buffer_copy(out.cpu().numpy().tobytes())
            one = dec.partitions(dec.search(tab, W, H, n, 0.1))[0]
            # one rectangle-table index per slice: 16-bit when every index fits
            # (slice counts with a compiled kernel, n <= 8), else 32-bit
            C_, R_ = -(-W // 128), -(-H // 128)
            entry_bytes = 2 if n <= 8 and C_ * (C_ + 1) // 2 * R_ * R_ <= 65536 else 4
            list_bytes = rec.candidates * n * entry_bytes
            res.append({"frame": "1920x1080", "n": n, "lambda": 0.1, "status": rec.status,
                        "slice_sets": rec.candidates, "list_build_s": round(build_s, 3),
                        "ms_per_search": ms, "searches_per_s": 1e3 / ms,
                        "slice_sets_per_s": rec.candidates / (ms / 1e3),
                        "list_bytes": list_bytes, "list_read_gbs": 2 * list_bytes / (ms / 1e3) / 1e9,
                        "launches_per_search": 1, "t_min_multi_tile": rec.t_min,
                        "t_min_single_tile_row": one.t_min, "q_multi_tile": rec.q, "q_single_tile_row": one.q})
    finally:
        dec.close()
    return {"searches": res,
            "note": "one graph launch per search: argument copy, two passes over the list, decode; "
                    "list_read_gbs counts two reads of the list (2 bytes per slice at 1920x1080)"}


def run_reference(args, rank, world):
    """Reference arm: the oracle timed on this host's cores, same metric."""
    if rank != 0:
        return
    frames, _, _ = make_inputs(min(NFRAMES, 8))
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
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-mixed", action="store_true")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the 832x480 n=4 and 1920x1080 n=8 configurations")
    ap.add_argument("--no-light", action="store_true")
    ap.add_argument("--no-mt", action="store_true", help="skip the multi-tile slice search timing")
    ap.add_argument("--mt-only", action="store_true",
                    help="only the multi-tile search at 1920x1080, n = 6, 7 and 8, 50 timed calls each")
    ap.add_argument("--no-tune", action="store_true",
                    help="keep the default launch shapes (short profiling runs)")
    ap.add_argument("--in-flight", type=int, default=IN_FLIGHT, choices=[1, 2, 3, 4],
                    help="batches in flight (contexts on separate streams)")
    ap.add_argument("--parts", type=int, default=PARTS, choices=[1, 2, 3, 4],
                    help="chunks a captured batch is pipelined in")
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
    if args.mt_only:
        import __graft_entry__
        __graft_entry__.build()
        from paper_2012_14792_gb300 import runtime, trs
        print(json.dumps({"multi_tile": run_multi_tile(runtime, trs, local)}), flush=True)
        return

    nfr = args.frames
    # spawn pool, before any CUDA call
    frames, mixed, cfg_frames = make_inputs(nfr, mixed=not args.no_mixed, configs=not args.no_configs)

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

    # --- batched, timed: a stream of batches, IN_FLIGHT of them in flight ----
    # Each step decides the whole 64-frame batch through trs_batch_decide.
    # Consecutive steps alternate between IN_FLIGHT contexts, each on its own
    # CUDA stream (double-buffered submission, as a serving pipeline runs),
    # so one batch's HBM-bound texture map overlaps another's ALU-bound search.
    tune = None if args.no_tune else dec.autotune(ins)  # launch shapes picked on this workload
    trs.trs_set_batch_parts(dec.ctx, args.parts)
    decs = [dec] + [runtime.Decider(max_width=3840, max_height=2160, max_regions=N_REGIONS, max_batch=nfr,
                                    device=local) for _ in range(args.in_flight - 1)]
    outs = [out] + [torch.zeros_like(out) for _ in range(args.in_flight - 1)]
    streams = [torch.cuda.Stream(dev) for _ in range(args.in_flight)]
    for d in decs[1:]:
        if tune is not None:
            trs.trs_set_tune(d.ctx, tune["band_warps"], tune["col_warps"], tune["col_batch"])
        trs.trs_set_batch_parts(d.ctx, args.parts)

    def run_steps(count: int, flight: int, inputs=None):
        for s in range(count):
            i = s % flight
            with torch.cuda.stream(streams[i]):
                decs[i].batch_decide(ins if inputs is None else inputs, outs[i])

    def timed(count: int, flight: int, inputs=None) -> float:
        """Device time of `count` steps: every stream starts after ev0, ev1 after all of them."""
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for st in streams[:flight]:
            st.wait_event(ev0)
        run_steps(count, flight, inputs)
        for st in streams[:flight]:
            e = torch.cuda.Event()
            e.record(st)
            stream.wait_event(e)
        ev1.record(stream)
        sync_all()
        return ev0.elapsed_time(ev1)

    run_steps(max(args.warmup, args.in_flight), args.in_flight)
    sync_all()
    launches = trs.trs_batch_kernels(dec.ctx) * args.steps  # the same graph every step
    with ClockSampler(local) as clk:
        ms = timed(args.steps, args.in_flight)
    stage_overlap = trs.trs_batch_stage_ms(dec.ctx)  # CUDA events inside the graph (this context's last step)
    overlap_frames = trs.trs_batch_stage_frames(dec.ctx)  # the first chunk of the batch
    ms = max_over_ranks(ms, dist, dev)
    value = job_throughput(nfr * args.steps, world, ms / 1e3)
    parts = dec.partitions(out, nfr)
    assert all(p.status == 0 for p in parts), [p.status for p in parts]
    for o in outs[1:]:
        assert bytes(o.cpu().numpy()) == bytes(out.cpu().numpy())  # every context decides the same bytes
    # the same steps one batch at a time on one stream
    one_ms = max_over_ranks(timed(max(3, args.steps // 2), 1), dist, dev)
    one_batch = {"value": job_throughput(nfr * max(3, args.steps // 2), world, one_ms / 1e3), "unit": UNIT,
                 "ms_per_step": one_ms / max(3, args.steps // 2), "form": "one batch in flight, one stream"}

    # the same stream of steps on device-resident packed planes (TRS_PACKED10)
    import synth
    lumas_pk = [torch.from_numpy(synth.pack10(p)).to(dev) for p, _ in frames]
    ins_pk = [(l, l.shape[1], 3840, 2160, trs.PACKED10, t, N_REGIONS, LAMBDA) for l, t in zip(lumas_pk, tts)]
    ref_bytes = bytes(out.cpu().numpy())
    run_steps(max(args.warmup, args.in_flight), args.in_flight, ins_pk)
    sync_all()
    pk_steps = max(3, args.steps // 2)
    pk_ms = max_over_ranks(timed(pk_steps, args.in_flight, ins_pk), dist, dev)
    for o in outs:
        assert bytes(o.cpu().numpy()) == ref_bytes  # the same decisions as the two-byte planes
    packed_res = {"value": job_throughput(nfr * pk_steps, world, pk_ms / 1e3), "unit": UNIT,
                  "ms_per_step": pk_ms / pk_steps,
                  "luma_bytes_per_step": int(sum(l.numel() for l in lumas_pk)),
                  "form": "the same stream of steps, planes in the packed 10-bit format (four samples in five "
                          "bytes) resident in HBM"}
    del lumas_pk, ins_pk

    # --- kernels alone: the batch as one launch chain, no second half running
    # beside it; the per-kernel durations of the roofline, averaged over steps
    trs.trs_set_batch_parts(dec.ctx, 1)
    for _ in range(3):
        dec.batch_decide(ins, out)
    iso_steps = max(5, args.steps // 10)
    acc = {}
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(iso_steps):
        dec.batch_decide(ins, out)
        torch.cuda.synchronize(dev)
        for k, v in trs.trs_batch_stage_ms(dec.ctx).items():
            acc[k] = acc.get(k, 0.0) + v / iso_steps
    e1.record(stream)
    torch.cuda.synchronize(dev)
    stage, stage_frames = acc, trs.trs_batch_stage_frames(dec.ctx)
    no_overlap = {"value": nfr * iso_steps / (e0.elapsed_time(e1) / 1e3), "unit": UNIT,
                  "note": "one launch chain over all frames, a host sync per step"}
    trs.trs_set_batch_parts(dec.ctx, args.parts)
    assert bytes(dec.partitions(out, 1)[0]) == bytes(parts[0])

    # --- lightweight search: every 4th area window --------------------------
    light = None
    if not args.no_light:
        for d in decs:
            trs.trs_set_window_step(d.ctx, 4)
        run_steps(max(args.warmup, args.in_flight), args.in_flight)
        sync_all()
        l_steps = max(3, args.steps // 4)
        l_ms = timed(l_steps, args.in_flight)  # the same stream of steps as `value`
        lp = dec.partitions(out, nfr)
        for d in decs:
            trs.trs_set_window_step(d.ctx, 1)
        tr = np.array([a.t_q / b.t_q for a, b in zip(lp, parts)])
        qr = np.array([a.q / max(1, b.q) for a, b in zip(lp, parts)])
        light = {"window_step": 4, "value": nfr * l_steps / (l_ms / 1e3), "unit": UNIT,
                 "in_flight": args.in_flight,
                 "identical_frac": float(np.mean([a.x_edges() == b.x_edges() and a.band_cuts() == b.band_cuts()
                                                  for a, b in zip(lp, parts)])),
                 "t_ratio_mean": float(tr.mean()), "t_ratio_max": float(tr.max()),
                 "q_ratio_mean": float(qr.mean()), "q_ratio_max": float(qr.max()),
                 "note": "T(P) and Q(P) of the lightweight decision over the exact one, same frames"}

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
    # Two input forms of the same 10-bit samples: the packed format
    # (TRS_PACKED10, four samples in five bytes: what a capture pipeline
    # hands over, 37.5 % fewer bytes on the host link) and two bytes per
    # sample.  Both decide the same bytes (checked).
    import synth
    pinned = [torch.from_numpy(np.ascontiguousarray(p).view(np.uint8)).pin_memory() for p, _ in frames]
    pinned_pk = [torch.from_numpy(synth.pack10(p)).pin_memory() for p, _ in frames]
    pinned_t = [torch.from_numpy(t).pin_memory() for _, t in frames]
    import threading

    # host threads of the end-to-end form: the host link bounds it, and a
    # third thread measured slower on two-byte planes (9.5 k against 12.1 k
    # decisions/s; 18.2 k either way on packed planes)
    e2e_threads = min(args.in_flight, E2E_THREADS)

    def e2e_run(descs, lumas, form):
        # a stream of steps like the timed region's: e2e_threads host threads,
        # each calling the synchronous host-buffer entry point on its own
        # context and stream, so one batch's copies overlap another's kernels
        for i in range(e2e_threads):
            for _ in range(2):
                trs.trs_batch_decide_host(decs[i].ctx, descs, streams[i])
        sync_all()
        e_steps = max(3, args.steps // 4)
        e_steps += (-e_steps) % e2e_threads
        results = [None] * e2e_threads

        def host_worker(i: int):
            for _ in range(e_steps // e2e_threads):
                results[i] = trs.trs_batch_decide_host(decs[i].ctx, descs, streams[i])

        workers = [threading.Thread(target=host_worker, args=(i,)) for i in range(e2e_threads)]
        t0 = time.perf_counter()
        for t in workers:
            t.start()
        for t in workers:
            t.join()
        sync_all()
        dt = max_over_ranks(time.perf_counter() - t0, dist, dev)
        for hp in results:
            assert bytes(hp[0]) == bytes(parts[0])
        return {"value": job_throughput(nfr * e_steps, world, dt), "unit": UNIT,
                "h2d_bytes_per_step": int(sum(p.numel() for p in lumas) + sum(t.numel() * 4 for t in pinned_t)),
                "d2h_bytes_per_step": nfr * trs.PARTITION_BYTES,
                "form": f"trs_batch_decide_host from pinned host buffers ({form}), {e2e_threads} host threads "
                        "with a context and stream each"}

    pk_bytes = (10 * 3840 + 7) // 8
    e2e = e2e_run([trs.frame_desc(pinned_pk[i], pinned_t[i], 3840, 2160, pk_bytes, trs.PACKED10, N_REGIONS,
                                  LAMBDA) for i in range(nfr)], pinned_pk,
                  "10-bit samples packed four in five bytes, TRS_PACKED10")
    e2e_two_byte = e2e_run([trs.frame_desc(pinned[i], pinned_t[i], 3840, 2160, 7680, 10, N_REGIONS, LAMBDA)
                            for i in range(nfr)], pinned, "two bytes per 10-bit sample")

    # --- rooflines: every kernel of the step, from the one-chunk stage times -
    hbm, sm_max, src = peaks()
    tex_bytes = sum(p.numel() for p in pinned[:stage_frames])  # each luma sample read once
    row_relax, col_relax = trs.trs_plan_work(3840, 2160, N_REGIONS)
    # each DP transition is one combine (max or +) and one minimum: 2 INT32
    # operations (step 1 runs on 32-bit values for these frames); the peak is
    # this GPU's measured INT32 add/min/max throughput
    alu_peak = trs.trs_alu_peak(local) / 1e12  # T INT32 ops / s
    lay = trs.trs_tables_layout_get(3840, 2160)
    # the tables kernel writes every slice's time and floor SSE (2 x 8 bytes), the
    # Q16 times and three SATs, and reads the statistics and the time map
    C_, R_ = lay.cols, lay.rows
    tab_bytes = stage_frames * (lay.bands * R_ * (R_ + 1) // 2 * 16 + C_ * R_ * (4 + 4 + 8 + 4 + 4)
                                + 3 * (C_ + 1) * (R_ + 1) * 8)
    stage_sum = sum(stage.values()) if stage else 0.0
    kernels = {"texture": "texture_kernel", "tables": "tables_kernel", "step1_rows": "band_kernel<1>",
               "step1_columns": "column_kernel<1>", "step2_rows": "band_kernel<2>",
               "step2_columns": "column_kernel<2>", "rebuild": "rebuild_kernel + cuts_kernel",
               "decode": "finish_kernel"}

    def hbm_roof(kind, nbytes):
        gbs = nbytes / (stage[kind] / 1e3) / 1e9
        return {"kernel": kernels[kind], "bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s",
                "frac": gbs / hbm, "traffic": ncu_traffic(kind, stage_frames), "algorithmic_bytes": nbytes,
                "ms": stage[kind], "share": stage[kind] / stage_sum, "peak_source": src}

    def alu_roof(kind, work, note):
        ops = 2.0 * work * stage_frames
        ach = ops / (stage[kind] / 1e3) / 1e12
        return {"kernel": kernels[kind], "bound": "alu", "achieved": ach, "peak": alu_peak,
                "unit": "T INT32 ops/s", "frac": ach / alu_peak, "traffic": ncu_traffic(kind, stage_frames),
                "algorithmic_ops": ops, "work": note, "ms": stage[kind], "share": stage[kind] / stage_sum,
                "peak_source": "measured: trs_alu_peak (32-bit add/min/max chains on every SM)"}

    rooflines = [
        hbm_roof("texture", tex_bytes),
        hbm_roof("tables", tab_bytes),
        alu_roof("step1_rows", row_relax, "trs_plan_work row_relax x 2 ops x frames"),
        alu_roof("step1_columns", col_relax, "trs_plan_work col_relax x 2 ops x frames"),
        alu_roof("step2_rows", row_relax, "trs_plan_work row_relax x 2 ops x frames; step 2 skips the items "
                                          "of windows that break Eq. 4, so this over-counts its work"),
        alu_roof("step2_columns", col_relax, "trs_plan_work col_relax x 2 ops x frames; over-counts like step-2 "
                                             "rows"),
    ] + [{"kernel": kernels[k], "bound": "latency", "ms": stage[k], "share": stage[k] / stage_sum,
          "note": "dependent warp chains per frame or tied window: no throughput roofline"}
         for k in ("rebuild", "decode")]
    by_name = {r["kernel"]: r for r in rooflines}
    roof = dict(by_name[ROOFLINE_KERNEL])  # a fixed kernel: the search family's largest, by measurement
    tex_roof = by_name["texture_kernel"]
    search_keys = ("step1_rows", "step1_columns", "step2_rows", "step2_columns", "rebuild", "decode")
    search_share = sum(stage[k] for k in search_keys) / stage_sum if stage_sum else None

    # the candidate space the exact search covers (distinct partitions of S(n), one tile row)
    space = trs.trs_count_partitions(3840, 2160, N_REGIONS)
    search_ms = sum(stage.get(k, 0.0) for k in ("step1_rows", "step1_columns", "step2_rows", "step2_columns",
                                                "rebuild", "decode"))
    search_space = {"partitions": space,
                    "effective_candidates_per_s": space * value,
                    "effective_candidates_per_s_search_only": space * nfr / (search_ms / 1e3) if search_ms else None,
                    "note": "|S(n)| at 3840x2160, n = 16, k = 3 (exact count, one tile row: tile rows add codes, "
                            "not partitions) x decisions/s; search only: over the search kernels' one-chunk time"}

    serving = None
    if not args.no_serving:
        serving = run_serving(trs, local)
    mixed_res = None
    if mixed is not None:
        mixed_res = run_mixed(runtime, trs, mixed, local, max(3, args.steps // 20), args.warmup, args.parts,
                              args.in_flight)

    multi_tile = None
    if not args.no_mt:
        try:
            multi_tile = run_multi_tile(runtime, trs, local)
        except Exception as e:  # a secondary figure: report it, keep the headline line
            multi_tile = {"error": f"{type(e).__name__}: {e}"}

    configs_res = None
    if cfg_frames is not None:
        import synth
        configs_res = {}
        for key, (name, n_cfg) in CONFIGS.items():
            configs_res[key] = run_config(runtime, trs, getattr(synth, name), n_cfg, cfg_frames[key], local,
                                          max(5, args.steps // 4), args.warmup, args.in_flight)

    cpu = cpu_all = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(frames)
        cpu_all = cpu_baseline_all_cores(frames)
        if configs_res:
            import synth
            for key, (name, n_cfg) in CONFIGS.items():
                bd = getattr(synth, name).bit_depth
                configs_res[key]["cpu_baseline"] = cpu_baseline(cfg_frames[key], 3.0, bd, n_cfg, LAMBDA,
                                                                "configuration")
                configs_res[key]["cpu_baseline_all_cores"] = cpu_baseline_all_cores(cfg_frames[key], bd, n_cfg,
                                                                                    LAMBDA, "configuration")

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
                "config": {"workload": WORKLOAD if nfr == NFRAMES else f"{WORKLOAD} (first {nfr} frames)",
                           "frames_per_step": nfr,
                           "form": f"batched, CUDA graph, {args.parts} pipelined chunks, "
                                   f"{args.in_flight} batches in flight (contexts on separate streams)",
                           "l2": f"inputs {nfr * 16588800 / 1e9:.2f} GB per step > L2, no flush"},
                "one_batch_in_flight": one_batch,
                "plain": {"value": plain_value, "unit": UNIT, "form": "one frame per launch chain"},
                "stage_ms": stage, "stage_frames": stage_frames,
                "stage_ms_overlapped": stage_overlap, "stage_frames_overlapped": overlap_frames,
                "no_overlap": no_overlap, "autotune": tune, "mixed_256": mixed_res, "lightweight": light,
                "serving": serving, "multi_tile": multi_tile,
                "clocks": clk.summary(), "e2e": e2e, "e2e_two_byte": e2e_two_byte, "packed": packed_res,
                "gpu_launches": launches, "roofline": roof, "roofline_texture": tex_roof,
                "rooflines": rooflines, "search_share_of_stage_sum": search_share,
                "config_480p8_n4": configs_res.get("config_480p8_n4") if configs_res else None,
                "config_1080p10_n8": configs_res.get("config_1080p10_n8") if configs_res else None,
                "search_space": search_space,
                "cpu_baseline": cpu, "cpu_baseline_all_cores": cpu_all}
        print(json.dumps(line), flush=True)
    for d in decs:
        d.close()
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
