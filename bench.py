#!/usr/bin/env python
"""Throughput benchmark of the forward-tracking path on GB300.

One step = one pass of the whole path over one batch: hit packing (bucket +
sort), windows, triplet seeding, extension and fit, selection and compaction
(persistent form, one CUDA graph per launch shape).  Inputs are synthetic,
seeded, generated on the device before timing; they are larger than L2, so no
flush is needed between steps.

Printed (rank 0): one JSON line with events/s, the roofline of the dominant
kernel measured live with CUDA events, the end-to-end number through the
host-buffer entry point lf_process_host, the plain (one kernel per stage)
form on the same data, the CPU oracle on a bounded sample, clocks.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun each rank runs its own replica (independent events, weak
scaling, no collective on the data path); rank 0 prints the max-over-ranks time.
"""
from __future__ import annotations

import argparse
import dataclasses
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

import numpy as np  # noqa: E402
import torch  # noqa: E402

METRIC = "events/s/GB300 at oracle match (plain vs batched/served); served p50/p99 latency"
UNIT = "events/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--config", type=int, default=2, help="synthetic workload id (2 = uneven 100k-event batch)")
    ap.add_argument("--events", type=int, default=None)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--no-no-ut", action="store_true", help="skip the no-UT variant measurement")
    ap.add_argument("--cpu-events", type=int, default=5000, help="oracle sample size (events)")
    ap.add_argument("--tuning", type=str, default=None, help="json of lf_tuning fields (skips the autotuner)")
    ap.add_argument("--no-tune", action="store_true", help="default launch shape instead of the autotuner's")
    return ap.parse_args()


# ------------------------------------------------------------------ helpers

def dist_setup(args):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    elif torch.cuda.is_available():
        torch.cuda.set_device(0)
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(ws, v: float) -> float:
    if ws <= 1:
        return v
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []
        self.th = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except OSError:
            self.proc = None

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.th:
            self.th.join(timeout=2)
        sm, mx, reasons, pw = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
                pw.append(float(f[3]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        load = [s for s, p in zip(sm, pw) if p > 200.0] or sm
        return {"sm_mhz": float(statistics.median(load)), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm), "power_w_max": max(pw)}


def host_copy(batch, arena_bytes_extra: int = 0):
    """Copy a device EventBatch into one page-locked arena (cudaHostAlloc
    through lf_host_alloc: copies from it overlap device work)."""
    from paper_2402_14670_gb300 import lf
    fields = ("raw_offsets", "x", "z", "dxdy", "w", "plane", "trk_offsets", "sx", "sy", "stx", "sty", "sqop")
    total = sum(getattr(batch, f).numel() * getattr(batch, f).element_size() + 256 for f in fields)
    arena = lf.HostArena(total + arena_bytes_extra)
    kw = {}
    for f in fields:
        src = getattr(batch, f)
        dst = arena.take(src.numel(), src.dtype)
        dst.copy_(src)
        kw[f] = dst
    from paper_2402_14670_gb300 import synth
    return synth.EventBatch(batch.n_events, **kw), arena


def on_node(node_cpus, fn):
    """Run fn with this process bound to the given CPUs (page-locked memory
    it allocates is placed on their NUMA node), then restore the binding."""
    if not node_cpus:
        return fn()
    old = os.sched_getaffinity(0)
    try:
        os.sched_setaffinity(0, node_cpus)
        return fn()
    finally:
        os.sched_setaffinity(0, old)


def numa_link(n_bytes: int = 1 << 30) -> dict:
    """The GPU's nearest host NUMA node and the host-to-device copy rate
    from page-locked memory placed on each node this process may use."""
    from paper_2402_14670_gb300 import lf
    nodes = lf.numa_node_cpus()
    out = {"gpu_host_numa_node": lf.lf_device_host_numa(), "nodes": {}}
    dst = torch.empty(n_bytes // 4, dtype=torch.float32, device="cuda")
    for node, cpus in nodes.items():
        arena = on_node(cpus, lambda: lf.HostArena(n_bytes + 256))
        src = arena.take(n_bytes // 4, torch.float32)
        src.fill_(1.0)
        best = 0.0
        for _ in range(3):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            dst.copy_(src, non_blocking=True)
            torch.cuda.synchronize()
            best = max(best, n_bytes / (time.perf_counter() - t0) / 1e9)
        out["nodes"][str(node)] = {"cpus": len(cpus), "h2d_gbps": best}
        del src
        arena.close()
    del dst
    return out


def sub_batches(batch, size: int):
    """Views of consecutive `size`-event sub-batches (offsets rebased)."""
    from paper_2402_14670_gb300 import synth
    ro = batch.raw_offsets.cpu().numpy().astype(np.int64)
    to = batch.trk_offsets.cpu().numpy().astype(np.int64)
    out = []
    for e0 in range(0, batch.n_events, size):
        e1 = min(e0 + size, batch.n_events)
        h0, h1, t0, t1 = int(ro[e0]), int(ro[e1]), int(to[e0]), int(to[e1])
        sub = synth.EventBatch(
            e1 - e0, (batch.raw_offsets[e0:e1 + 1] - h0).contiguous(), batch.x[h0:h1], batch.z[h0:h1],
            batch.dxdy[h0:h1], batch.w[h0:h1], batch.plane[h0:h1], (batch.trk_offsets[e0:e1 + 1] - t0).contiguous(),
            batch.sx[t0:t1], batch.sy[t0:t1], batch.stx[t0:t1], batch.sty[t0:t1], batch.sqop[t0:t1])
        out.append((sub, h0, h1, t0, t1))
    return out


def per_batch_plain(tr, batch, packed, out, size: int):
    """Closure running the plain form per `size`-event batch (pack + one
    launch per stage per batch) over the whole workload."""
    from paper_2402_14670_gb300 import lf
    subs = sub_batches(batch, size)
    dev = batch.x.device
    plans = []
    for sub, h0, h1, t0, t1 in subs:
        pk = {k: packed[k][h0:h1] for k in ("x", "z", "dxdy", "w", "layer", "perm")}
        pk["hit_offsets"] = torch.empty(24 * sub.n_events + 1, dtype=torch.int32, device=dev)
        pk["x_coarse"] = torch.empty(lf.coarse_count(h1 - h0), dtype=torch.float32, device=dev)
        ot = {k: out[k][t0:t1] for k in ("found", "nhits", "hit_idx", "state", "quality")}
        ot["out_offsets"] = torch.empty(sub.n_events + 1, dtype=torch.int32, device=dev)
        ot["out_trk"] = out["out_trk"][t0:t1] if t1 > t0 else out["out_trk"][:1]
        ot["n_out"] = torch.empty(1, dtype=torch.int32, device=dev)
        plans.append((sub, pk, ot))

    def run():
        for sub, pk, ot in plans:
            tr.pack(sub, out=pk)
            tr.find(pk, sub, sub.n_events, "plain", out=ot)
    return run


def workload_recipe(cfg) -> str:
    """One line describing a synthetic workload's event recipe."""
    n_in = cfg.n_in
    if n_in[0] == "negbin":
        trk = "NegBin(mean %g, r=%g) input tracks per event clipped to [%d,%d]" % n_in[1:]
    elif n_in[0] == "poisson":
        trk = "Poisson(%g) input tracks per event" % n_in[1]
    elif n_in[0] == "uniform":
        trk = "U{%d..%d} input tracks per event" % n_in[1:]
    else:
        trk = "%d input tracks per event" % n_in[1]
    noise = ("%d%% noise hits" % round(100 * cfg.noise[1])) if cfg.noise[0] == "frac" else \
        ("%d noise hits per layer" % cfg.noise[1])
    return "%s, %d%% matched to a particle, p %g-%g GeV, %s" % (trk, round(100 * cfg.match_frac), cfg.p_min,
                                                               cfg.p_max, noise)


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def algorithmic_bytes(n_events, n_hits, n_tracks, n_found):
    """Each input read once and each output written once: 16 B per packed
    hit (x, z, dxdy, w), 25 offsets per event, 20 B per input state, 84 B per
    found track (12 hit indices, 6 state words, Q, counts, compact index)."""
    return 16 * n_hits + 4 * 25 * n_events + 20 * n_tracks + 84 * n_found


def pack_bytes(n_events, n_hits):
    """Packing: 17 B read per raw hit (x, z, dxdy, w, plane) and 21 B written
    (x, z, dxdy, w, layer, perm) plus the raw and bucket offsets."""
    return 38 * n_hits + 4 * (24 + 1 + 1) * n_events


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    for f in ("lf_track.cu", "lf_device.cuh", "lf_internal.h"):
        h.update(open(os.path.join(ROOT, "paper_2402_14670_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def pack_source_hash() -> str:
    h = hashlib.sha256()
    for f in ("lf_pack.cu", "lf_internal.h"):
        h.update(open(os.path.join(ROOT, "paper_2402_14670_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def profile_for(config: int, key: str, digest: str):
    """The committed ncu figures of one workload (DRAM bytes and warp
    instructions of the captured launches), or None when that workload has
    no capture or the captured sources (key: their hash field) changed."""
    p = os.path.join(ROOT, "profiles", "find_traffic.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p))
    if d.get(key) != digest:
        return None
    if int(d.get("config", 2)) == config:
        return d
    return d.get("configs", {}).get(str(config))


def pack_traffic_per_launch(config: int, units_hits: int):
    """DRAM bytes of k_pack_event from the committed capture of this
    workload, scaled to this launch by hits, or None (no capture, or the pack
    kernel changed since)."""
    d = profile_for(config, "pack_source_sha256_16", pack_source_hash())
    if d is None:
        return None
    k = [v for n, v in d.get("kernels", {}).items() if "k_pack" in n]
    if len(k) != 1:
        return None
    return (float(k[0]["read_gb"]) + float(k[0]["write_gb"])) * 1e9 * units_hits / float(d["hits"])


def find_profile(config: int):
    """The committed ncu figures of the find kernels on this workload (one
    launch on a slice of it), or None (no capture, or the kernels changed
    since)."""
    return profile_for(config, "kernel_source_sha256_16", kernel_source_hash())


def traffic_per_launch(config: int, units_hits: int):
    """DRAM bytes of the find kernels from the committed capture of this
    workload, scaled to this launch by hits, or None."""
    d = find_profile(config)
    if d is None:
        return None
    return float(d["dram_bytes_per_launch"]) * units_hits / float(d["hits"])


# --------------------------------------------------------------- oracle arm

def time_oracle(batch_cpu, threads: int):
    import oracle
    t = lambda a: a.numpy()
    t0 = time.perf_counter()
    pk = oracle.pack(t(batch_cpu.raw_offsets), t(batch_cpu.x), t(batch_cpu.z), t(batch_cpu.dxdy), t(batch_cpu.w),
                     t(batch_cpu.plane), n_threads=threads)
    states = dict(trk_offsets=t(batch_cpu.trk_offsets), sx=t(batch_cpu.sx), sy=t(batch_cpu.sy),
                  stx=t(batch_cpu.stx), sty=t(batch_cpu.sty), sqop=t(batch_cpu.sqop))
    res = oracle.find_tracks(pk, states, dumps=False, n_threads=threads)
    oracle.compact(states["trk_offsets"], res["found"])
    return time.perf_counter() - t0, res


def run_reference(args, ws, rank):
    if rank != 0:
        return
    from paper_2402_14670_gb300 import synth
    cfg = synth.CONFIGS[args.config]
    threads = len(os.sched_getaffinity(0)) or 1
    n = min(args.cpu_events, cfg.n_events)
    sample = synth.generate(args.config, n_events=n, truth=False)
    times = []
    for i in range(args.warmup + args.steps):
        dt, res = time_oracle(sample, threads)
        if i >= args.warmup:
            times.append(dt)
    total = sum(times)
    value = n * len(times) / total
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / len(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "%s (config %d) oracle sample" % (cfg.name, args.config), "events_per_step": n,
                   "parallelism": "host threads over events"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": "%d events of the %s workload per step, pack+find+compact" % (n, cfg.name)},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- GPU arm

def main():
    args = parse()
    ws, rank, local = dist_setup(args)
    if args.impl == "reference":
        run_reference(args, ws, rank)
        if ws > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device")
    from paper_2402_14670_gb300 import build
    build.build()
    from paper_2402_14670_gb300 import lf, synth

    cfg = synth.CONFIGS[args.config]
    n_ev = args.events or cfg.n_events
    # weak scaling: every rank draws its own events
    cfg_r = cfg if rank == 0 else dataclasses.replace(cfg, seed=cfg.seed * 1000 + rank)
    batch = synth.generate(cfg_r, n_events=n_ev, device="cuda", truth=False)
    torch.cuda.synchronize()
    tuning = json.loads(args.tuning) if args.tuning else None
    tr = lf.Tracker()
    stream = torch.cuda.current_stream()
    packed = tr.pack(batch)
    tune_times = None
    if tuning is None and not args.no_tune:
        # the launch shape from the autotuner (timed candidates on this batch,
        # outside the timed region)
        from paper_2402_14670_gb300.autotune import Autotuner, bucket_of
        tuner = Autotuner(reps=2)
        tuning = tuner.tune(tr, packed, batch, n_ev)
        tune_times = tuner.timings[tuner._key(bucket_of(n_ev, batch.n_tracks))]
    out = tr.find(packed, batch, n_ev, "batched", tuning)
    torch.cuda.synchronize()
    flags = tr.status()
    assert flags == 0, "device status 0x%x" % flags
    n_found = int(out["found"].sum())

    # ---------------- device-resident timed loop (pack + persistent find)
    def step(ev):
        ev[0].record(stream)
        tr.pack(batch, out=packed)
        ev[1].record(stream)
        tr.find(packed, batch, n_ev, "batched", tuning, out=out)
        ev[2].record(stream)

    mk = lambda: [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    for _ in range(args.warmup):
        step(mk())
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.5)
    barrier(ws)
    torch.cuda.synchronize()
    evs = [mk() for _ in range(args.steps)]
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    for i in range(args.steps):
        step(evs[i])
    t_end.record(stream)
    torch.cuda.synchronize()
    barrier(ws)
    clk = clocks.stop()
    total_ms = t_start.elapsed_time(t_end)
    pack_ms = [e[0].elapsed_time(e[1]) for e in evs]
    find_ms = [e[1].elapsed_time(e[2]) for e in evs]
    total_ms = max_over_ranks(ws, total_ms)
    ms_per_step = total_ms / args.steps
    value = ws * n_ev / (ms_per_step / 1e3)

    # ---------------- plain form on the same data: per 1000-event batch (the
    # minimum-bias batch granularity), and in one pass over the whole batch
    plain = None
    if not args.no_plain:
        def timed(fn):
            for _ in range(args.warmup):
                fn()
            torch.cuda.synchronize()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            for _ in range(args.steps):
                fn()
            b.record(stream)
            torch.cuda.synchronize()
            return max_over_ranks(ws, a.elapsed_time(b)) / args.steps

        def whole():
            tr.pack(batch, out=packed)
            tr.find(packed, batch, n_ev, "plain", out=out)
        p1k = timed(per_batch_plain(tr, batch, packed, out, 1000))
        pall = timed(whole)
        plain = {"value": ws * n_ev / (p1k / 1e3), "unit": UNIT, "ms_per_step": p1k,
                 "form": "plain form launched per 1000-event batch (pack + one launch per stage per batch)",
                 "whole_batch": {"value": ws * n_ev / (pall / 1e3), "ms_per_step": pall,
                                 "form": "plain form, one launch per stage over the whole batch"}}
        tr.find(packed, batch, n_ev, "batched", tuning, out=out)
        torch.cuda.synchronize()

    # ---------------- the no-UT variant (Sec. "No-UT tuning") on the same events:
    # pack + persistent find with two window sets per track, q/p unused
    no_ut = None
    if not args.no_no_ut:
        tr_nu = lf.Tracker(None, lf.no_ut_params())
        out_nu = tr_nu.find(packed, batch, n_ev, "batched")
        torch.cuda.synchronize()
        assert tr_nu.status() == 0
        ev_nu = []
        for i in range(args.warmup + args.steps):
            e3 = mk()
            e3[0].record(stream)
            tr_nu.pack(batch, out=packed)
            e3[1].record(stream)
            tr_nu.find(packed, batch, n_ev, "batched", out=out_nu)
            e3[2].record(stream)
            if i >= args.warmup:
                ev_nu.append(e3)
        torch.cuda.synchronize()
        nu_step = max_over_ranks(ws, statistics.mean(e[0].elapsed_time(e[2]) for e in ev_nu))
        nu_find = statistics.mean(e[1].elapsed_time(e[2]) for e in ev_nu)
        nu_found = int(out_nu["found"].sum())
        nu_algo = algorithmic_bytes(n_ev, batch.n_hits, batch.n_tracks, nu_found)
        no_ut = {"value": ws * n_ev / (nu_step / 1e3), "unit": UNIT, "ms_per_step": nu_step, "find_ms": nu_find,
                 "found_tracks": nu_found, "find_hbm_frac": nu_algo / (nu_find / 1e3) / 1e9 / peaks()[0],
                 "form": "no-UT parameters (two one-sided window sets per track, 64-hit cap, 20 triplets), "
                         "batched persistent stage pipeline"}
        tr_nu.close()
        del out_nu

    # ---------------- end to end through lf_process_host on pinned host buffers
    e2e = None
    if not args.no_e2e:
        numa = numa_link()
        # the page-locked host batch on the GPU's nearest NUMA node when the
        # host reports one this process may use
        near = lf.numa_node_cpus().get(numa["gpu_host_numa_node"])
        host, arena = on_node(near, lambda: host_copy(batch))
        hout = tr.alloc_host_output(host.n_tracks)
        for _ in range(args.warmup):
            tr.process_host(host, out=hout, tuning=tuning)
        barrier(ws)
        steps_ms = []
        t0 = time.perf_counter()
        for _ in range(args.steps):
            ta = time.perf_counter()
            tr.process_host(host, out=hout, tuning=tuning)
            steps_ms.append((time.perf_counter() - ta) * 1e3)
        e2e_s = max_over_ranks(ws, time.perf_counter() - t0) / args.steps
        # the host link alone: copies of the x array to the device (the best
        # of two, so that the first touch of the destination is not timed)
        dx = torch.empty(host.x.numel(), dtype=torch.float32, device="cuda")
        h2d_gbps = 0.0
        for _ in range(2):
            torch.cuda.synchronize()
            ta = time.perf_counter()
            dx.copy_(host.x, non_blocking=True)
            torch.cuda.synchronize()
            h2d_gbps = max(h2d_gbps, host.x.numel() * 4 / (time.perf_counter() - ta) / 1e9)
        del dx
        h2d = sum(int(t.numel() * t.element_size()) for t in
                  (host.raw_offsets, host.x, host.z, host.dxdy, host.w, host.plane, host.trk_offsets,
                   host.sx, host.sy, host.stx, host.sty, host.sqop))
        d2h = sum(int(t.numel() * t.element_size()) for t in hout.values())
        e2e = {"value": ws * n_ev / e2e_s, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
               "ms_per_step": 1e3 * e2e_s, "step_ms": steps_ms, "h2d_gbps_x_copy": h2d_gbps,
               "api": "lf_process_host (chunked; copies in, compute and copies out on three streams)"}
        n_hits, n_trk = host.n_hits, host.n_tracks
        cpu_src = host
        e2e["host_memory"] = "cudaHostAlloc (lf_host_alloc)%s" % (
            " on NUMA node %d (nearest to the GPU)" % numa["gpu_host_numa_node"] if near else "")
        e2e["numa_link"] = numa
    else:
        n_hits, n_trk = batch.n_hits, batch.n_tracks
        cpu_src = None

    # ---------------- served stream (the served workload: events of the
    # uneven distribution arriving as a Poisson process at 10 %..120 % of the
    # batched rate; continuous batching over S slots, 16 GB budget).  Stated
    # before measuring: with events arriving in device memory the loop holds
    # p99 <= 5 ms up to 80 % of the batched rate.
    served = None
    if not args.no_serve and e2e is not None:
        from paper_2402_14670_gb300 import serve
        P99_BOUND_MS = 5.0
        # each rank serves its own GPU: offered rates and fractions against
        # this rank's batched rate, not the whole job's
        rate_rank = value / ws

        def sweep_rates(srv, fracs, seed0):
            pts = []
            for frac in fracs:
                rate = frac * rate_rank
                n_pt = int(min(n_ev, max(2000, rate * 0.5)))
                st = srv.run(serve.poisson_arrivals(n_pt, rate, seed=seed0 + int(frac * 1000)))
                pts.append({"offered_frac_of_batched": frac, "offered_rate": rate, "events_per_s": st.events_per_s,
                            "p50_ms": st.p50_ms, "p99_ms": st.p99_ms, "mean_batch_events": st.mean_batch_events,
                            "events": st.n_events})
            return pts

        fracs = (0.1, 0.2, 0.4, 0.6, 0.8, 1.0, 1.2)
        graphs = lambda srv: sum(sl.tr.graph_count() for sl in srv.slots)
        # events arriving in device memory (arrivals written straight to HBM)
        srv = serve.Server(batch, n_slots=4, max_events=2048, budget_bytes=16 << 30)
        srv.tune_buckets((256, 2048))
        g0 = graphs(srv)
        n_sat = min(n_ev, 60000)
        sat_d = srv.run(np.zeros(n_sat))
        pts_d = sweep_rates(srv, fracs, 100)
        at80 = [p for p in pts_d if p["offered_frac_of_batched"] == 0.8][0]
        served = {"p99_bound_ms": P99_BOUND_MS, "bound_load_frac_of_batched": 0.8,
                  "bound_met": bool(at80["p99_ms"] <= P99_BOUND_MS),
                  "slots": len(srv.slots), "slot_events": 2048, "host_fed_slot_events": 1024,
                  "budget_bytes": 16 << 30,
                  "batching": "oldest pending events in arrival order up to the slot's capacity in events, "
                              "hits and tracks; one lf_process_slot graph per slot and launch shape, replayed "
                              "for every batch size",
                  "device_resident": {
                      "saturation_events_per_s": sat_d.events_per_s, "saturation_p50_ms": sat_d.p50_ms,
                      "saturation_p99_ms": sat_d.p99_ms, "saturation_frac_of_batched": sat_d.events_per_s / rate_rank,
                      "points": pts_d, "graphs_captured_before_serving": g0,
                      "graphs_captured_while_serving": graphs(srv) - g0,
                      "note": "events arrive in device memory; each batch's hits are read in place by the pack "
                              "(per-event source offsets), its states gathered; per-track results copied back; "
                              "latency = arrival to results on host"}}
        srv.close()
        # the same load batched by size class, for comparison
        srv = serve.Server(batch, n_slots=4, max_events=2048, budget_bytes=16 << 30, group_by_size=True)
        srv.tune_buckets((256, 2048))
        served["device_resident"]["by_size_class_at_80"] = sweep_rates(srv, (0.8,), 100)[0]
        srv.close()
        # events arriving in page-locked host memory: copied into the device
        # arrival ring in arrival order, batches gathered from it
        srv = serve.Server(host, n_slots=4, max_events=1024, budget_bytes=16 << 30)
        srv.tune_buckets((256, 1024))
        g0 = graphs(srv)
        sat = srv.run(np.zeros(n_sat))
        served["host_fed"] = {
            "saturation_events_per_s": sat.events_per_s, "saturation_p50_ms": sat.p50_ms,
            "saturation_p99_ms": sat.p99_ms, "saturation_frac_of_batched": sat.events_per_s / rate_rank,
            "points": sweep_rates(srv, (0.1, 0.2, 0.3, 0.4, 0.6), 200),
            "ring_bytes": srv.ring.cap_h * serve.RING_BYTES_PER_HIT + srv.ring.cap_t * serve.RING_BYTES_PER_TRACK,
            "graphs_captured_while_serving": graphs(srv) - g0,
            "note": "events arrive in pinned host memory; copied in arrival order into a device arrival ring "
                    "(admission by its free space), batches gathered from it once their events' copies are "
                    "done; per-track results copied back"}
        srv.close()

    # ---------------- roofline of the dominant kernel (persistent find)
    peak, peak_kind = peaks()
    find_avg = statistics.mean(find_ms)
    pack_avg = statistics.mean(pack_ms)
    algo = algorithmic_bytes(n_ev, n_hits, n_trk, n_found)
    achieved = algo / (find_avg / 1e3) / 1e9
    roof = {"kernel": "find pipeline of lf_find_tracks_batched (persistent windows, triplet, extension and "
                      "selection kernels + compaction), one graph launch", "bound": "hbm",
            "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "peak_kind": peak_kind, "traffic": traffic_per_launch(args.config, n_hits), "algorithmic_bytes": algo,
            "launch_ms": find_avg}
    # the find kernels are bound by instruction issue, not by DRAM: their warp
    # instructions (committed ncu count, scaled by input tracks) per second
    # against the issue peak (4 warp instructions per SM per cycle at the
    # median SM clock of the timed region)
    roof_issue = None
    fp = find_profile(args.config)
    if fp is not None and torch.cuda.is_available():
        n_sm = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
        mhz = clk.get("sm_mhz") or clk.get("sm_max_mhz") or 2070.0
        inst = float(fp["warp_instructions_per_launch"]) * n_trk / float(fp["tracks"])
        ach = inst / (find_avg / 1e3)
        pk_issue = n_sm * 4 * mhz * 1e6
        roof_issue = {"kernel": "k_windows + k_triplets + k_extend_block (persistent)", "bound": "issue",
                      "achieved": ach, "peak": pk_issue, "unit": "warp-instructions/s", "frac": ach / pk_issue,
                      "warp_instructions_per_launch": inst,
                      "peak_kind": "%d SMs x 4 schedulers x %.0f MHz (median SM clock, timed region)" % (n_sm, mhz)}
    pk_algo = pack_bytes(n_ev, n_hits)
    roof_pack = {"kernel": "k_pack_event (persistent per-event distribution sort, payload through shared memory)", "bound": "hbm",
                 "achieved": pk_algo / (pack_avg / 1e3) / 1e9, "peak": peak, "unit": "GB/s",
                 "frac": pk_algo / (pack_avg / 1e3) / 1e9 / peak, "launch_ms": pack_avg,
                 "algorithmic_bytes": pk_algo, "traffic": pack_traffic_per_launch(args.config, n_hits)}

    # ---------------- CPU oracle on a bounded sample (rank 0, N = 1)
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu:
        try:
            if cpu_src is None:
                cpu_src = batch.to("cpu")
            n_s = min(args.cpu_events, n_ev)
            sample = cpu_src.select_events(range(n_s))
            threads = len(os.sched_getaffinity(0)) or 1
            dt, _ = time_oracle(sample, threads)
            cpu = {"value": n_s / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
                   "sample": "first %d events of the same batch: pack + find + compact" % n_s}
            n_1 = min(300, n_s)
            dt1, _ = time_oracle(cpu_src.select_events(range(n_1)), 1)
            cpu["single_thread"] = {"value": n_1 / dt1, "unit": UNIT, "cores": 1,
                                    "sample": "first %d events, one thread" % n_1}
        except Exception as e:  # the oracle is test infrastructure; report why it did not run
            cpu = {"value": None, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle", "error": str(e)}

    # pack: one persistent kernel (k_pack_event, which also writes the coarse
    # index of x); find (default queue mode): track->event map, three
    # persistent stage kernels (windows, triplets, extension with the
    # selection), three compaction kernels
    launches_per_step = 1 + (1 + 3) + 3
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "%s (config %d): %d events, %d hits, %d input tracks; %s"
                                   % (cfg.name, args.config, n_ev, n_hits, n_trk, workload_recipe(cfg)),
                       "form": "batched: persistent stage kernels with device work queues, one CUDA graph",
                       "tuning": tuning or "defaults", "tuning_candidates_ms": tune_times,
                       "l2": "inputs larger than L2 (no flush)", "parallelism": "replicas" if ws > 1 else "single"},
            "e2e": e2e, "gpu_launches": launches_per_step * args.steps, "clocks": clk,
            "roofline": roof, "roofline_issue": roof_issue, "roofline_pack": roof_pack, "plain": plain,
            "served": served, "no_ut": no_ut,
            "cpu_baseline": cpu,
            "stage_ms": {"pack": pack_avg, "find": find_avg}, "found_tracks": n_found,
        }
        print(json.dumps(line), flush=True)
    tr.close()
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
