"""The N > 1 path on CPU: events sharded over two gloo ranks.

Events are independent, so a batch shards by events with no exchange on the
data path.  These tests check the partition, that two ranks running the
oracle on their shards and gathering on the host reproduce the whole-batch
results event by event, and that the benchmark's reference arm runs under
torchrun with two ranks (rank 0 alone prints).
"""
import json
import os
import socket
import subprocess
import sys

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
from paper_2402_14670_gb300 import shard, synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def test_partition_covers_every_event_once_and_balances():
    rng = np.random.default_rng(3)
    nh = rng.integers(0, 60000, 997)
    nt = rng.integers(0, 400, 997)
    ro = np.concatenate([[0], np.cumsum(nh)])
    to = np.concatenate([[0], np.cumsum(nt)])
    costs = shard.event_costs(ro, to)
    for world in (1, 2, 3, 8):
        parts = shard.partition(costs, world)
        allev = np.sort(np.concatenate(parts))
        assert np.array_equal(allev, np.arange(997))
        for p in parts:
            assert np.all(np.diff(p) > 0)
        loads = np.array([costs[p].sum() for p in parts])
        # greedy LPT: no rank above the mean by more than the largest event
        assert loads.max() - loads.mean() <= costs.max()


def test_partition_edge_cases():
    # more ranks than events, events without hits or tracks (each factor at least 1), a single event
    ro = np.array([0, 0, 5, 5, 9])
    to = np.array([0, 0, 0, 3, 3])
    costs = shard.event_costs(ro, to)
    assert costs.tolist() == [1, 5, 3, 4]
    parts = shard.partition(costs, 6)
    assert sorted(np.concatenate(parts).tolist()) == [0, 1, 2, 3]
    assert sum(len(p) == 0 for p in parts) == 2
    assert [len(p) for p in shard.partition([7.0], 3)] == [1, 0, 0]
    with pytest.raises(ValueError):
        shard.partition(costs, 0)
    # gather puts results in batch order and refuses a missing event
    parts = shard.partition(costs, 2)
    res = {r: {int(e): ("ev", int(e)) for e in p} for r, p in enumerate(parts)}
    assert shard.gather(res, parts, 4) == [("ev", e) for e in range(4)]
    del res[0][int(parts[0][0])]
    with pytest.raises((ValueError, KeyError)):
        shard.gather(res, parts, 4)


def _event_results(batch_cpu, res):
    """Per event: found flags, hit lists as raw indices inside the event,
    state and Q bits of the found tracks."""
    ro = batch_cpu.raw_offsets.numpy().astype(np.int64)
    to = batch_cpu.trk_offsets.numpy().astype(np.int64)
    perm = res["packed"]["perm"]
    out = []
    for e in range(batch_cpu.n_events):
        a, b = int(to[e]), int(to[e + 1])
        f = res["found"][a:b].astype(bool)
        h = res["hit_idx"][a:b]
        raw = np.where((h >= 0) & f[:, None], perm[np.maximum(h, 0)] - ro[e], -1)
        st = res["state"][a:b][f].view(np.uint32)
        q = res["quality"][a:b][f].view(np.uint32)
        out.append((f.tobytes(), raw.tobytes(), st.tobytes(), q.tobytes()))
    return out


def _rank_main(rank, world, port, n_events):
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=world)
    batch = synth.generate(1, n_events=n_events, truth=False)
    costs = shard.event_costs(batch.raw_offsets.numpy(), batch.trk_offsets.numpy())
    parts = shard.partition(costs, world)
    mine = parts[rank]
    sub = batch.select_events(mine.tolist())
    res = oracle.run_batch(sub, dumps=False)
    local = dict(zip((int(e) for e in mine), _event_results(sub, res)))
    gathered = [None] * world
    dist.all_gather_object(gathered, local)
    if rank == 0:
        merged = shard.gather({r: g for r, g in enumerate(gathered)}, parts, n_events)
        whole = _event_results(batch, oracle.run_batch(batch, dumps=False))
        bad = [e for e in range(n_events) if merged[e] != whole[e]]
        if bad:
            raise AssertionError("events differ between sharded and whole-batch runs: %s" % bad[:10])
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_and_gather():
    mp.spawn(_rank_main, args=(2, _free_port(), 24), nprocs=2, join=True)


def test_bench_reference_arm_under_torchrun_two_ranks():
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()),
           os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0",
           "--config", "1", "--cpu-events", "8"]
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="")
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=600, cwd=ROOT, env=env)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["e2e"]["h2d_bytes_per_step"] == 0
