"""Multi-rank logic without GPUs.

1. Ray-range sharding of one trace (the exchange a multi-GPU version would
   use): each shard dedups its own receptions, the shards' keys are merged
   with the same min(dist, ray) rule, and the merge equals the unsharded run
   (the rule is commutative and associative). Run on the FP64 oracle.
2. bench.py's rank reduction (slowest rank's time, summed work) under a
   world-size-2 gloo group on CPU, and the independent Tx per rank.
"""
import os
import socket

import numpy as np
import pytest

import oracle
import scenes


def _merge(key_sets):
    """Per (rx, surface sequence): the smallest (dist, ray) over shards."""
    best = {}
    for keys in key_sets:
        for k in keys:
            key = (int(k["rx"]), int(k["nb"]), tuple(int(x) for x in k["seq"][: k["nb"]]))
            v = (float(k["dist"]), int(k["ray"]))
            if key not in best or v < best[key]:
                best[key] = v
    return best


@pytest.mark.parametrize("shards", [2, 3, 7])
def test_ray_range_shards_merge_to_the_unsharded_result(shards):
    sc = scenes.shoebox(N=50, K=3, n_rx=4)
    R = 10 * sc["N"] ** 2 + 2
    full, _, _ = oracle.trace(sc)
    keys_full, _, _ = oracle.dedup(full)
    bounds = [R * s // shards for s in range(shards + 1)]
    parts = []
    for s in range(shards):
        c, _, _ = oracle.trace(sc, ray_begin=bounds[s], ray_end=bounds[s + 1])
        k, _, _ = oracle.dedup(c)
        parts.append(k)
    merged = _merge(parts)
    ref = _merge([keys_full])
    assert merged == ref
    # and in any shard order
    assert _merge(parts[::-1]) == ref


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t, w = bench.reduce_over_ranks(1.0 + rank, 10.0 * (rank + 1))
    q.put((rank, t, w, bench.CROSSINGS[rank % len(bench.CROSSINGS)]))
    dist.barrier()
    dist.destroy_process_group()


def test_bench_rank_reduction_gloo_world2():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    out.sort()
    # every rank sees the slowest rank's time and the summed work
    assert [(t, w) for _, t, w, _ in out] == [(2.0, 30.0), (2.0, 30.0)]
    # the two ranks trace different Tx positions
    assert out[0][3] != out[1][3]


def test_reduction_without_process_group_is_identity():
    import bench
    assert bench.reduce_over_ranks(3.5, 7.0) == (3.5, 7.0)
