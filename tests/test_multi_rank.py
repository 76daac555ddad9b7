"""Multi-rank logic without GPUs.

1. Ray-range sharding of one trace (the exchange a multi-GPU version would
   use): each shard dedups its own receptions, the shards' keys are merged
   with the same min(dist, ray) rule, and the merge equals the unsharded run
   (the rule is commutative and associative). Run on the FP64 oracle.
2. The exchange of bench.py's ray-range split under a world-size-2 gloo group
   on CPU: each rank packs the records of its oracle shard in the layout of
   sbr_trace_entries, all-gathers them (bench.gather_records) and merges
   them; every rank then holds the records of the unsharded run.
3. bench.py's rank reduction (slowest rank's time, summed work) and the
   ray-range split of the launch grid.
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


def _pack(keys):
    """Oracle dedup records in the layout of sbr_trace_entries: keys [n, 10]
    (rx, reflections, 8 surface ids, -1 padded), vals = FP32 distance bits
    << 32 | ray id (non-negative, so ordered as the (dist, ray) pairs)."""
    n = len(keys)
    k = np.full((n, 10), -1, np.int32)
    k[:, 0] = keys["rx"]
    k[:, 1] = keys["nb"]
    for i in range(n):
        m = int(keys["nb"][i])
        k[i, 2:2 + m] = keys["seq"][i][:m]
    bits = np.asarray(keys["dist"], np.float32).view(np.uint32).astype(np.int64)
    v = (bits << 32) | np.asarray(keys["ray"], np.int64)
    return k, v


def _merge_packed(k, v):
    best = {}
    for row, val in zip(k, v):
        key = tuple(int(x) for x in row)
        if key not in best or val < best[key]:
            best[key] = int(val)
    return best


SPLIT_SCENE = dict(N=50, K=3, n_rx=4)


def _worker(rank, world, port, q):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t, w = bench.reduce_over_ranks(1.0 + rank, 10.0 * (rank + 1))
    sc = scenes.shoebox(**SPLIT_SCENE)
    R = 10 * sc["N"] ** 2 + 2
    b0, b1 = bench.ray_range(R, rank, world)
    c, _, _ = oracle.trace(sc, ray_begin=b0, ray_end=b1)
    keys, _, _ = oracle.dedup(c)
    k, v = _pack(keys)
    K, V = bench.gather_records(torch.as_tensor(k), torch.as_tensor(v))
    q.put((rank, t, w, (b0, b1), _merge_packed(K.numpy(), V.numpy())))
    dist.barrier()
    dist.destroy_process_group()


def test_split_exchange_and_rank_reduction_gloo_world2():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=300) for _ in procs]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    out.sort(key=lambda x: x[0])
    # every rank sees the slowest rank's time and the summed work
    assert [(t, w) for _, t, w, _, _ in out] == [(2.0, 30.0), (2.0, 30.0)]
    # the two ranks trace complementary id ranges of the grid
    sc = scenes.shoebox(**SPLIT_SCENE)
    R = 10 * sc["N"] ** 2 + 2
    assert out[0][3] == (0, R // 2) and out[1][3] == (R // 2, R)
    # after the all-gather and the merge both ranks hold the unsharded records
    full, _, _ = oracle.trace(sc)
    keys_full, _, _ = oracle.dedup(full)
    ref = _merge_packed(*_pack(keys_full))
    assert len(ref) > 10
    assert out[0][4] == ref and out[1][4] == ref


def test_ray_ranges_tile_the_grid():
    import bench
    for R, world in ((10002, 2), (10002, 3), (1002, 8), (42, 8)):
        rs = [bench.ray_range(R, r, world) for r in range(world)]
        assert rs[0][0] == 0 and rs[-1][1] == R
        assert all(a[1] == b[0] for a, b in zip(rs, rs[1:]))
        assert max(b - a for a, b in rs) - min(b - a for a, b in rs) <= 1


def test_reduction_without_process_group_is_identity():
    import bench
    assert bench.reduce_over_ranks(3.5, 7.0) == (3.5, 7.0)
