"""Ray-range split of one trace (the exchange a multi-GPU run makes), on one
GPU through the C ABI: traces of disjoint ray ranges, their deduplicated
records (sbr_trace_entries) concatenated in any order and merged
(sbr_trace_merge) give, after sbr_paths, the path list of the unsharded trace
bit for bit; the shards' ray counts and segments add up to the unsharded ones.
"""
import numpy as np
import pytest

import scenes
from parity import to_numpy

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sbr():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2208_10006_gb300 import build as b
    b.build()
    import paper_2208_10006_gb300 as m
    return m


CASES = {
    "urban_small": (lambda: scenes.config2(N=60, K=3, nx=2, ny=2, sub=3, ground_sub=6, rx_grid=6), 2),
    "shoebox_K5": (lambda: scenes.shoebox(N=61, K=5, sub=3), 3),
    "urban_med": (lambda: scenes.config2(N=150, K=4, nx=3, ny=3, sub=4, ground_sub=8, rx_grid=8), 3),
    "indoor_small": (lambda: scenes.config3(N=40, K=3, F=8), 4),
}


@pytest.mark.parametrize("name", list(CASES))
def test_ray_range_traces_merge_to_the_unsharded_path_list(sbr, name):
    make, parts = CASES[name]
    sc = make()
    d = sbr.scene_to_device(sc)
    N, K = sc["N"], sc["K"]
    R = 10 * N * N + 2
    bvh = sbr.build_bvh(d["tri"], d["surface_id"], d["S"])
    ref_tr = sbr.trace(bvh, d["tx"], d["rx"], N, K)
    ref_st = ref_tr.stats()
    ref_pl = sbr.paths(ref_tr, bvh)
    ref = to_numpy(ref_pl.export())
    ref_g = sbr.path_gains(ref_pl, d["mats"], d["freqs"], d["gamma"], d["disp"], d["pol"]).cpu().numpy()
    # uneven cut points, one of them odd
    rng = np.random.default_rng(parts)
    cuts = np.sort(rng.choice(np.arange(1, R), parts - 1, replace=False))
    bounds = [0] + [int(c) for c in cuts] + [R]
    recs, rays, segs = [], 0, 0
    for b0, b1 in zip(bounds[:-1], bounds[1:]):
        tr = sbr.trace(bvh, d["tx"], d["rx"], N, K, ray_range=(b0, b1))
        st = tr.stats()
        rays += st["rays"]
        segs += st["ray_bounces"]
        keys, vals = tr.entries()
        assert keys.shape[0] == st["keys"]
        recs.append((keys, vals))
    assert rays == R and segs == ref_st["ray_bounces"]
    # the records of the shards in reversed order, each shard's records reversed too
    keys = torch.cat([k.flip(0) for k, _ in recs[::-1]])
    vals = torch.cat([v.flip(0) for _, v in recs[::-1]])
    m = sbr.trace_merge(d["tx"], d["rx"], N, K, keys, vals)
    assert m.stats()["keys"] == ref_st["keys"]
    pl = sbr.paths(m, bvh)
    got = to_numpy(pl.export())
    assert got.keys() == ref.keys()
    for k in ref:
        assert np.array_equal(got[k], ref[k]), k
    g = sbr.path_gains(pl, d["mats"], d["freqs"], d["gamma"], d["disp"], d["pol"]).cpu().numpy()
    assert np.array_equal(g, ref_g)


def test_ray_range_is_checked_on_the_host(sbr):
    sc = scenes.config1(N=9, K=2)
    d = sbr.scene_to_device(sc)
    bvh = sbr.build_bvh(d["tri"], d["surface_id"], d["S"])
    R = 10 * 9 * 9 + 2
    for rr in ((5, 5), (-1, 10), (0, R + 1), (R, 0)):
        with pytest.raises(sbr.SbrError) as e:
            sbr.trace(bvh, d["tx"], d["rx"], 9, 2, ray_range=rr)
        assert e.value.status == 1
    # an empty record list merges to an empty path list
    keys = torch.zeros((0, 10), dtype=torch.int32, device="cuda")
    vals = torch.zeros(0, dtype=torch.int64, device="cuda")
    m = sbr.trace_merge(d["tx"], d["rx"], 9, 2, keys, vals)
    assert sbr.paths(m, bvh).n == 0
