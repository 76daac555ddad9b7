"""Batched jobs (sbr_batch_*) through the C ABI: per job the same paths, gains
and H as the per-pair calls (sbr_trace, sbr_paths, sbr_path_gains,
sbr_synthesize_H) on the same inputs, and the FP64 oracle's path set.

The workload is the batched uneven one at test sizes: 3 scenes of 0.3k-3k
triangles, 24 jobs with N in {12, ..., 40} (1,442 - 16,002 rays), K 1-4,
F 4-32, up to 8 x 8 transmit and 16 receive elements: several waves when the
ray-queue capacity is small, ragged tensor-core tiles.
"""
import numpy as np
import pytest

import oracle
import scenes
from parity import assert_parity, compare_paths, to_numpy

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


def _workload(sbr, n_jobs=24, seed=7):
    scs = [scenes.batch_scene(s, t_min=300, t_max=3000) for s in range(3)]
    jobs = scenes.batch_jobs(scs, n_jobs=n_jobs, seed=seed, n_values=[12, 17, 23, 31, 40], k_range=(1, 4),
                             f_exp_range=(2, 5), max_elem_exp=4)
    dev = torch.device("cuda")
    sdev = []
    for sc in scs:
        tri = torch.as_tensor(sc["tri"].reshape(-1, 9), dtype=torch.float32, device=dev)
        sid = torch.as_tensor(sc["surface_id"], dtype=torch.int32, device=dev)
        mats = torch.as_tensor(sc["materials"], dtype=torch.float64, device=dev)
        sdev.append((sbr.build_bvh(tri, sid, len(sc["materials"])), mats))
    t = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device=dev)
    jdev = [dict(scene=j["scene"], N=j["N"], K=j["K"], tx=j["tx"], rx=j["rx"], pol=j["pol"],
                 freqs=t(j["freqs"], torch.float64), gamma=t(j["gamma"], torch.float32),
                 tx_elem=t(j["tx_elem"], torch.float64), rx_elem=t(j["rx_elem"], torch.float64))
            for j in jobs]
    return scs, jobs, sdev, jdev


def _per_pair(sbr, sdev, j, precision):
    bvh, mats = sdev[j["scene"]]
    rx = torch.as_tensor(np.asarray(j["rx"], dtype=np.float64).reshape(1, 3), device="cuda")
    tr = sbr.trace(bvh, j["tx"], rx, j["N"], j["K"])
    pl = sbr.paths(tr, bvh)
    pol = sbr.POL_V if j["pol"] == "V" else sbr.POL_H
    g = sbr.path_gains(pl, mats, j["freqs"], j["gamma"], None, pol)
    H = sbr.synthesize_H(pl, g, j["freqs"], j["tx_elem"], j["rx_elem"], 0, precision)
    return pl, to_numpy(pl.export()), g.cpu().numpy(), H.cpu().numpy()


@pytest.mark.parametrize("cfg", [dict(tile_n=64, wave_rays=40000), dict(tile_n=128),
                                 dict(tile_n=256, use_graph=0, breadth_first=1),
                                 dict(tile_n=64, wave_rays=40000, breadth_first=1)])
def test_batch_equals_per_pair_calls(sbr, cfg):
    scs, jobs, sdev, jdev = _workload(sbr)
    b = sbr.batch_create(sdev, jdev, config=dict(path_cap=256, **cfg))
    b.run()
    n_paths, status, info = b.query()
    assert (status == 0).all(), status
    assert info["n_jobs"] == len(jobs)
    if "wave_rays" in cfg:
        assert info["n_waves"] > 1
    assert info["rays"] == sum(10 * j["N"] ** 2 + 2 for j in jobs)
    rb = 0
    for i, j in enumerate(jdev):
        pl, ex, g, H = _per_pair(sbr, sdev, j, sbr.SYNTH_FP16X3)
        assert n_paths[i] == pl.n, (i, n_paths[i], pl.n)
        bx = {k: v.cpu().numpy() for k, v in b.export(i, int(n_paths[i])).items()}
        for k in ("nb", "seq", "face", "pts", "L", "aod", "aoa", "dist"):
            assert np.array_equal(bx[k], ex[k]), (i, k)
        assert np.array_equal(bx["ray"].astype(np.int64) & 0xffffffff, ex["ray"]), i
        assert np.array_equal(bx["g"], g.reshape(bx["g"].shape)), i
        Hb = j["H"].cpu().numpy()
        # the same path list, weights and tensor-core arithmetic: bit-identical H
        assert np.array_equal(Hb, H), (i, np.abs(Hb - H).max())
        rb += pl.n
    assert info["paths"] == rb


def test_batch_matches_oracle(sbr):
    scs, jobs, sdev, jdev = _workload(sbr, n_jobs=8, seed=11)
    b = sbr.batch_create(sdev, jdev, config=dict(path_cap=256))
    b.run()
    n_paths, status, _ = b.query()
    assert (status == 0).all()
    for i, j in enumerate(jobs):
        sc = scenes.batch_job_scene(scs[j["scene"]], j)
        orc = oracle.run(sc)
        bx = {k: v.cpu().numpy() for k, v in b.export(i, int(n_paths[i])).items()}
        gpu = dict(rx=np.zeros(len(bx["nb"]), np.int32), nb=bx["nb"], seq=bx["seq"], face=bx["face"],
                   pts=bx["pts"], L=bx["L"], aod=bx["aod"], aoa=bx["aoa"],
                   ray=bx["ray"].astype(np.int64) & 0xffffffff)
        rep = compare_paths(gpu, bx["g"], orc)
        assert_parity(rep)
        assert rep["exempt"] <= max(2, 0.05 * rep["n_orc"]), rep


def test_batch_graph_replay_is_deterministic(sbr):
    scs, jobs, sdev, jdev = _workload(sbr, n_jobs=12, seed=5)
    b = sbr.batch_create(sdev, jdev, config=dict(path_cap=256, tile_n=128))
    c0 = sbr.launch_count()
    b.run()
    n1, _, info = b.query()
    assert info["graph_kernels"] > 0
    assert sbr.launch_count() - c0 == info["graph_kernels"]
    H1 = [j["H"].clone() for j in jdev]
    for j in jdev:
        j["H"].zero_()
    b.run()
    n2, _, _ = b.query()
    assert np.array_equal(n1, n2)
    for a, j in zip(H1, jdev):
        assert torch.equal(a, j["H"])


def test_batch_reports_a_full_path_store(sbr):
    scs, jobs, sdev, jdev = _workload(sbr, n_jobs=6, seed=3)
    b = sbr.batch_create(sdev, jdev, config=dict(path_cap=2))
    b.run()
    n_paths, status, info = b.query()
    assert info["max_keys"] > 2
    assert (status == 3).any()          # SBR_ERR_CAPACITY on the jobs with more keys
    assert (n_paths <= 2).all()


def test_batch_rejects_bad_jobs(sbr):
    scs, jobs, sdev, jdev = _workload(sbr, n_jobs=2, seed=3)
    bad = [dict(jdev[0], N=5000), dict(jdev[0], scene=7), dict(jdev[0], K=9)]
    for j in bad:
        with pytest.raises(sbr.SbrError) as e:
            sbr.batch_create(sdev, [j])
        assert e.value.status == 1
    with pytest.raises(sbr.SbrError):
        sbr.batch_create(sdev, jdev, config=dict(tile_n=96))


def test_autotuner_returns_a_working_config(sbr):
    scs, jobs, sdev, jdev = _workload(sbr, n_jobs=6, seed=9)
    cfg, ms = sbr.batch_tune(sdev, jdev)
    assert ms > 0
    assert cfg["tile_n"] in (64, 128, 256) and 1 <= cfg["trace_blocks_per_sm"] <= 16
    assert cfg["path_cap"] >= 64 and cfg["wave_rays"] > 0
    b = sbr.batch_create(sdev, jdev, config=cfg)
    b.run()
    _, status, _ = b.query()
    assert (status == 0).all()


def test_batch_with_64x64_upa_matches_per_pair(sbr):
    # the top of the array range read as a 64 x 64 Tx UPA (4096 elements): jobs
    # with square UPAs up to 64 x 64 through the batch (tile width 64: 64 N tiles
    # per frequency) give the per-pair H bit for bit
    scs = [scenes.batch_scene(s, t_min=300, t_max=3000) for s in range(2)]
    jobs = scenes.batch_jobs(scs, n_jobs=6, seed=11, n_values=[12, 17], k_range=(1, 3), f_exp_range=(2, 3),
                             max_elem_exp=3, tx_exp_range=(4, 6), square_tx=True)
    jobs[0]["tx_elem"] = scenes.upa_yz(jobs[0]["tx"], 64, 64, 299792458.0 / float(np.mean(jobs[0]["freqs"])) / 2)
    dev = torch.device("cuda")
    sdev = []
    for sc in scs:
        tri = torch.as_tensor(sc["tri"].reshape(-1, 9), dtype=torch.float32, device=dev)
        sid = torch.as_tensor(sc["surface_id"], dtype=torch.int32, device=dev)
        mats = torch.as_tensor(sc["materials"], dtype=torch.float64, device=dev)
        sdev.append((sbr.build_bvh(tri, sid, len(sc["materials"])), mats))
    t = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device=dev)
    jdev = [dict(scene=j["scene"], N=j["N"], K=j["K"], tx=j["tx"], rx=j["rx"], pol=j["pol"],
                 freqs=t(j["freqs"], torch.float64), gamma=t(j["gamma"], torch.float32),
                 tx_elem=t(j["tx_elem"], torch.float64), rx_elem=t(j["rx_elem"], torch.float64))
            for j in jobs]
    assert len(jobs[0]["tx_elem"]) == 4096 and all(len(j["tx_elem"]) >= 256 for j in jobs)
    b = sbr.batch_create(sdev, jdev, config=dict(path_cap=256, tile_n=64))
    b.run()
    n_paths, status, info = b.query()
    assert (status == 0).all()
    for i, j in enumerate(jdev):
        _, ex, g, H = _per_pair(sbr, sdev, j, sbr.SYNTH_FP16X3)
        assert len(ex["rx"]) == n_paths[i]
        Hb = j["H"].cpu().numpy()
        assert Hb.shape == H.shape
        assert np.array_equal(Hb, H), (i, np.abs(Hb - H).max())
