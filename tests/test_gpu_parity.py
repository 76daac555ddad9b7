"""CUDA path vs FP64 oracle, element by element, through the C ABI.

Sizes are chosen so the oracle finishes in seconds while the scenes span
many BVH levels, several bounces and ragged tails (ray counts that are not
multiples of the warp or block size). Tolerances: path sets exact (edge-
ambiguous exemptions counted), faces exact, L 1e-9 relative, gains 1e-4
relative, PDP taps 0.01 dB.
"""
import numpy as np
import pytest

import oracle
import scenes
from parity import assert_parity, compare_paths, to_numpy

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

C0 = 299792458.0


@pytest.fixture(scope="module")
def sbr():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2208_10006_gb300 import build as b
    b.build()
    import paper_2208_10006_gb300 as m
    return m


SCENES = {
    "config1": lambda: scenes.config1(),
    "config1_N37_K3": lambda: scenes.config1(N=37, K=3),
    "corner": lambda: scenes.corner_reflector(),
    "two_ray_H": lambda: scenes.two_ray(pol="H", N=97),
    "shoebox": lambda: scenes.shoebox(),
    "shoebox_K5": lambda: scenes.shoebox(N=61, K=5, sub=3),
    "urban_small": lambda: scenes.config2(N=60, K=3, nx=2, ny=2, sub=3, ground_sub=6, rx_grid=6),
    "urban_med": lambda: scenes.config2(N=150, K=4, nx=3, ny=3, sub=4, ground_sub=8, rx_grid=8),
    "indoor_small": lambda: scenes.config3(N=40, K=3, F=8),
    "indoor_small_dispersive": lambda: dict(scenes.config3(N=40, K=3, F=8),
                                            disp_deg_km=np.linspace(-50.0, 80.0, 8).astype(np.float32)),
}


@pytest.mark.parametrize("N", [1, 2, 7, 50, 101])
def test_launch_dirs_and_alpha(sbr, N):
    d, a = sbr.launch_dirs(N)
    ref = oracle.geodesic_dirs(N)
    dd = d.cpu().numpy()
    assert dd.shape == ref.shape
    assert np.abs(dd - ref).max() < 4e-16
    assert abs(float(a.cpu()[0]) - oracle.alpha(N)) <= 1e-14 * oracle.alpha(N)


@pytest.mark.parametrize("N", [1, 2, 3, 7, 50, 101, 1000])
def test_directions_decoded_in_the_trace_kernels(sbr, N, monkeypatch):
    # the double-float directions the trace kernels decode from the ray id
    # (exact integer lattice point, normalised in double-float) against the
    # oracle's FP64 directions, every ray: unit vectors within 1e-13 (the
    # double-float ray state carries ~2^-48)
    monkeypatch.setenv("SBR_DIRS_DF", "1")
    d, _ = sbr.launch_dirs(N, with_alpha=False)
    monkeypatch.delenv("SBR_DIRS_DF")
    ref = oracle.geodesic_dirs(N)
    dd = d.cpu().numpy()
    assert dd.shape == ref.shape == (10 * N * N + 2, 3)
    err = np.abs(dd - ref).max()
    print("N", N, "double-float directions: max |d - d_oracle| =", err)
    assert err < 1e-13


@pytest.mark.parametrize("N", [1, 2, 5, 37, 100, 632, 1000])
def test_trace_alpha_matches_oracle(sbr, N):
    # the reception-sphere angle a trace computes when given none (one face of
    # the lattice, double-float chords) against the oracle's FP64 maximum over
    # all 20 faces
    d = sbr.scene_to_device(scenes.config1(N=N, K=0))
    bvh = sbr.build_bvh(d["tri"], d["surface_id"], d["S"])
    a = sbr.trace(bvh, d["tx"], d["rx"], N, 0).stats()["alpha"]
    ref = oracle.alpha(N)
    print("N", N, "alpha", a, "oracle", ref, "rel", abs(a - ref) / ref)
    assert abs(a - ref) <= 1e-13 * ref


@pytest.mark.parametrize("name", list(SCENES))
def test_paths_and_gains_match_oracle(sbr, name):
    sc = SCENES[name]()
    r = sbr.run_scene(sc)
    ex = to_numpy(r["export"])
    g = r["g"].cpu().numpy()
    orc = oracle.run(sc)
    rep = compare_paths(ex, g, orc)
    print(name, {k: v for k, v in rep.items() if k not in ("only_gpu", "only_orc")},
          "gpu stats", r["stats"])
    assert_parity(rep)
    assert rep["n_common"] >= 1
    # exemptions are rare: at most a few percent of the keys
    assert rep["exempt"] <= max(2, 0.05 * rep["n_orc"]), rep
    st = r["stats"]
    assert st["ray_bounces"] == orc["counters"]["segments"]
    assert st["rays"] == 10 * sc["N"] ** 2 + 2
    info = r["paths"].info()
    assert info["n_paths"] == len(ex["rx"])


@pytest.mark.parametrize("name", ["config1", "urban_med", "indoor_small"])
def test_pdp_and_stats_match_oracle(sbr, name):
    sc = SCENES[name]()
    r = sbr.run_scene(sc)
    ex = to_numpy(r["export"])
    orc = oracle.run(sc)
    rep = compare_paths(ex, r["g"].cpu().numpy(), orc)
    assert_parity(rep)
    # a receiver that has an edge-ambiguous (exempted) key on one side only has
    # different per-receiver sums by construction: the taps and statistics are
    # compared on every other receiver, and those must be nearly all of them
    n_rx = len(sc["rx"])
    odd = {k[0] for k in rep["only_gpu"]} | {k[0] for k in rep["only_orc"]}
    keep = np.array([q not in odd for q in range(n_rx)])
    assert keep.sum() >= max(1, n_rx - max(1, n_rx // 20)), (keep.sum(), n_rx)
    print(name, "PDP compared on", int(keep.sum()), "of", n_rx, "receivers")
    fc = float(sc["freqs"][len(sc["freqs"]) // 2])
    fi = len(sc["freqs"]) // 2
    n_bins = 2048
    pdp, st = sbr.pdp_angles(r["paths"], r["g"], fi, fc, 1e-9, n_bins)
    pdp, st = pdp.cpu().numpy()[keep], st.cpu().numpy()[keep]
    opdp, ost = oracle.pdp_stats(orc["paths"], orc["g"], fi, fc, 1e-9, n_bins, n_rx)
    opdp, ost = opdp[keep], ost[keep]
    assert np.isfinite(ost[:, 1]).sum() >= 1
    empty = np.isneginf(opdp)
    assert np.array_equal(empty, np.isneginf(pdp))
    assert np.abs(pdp[~empty] - opdp[~empty]).max(initial=0) < 0.01
    has = np.isfinite(ost[:, 1])
    assert np.array_equal(has, np.isfinite(st[:, 1]))
    assert np.abs(st[has, :2] - ost[has, :2]).max(initial=0) < 0.01          # dB
    assert np.abs(st[has, 2] - ost[has, 2]).max(initial=0) < 1e-4 * max(ost[has, 2].max(initial=0), 1e-12)
    assert np.abs(st[has, 3:] - ost[has, 3:]).max(initial=0) < 1e-4          # degrees


def test_calls_on_user_streams_give_the_same_paths(sbr):
    # build and trace on one user stream, the path list and gains on another (the
    # path list call then waits on the host for the trace): the same path list
    # and gains as on the current stream
    sc = SCENES["urban_small"]()
    ref = sbr.run_scene(sc)
    d = sbr.scene_to_device(sc)
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    s1.wait_stream(torch.cuda.current_stream())
    bvh = sbr.build_bvh(d["tri"], d["surface_id"], d["S"], stream=s1)
    tr = sbr.trace(bvh, d["tx"], d["rx"], sc["N"], sc["K"], stream=s1)
    s2.wait_stream(torch.cuda.current_stream())
    pl = sbr.paths(tr, bvh, stream=s2)
    g = sbr.path_gains(pl, d["mats"], d["freqs"], d["gamma"], d["disp"], d["pol"], stream=s2)
    ex = pl.export(stream=s2)
    s2.synchronize()
    assert tr.stats()["ray_bounces"] == ref["stats"]["ray_bounces"]
    a, b = to_numpy(ref["export"]), to_numpy(ex)
    for k in a:
        assert np.array_equal(a[k], b[k]), k
    assert np.array_equal(ref["g"].cpu().numpy(), g.cpu().numpy())


def _capture(fn):
    # one CUDA graph of fn's launches on a side stream (warmed up there first)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        fn()
    torch.cuda.current_stream().wait_stream(s)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        fn()
    return graph


def test_gains_and_pdp_replay_in_a_cuda_graph(sbr):
    # the asynchronous calls (kernels launched as programmatic dependents)
    # captured into a CUDA graph and replayed: bit-identical to the eager calls
    sc = SCENES["indoor_small"]()
    r = sbr.run_scene(sc)
    d, pl = r["dev"], r["paths"]
    fc = float(sc["freqs"][0])
    g_ref = sbr.path_gains(pl, d["mats"], d["freqs"], d["gamma"], d["disp"], d["pol"])
    pdp_ref, st_ref = sbr.pdp_angles(pl, g_ref, 0, fc, 1e-9, 256)
    torch.cuda.synchronize()
    g, pdp, st = torch.empty_like(g_ref), torch.empty_like(pdp_ref), torch.empty_like(st_ref)

    def fn():
        sbr.path_gains(pl, d["mats"], d["freqs"], d["gamma"], d["disp"], d["pol"], out=g)
        sbr.pdp_angles(pl, g, 0, fc, 1e-9, 256, out=(pdp, st))

    graph = _capture(fn)
    for t in (g, pdp, st):
        t.zero_()
    for _ in range(2):
        graph.replay()
    torch.cuda.synchronize()
    assert np.array_equal(g.cpu().numpy(), g_ref.cpu().numpy())
    assert np.array_equal(pdp.cpu().numpy(), pdp_ref.cpu().numpy())
    assert np.array_equal(st.cpu().numpy(), st_ref.cpu().numpy(), equal_nan=True)


def test_synthesis_replays_in_a_cuda_graph(sbr):
    # the tensor-core synthesis (operand prologue, then the kernel as its
    # programmatic dependent, operands from the stream-ordered pool) captured
    # into a CUDA graph and replayed: bit-identical to the eager call
    sc = SCENES["indoor_small"]()
    r = sbr.run_scene(sc)
    d, pl = r["dev"], r["paths"]
    H_ref = sbr.synthesize_H(pl, r["g"], d["freqs"], d["tx_elem"], d["rx_elem"], 0, sbr.SYNTH_FP16X3)
    torch.cuda.synchronize()
    H = torch.empty_like(H_ref)
    graph = _capture(lambda: sbr.synthesize_H(pl, r["g"], d["freqs"], d["tx_elem"], d["rx_elem"], 0,
                                              sbr.SYNTH_FP16X3, out=H))
    H.zero_()
    for _ in range(2):
        graph.replay()
    torch.cuda.synchronize()
    assert np.array_equal(H.cpu().numpy(), H_ref.cpu().numpy())


def test_foreign_kernels_between_calls_keep_stream_order(sbr):
    # the library's kernels wait for their predecessor on the stream before
    # their first memory access, whoever launched it: gains scaled in place by
    # a torch kernel between path_gains and pdp_angles raise every PDP tap by
    # exactly 20 log10(2) dB and leave the delay statistics unchanged
    sc = SCENES["urban_med"]()
    r = sbr.run_scene(sc)
    pl, fc = r["paths"], float(sc["freqs"][0])
    pdp0, st0 = sbr.pdp_angles(pl, r["g"], 0, fc, 1e-9, 512)
    g = r["g"].clone()
    for _ in range(3):
        g.mul_(2.0)
        pdp, st = sbr.pdp_angles(pl, g, 0, fc, 1e-9, 512)
        g.mul_(0.5)
    torch.cuda.synchronize()
    a, b = pdp0.cpu().numpy(), pdp.cpu().numpy()
    fin = np.isfinite(a)
    assert fin.any() and np.array_equal(fin, np.isfinite(b))
    assert np.abs(b[fin] - a[fin] - 20.0 * np.log10(2.0)).max() < 1e-4
    s0, s1 = st0.cpu().numpy(), st.cpu().numpy()
    ok = np.isfinite(s0[:, 2])
    assert np.allclose(s1[ok, 2], s0[ok, 2], rtol=1e-12, atol=0.0)   # rms delay spread: scale-free


def test_pdp_into_pinned_host_memory_equals_device_output(sbr):
    # the PDP kernel writes straight into pinned host tensors: bit-identical to
    # its device output
    sc = SCENES["urban_med"]()
    r = sbr.run_scene(sc)
    n_rx, n_bins = r["paths"].n_rx, 512
    pdp_d, st_d = sbr.pdp_angles(r["paths"], r["g"], 0, float(sc["freqs"][0]), 1e-9, n_bins)
    out = (torch.full((max(n_rx, 1), n_bins), 7.0, dtype=torch.float32, pin_memory=True),
           torch.full((max(n_rx, 1), sbr.NSTATS), 7.0, dtype=torch.float64, pin_memory=True))
    pdp_h, st_h = sbr.pdp_angles(r["paths"], r["g"], 0, float(sc["freqs"][0]), 1e-9, n_bins, out=out)
    torch.cuda.synchronize()
    assert not pdp_h.is_cuda and pdp_h.data_ptr() == out[0].data_ptr()
    assert np.array_equal(pdp_h.numpy(), pdp_d.cpu().numpy())
    assert np.array_equal(st_h.numpy(), st_d.cpu().numpy(), equal_nan=True)
    with pytest.raises(ValueError):
        sbr.pdp_angles(r["paths"], r["g"], 0, 1e9, 1e-9, n_bins + 1, out=out)


@pytest.mark.parametrize("precision,tol", [(0, 1e-9), (1, 2e-5)])
def test_synthesis_matches_oracle(sbr, precision, tol):
    sc = scenes.config3(N=40, K=3, F=12)
    r = sbr.run_scene(sc)
    ex = to_numpy(r["export"])
    d = r["dev"]
    H = sbr.synthesize_H(r["paths"], r["g"], d["freqs"], d["tx_elem"], d["rx_elem"], 0,
                         precision).cpu().numpy()
    # the oracle synthesises from the GPU's own path list, so this isolates Eq. 13-14
    paths = dict(rx=ex["rx"], nb=ex["nb"], pts=ex["pts"], L=ex["L"])
    g_ref = oracle.gains(sc, dict(rx=ex["rx"], nb=ex["nb"], seq=ex["seq"], pts=ex["pts"], L=ex["L"]))
    Ho = oracle.synth_H(paths, g_ref, sc["freqs"], sc["tx"], sc["rx"][0], sc["tx_elem"], sc["rx_elem"])
    err = np.abs(H - Ho).max() / np.abs(Ho).max()
    print("synthesis precision", precision, "max|dH|/max|H| =", err)
    # gains are FP32 on the GPU (1e-6 relative), which bounds the FP64 form too
    assert err < max(tol, 5e-6 if precision == 0 else tol)


def test_synthesis_los_and_empty_receivers(sbr):
    # free space: a single LoS path, spherical-wave response across the arrays
    sc = dict(name="free", tri=np.zeros((0, 3, 3), np.float32), surface_id=np.zeros(0, np.int32),
              materials=np.zeros((0, 3)), tx=np.array([0.0, 0.0, 1.0]),
              rx=np.array([[3.0, 0.5, 1.2], [50.0, 0.0, 0.0]]), rx_valid=np.ones(2, bool),
              freqs=np.array([27e9, 28e9, 29e9]), gamma_db_km=np.zeros(3, np.float32),
              disp_deg_km=np.zeros(3, np.float32), N=30, K=1, pol="V",
              tx_elem=scenes.upa_yz([0.0, 0.0, 1.0], 4, 4, 0.05),
              rx_elem=scenes.ula_y([3.0, 0.5, 1.2], 6, 0.05))
    r = sbr.run_scene(sc)
    ex = to_numpy(r["export"])
    assert ex["nb"].tolist() == [0, 0]
    d = r["dev"]
    for prec, tol in ((0, 1e-6), (1, 1e-5)):
        H = sbr.synthesize_H(r["paths"], r["g"], d["freqs"], d["tx_elem"], d["rx_elem"], 0, prec)
        H = H.cpu().numpy()
        d0 = np.linalg.norm(sc["tx"] - sc["rx"][0])
        dist = np.linalg.norm(sc["rx_elem"][:, None, :] - sc["tx_elem"][None, :, :], axis=2)
        f = sc["freqs"]
        ref = (C0 / (4 * np.pi * f * d0))[:, None, None] * np.exp(-2j * np.pi * f[:, None, None] * dist / C0)
        assert np.abs(H - ref).max() < tol * np.abs(ref).max()


def test_capacity_matches_oracle(sbr):
    rng = np.random.default_rng(0)
    # both Gram orientations, square, the 64 limit, and single-antenna ends (SISO, SIMO, MISO)
    for (F, Nr, Nt) in ((5, 4, 7), (3, 9, 5), (4, 64, 256), (2, 64, 64), (3, 1, 1), (2, 1, 16), (2, 16, 1)):
        H = (rng.normal(size=(F, Nr, Nt)) + 1j * rng.normal(size=(F, Nr, Nt))).astype(np.complex64)
        Ht = torch.as_tensor(H, device="cuda")
        snr = np.arange(0.0, 31.0, 5.0)
        C = sbr.capacity(Ht, snr).cpu().numpy()
        Co = oracle.capacity(H.astype(np.complex128), snr)
        assert np.abs(C - Co).max() < 1e-5 * np.abs(Co).max(), (F, Nr, Nt, C, Co)


def test_edge_cases(sbr):
    # K = 0: only the LoS path survives dedup and refinement
    r = sbr.run_scene(scenes.config1(N=23, K=0))
    assert to_numpy(r["export"])["nb"].tolist() == [0]
    # empty scene: LoS to every receiver, no reflections
    sc = scenes.config1(N=11, K=3)
    sc["tri"] = np.zeros((0, 3, 3), np.float32)
    sc["surface_id"] = np.zeros(0, np.int32)
    r = sbr.run_scene(sc)
    assert to_numpy(r["export"])["nb"].tolist() == [0]
    # single-triangle scene (one-leaf BVH)
    sc = scenes.two_ray(N=64)
    sc["tri"], sc["surface_id"] = sc["tri"][:1], sc["surface_id"][:1]
    r = sbr.run_scene(sc)
    orc = oracle.run(sc)
    assert_parity(compare_paths(to_numpy(r["export"]), r["g"].cpu().numpy(), orc))
    # receivers: none
    d = sbr.scene_to_device(scenes.config1(N=9, K=2))
    bvh = sbr.build_bvh(d["tri"], d["surface_id"], d["S"])
    tr = sbr.trace(bvh, d["tx"], None, 9, 2)
    pl = sbr.paths(tr, bvh)
    assert pl.n == 0
    # vanishing reception sphere
    tr = sbr.trace(bvh, d["tx"], d["rx"], 9, 2, alpha=1e-12)
    assert sbr.paths(tr, bvh).n == 0
    # invalid arguments are rejected on the host
    with pytest.raises(sbr.SbrError) as e:
        sbr.trace(bvh, d["tx"], d["rx"], 9, 9)
    assert e.value.status == 1
    with pytest.raises(sbr.SbrError):
        sbr.trace(bvh, [float("nan"), 0, 0], d["rx"], 9, 2)
    # a dedup table too small reports SBR_ERR_CAPACITY instead of corrupting memory
    sc = scenes.shoebox(N=40, K=3, n_rx=8)
    d = sbr.scene_to_device(sc)
    bvh = sbr.build_bvh(d["tri"], d["surface_id"], d["S"])
    tr = sbr.trace(bvh, d["tx"], d["rx"], 40, 3, table_log2=4)
    st = tr.stats(check=False)
    assert st["status"] == 3
    with pytest.raises(sbr.SbrError) as e:
        sbr.paths(tr, bvh)
    assert e.value.status == 3


def test_bvh_shape(sbr):
    for sc in (scenes.config1(), scenes.config2(N=10, K=1), scenes.config3(N=10, K=1, F=2)):
        d = sbr.scene_to_device(sc)
        info = sbr.build_bvh(d["tri"], d["surface_id"], d["S"]).info()
        T = len(sc["tri"])
        # two-child nodes over leaves of up to two triangles: at most T-1 nodes
        assert info["T"] == T and 1 <= info["n_nodes"] <= max(1, T - 1)
        assert 1 <= info["depth"] <= 64


@pytest.mark.parametrize("name", ["config1_N37_K3", "shoebox_K5", "urban_small"])
def test_schedules_give_identical_paths(sbr, name):
    # breadth first, depth first from a middle bounce and depth first throughout:
    # the same segments are traced, so the path lists agree exactly
    sc = SCENES[name]()
    d = sbr.scene_to_device(sc)
    bvh = sbr.build_bvh(d["tri"], d["surface_id"], d["S"])
    outs = []
    for df in (sc["K"] + 1, 2, 0):
        tr = sbr.trace(bvh, d["tx"], d["rx"], sc["N"], sc["K"], depth_first_from=df)
        st = tr.stats()
        ex = to_numpy(sbr.paths(tr, bvh).export())
        outs.append((st["ray_bounces"], st["candidates"], st["keys"], st["queue"], ex))
    for o in outs[1:]:
        assert o[:4] == outs[0][:4]
        for k in ("rx", "nb", "seq", "face", "L", "pts", "ray", "dist"):
            assert np.array_equal(o[4][k], outs[0][4][k]), k


@pytest.mark.parametrize("N", [20, 33])
def test_near_edge_hits_are_counted(sbr, N):
    # rays with d_x == 0 that go up hit the ceiling on its shared edge; the
    # instrumented trace counts them, and so does the oracle's edge flag
    sc = scenes.edge_ceiling(N=N)
    dirs = oracle.geodesic_dirs(N)
    up = dirs[:, 2] > 0
    xh = 10.0 * dirs[:, 0] / np.where(up, dirs[:, 2], 1.0)
    yh = 10.0 * dirs[:, 1] / np.where(up, dirs[:, 2], 1.0)
    expect = int(np.sum(up & (np.abs(xh) <= 1e-4) & (np.abs(yh) < 99.0)))
    assert expect >= N + 1
    _, fl, _ = oracle.trace(sc)
    assert int(np.sum((fl & oracle.FLAG_NEAR_EDGE) != 0)) == expect
    d = sbr.scene_to_device(sc)
    bvh = sbr.build_bvh(d["tri"], d["surface_id"], d["S"])
    st = sbr.trace(bvh, d["tx"], d["rx"], N, 1, count_visits=True).stats()
    assert st["near_edge_hits"] == expect
    # the default (uninstrumented) kernel leaves the counter at zero
    assert sbr.trace(bvh, d["tx"], d["rx"], N, 1).stats()["near_edge_hits"] == 0


def _oracle_H_of(sc, ex, tx_elem=None, rx_elem=None, freqs=None, fsel=None):
    """The oracle's direct FP64 sum of Eq. 13-14 over the GPU's own path list,
    with the oracle's own gains (so the comparison isolates the synthesis)."""
    paths = dict(rx=ex["rx"], nb=ex["nb"], seq=ex["seq"], pts=ex["pts"], L=ex["L"])
    f = sc["freqs"] if fsel is None else sc["freqs"][fsel]
    kw = {} if fsel is None else dict(freqs=f, gamma=sc["gamma_db_km"][fsel], disp=sc["disp_deg_km"][fsel])
    g_ref = oracle.gains(sc, paths, **kw)
    return oracle.synth_H(paths, g_ref, f, sc["tx"], sc["rx"][0],
                          sc["tx_elem"] if tx_elem is None else tx_elem,
                          sc["rx_elem"] if rx_elem is None else rx_elem)


def _h_errors(H, Ho):
    """Per-output error against the oracle: max |dH| / max |H|, and the median
    of |dH| / |H| over the outputs with |H| > 1e-3 max |H|."""
    a = np.abs(Ho)
    big = a > 1e-3 * a.max()
    return float(np.abs(H - Ho).max() / a.max()), float(np.median(np.abs(H - Ho)[big] / a[big]))


# Error budget of the split-precision forms, per product of two operands x, y:
# x = hi + lo with |x - hi| <= 2^-(s+1) |x| and lo itself rounded to s bits,
# so hi*hi + hi*lo + lo*hi leaves ~3 * 2^-(2s+1) |x y| (BF16: s = 8 -> 1.1e-5;
# FP16: s = 11 -> 1.8e-7); the on-chip phase adds the FP32 rounding of f*delay
# (a few 1e-7 of a cycle for delays of a few cm at 100 GHz). Summed over the
# paths, the maximum error stays within a few of those units of max |H| and
# the median within one.
TC_TOL = {2: (3e-5, 1e-5), 3: (1e-5, 3e-6)}   # form: (max |dH|/max|H|, median rel.)


@pytest.mark.parametrize("form", [2, 3])
@pytest.mark.parametrize("ny,nz,nr,F", [(16, 16, 64, 16), (10, 10, 10, 5), (20, 15, 70, 3), (9, 7, 13, 4)])
def test_tensor_core_synthesis_matches_oracle(sbr, ny, nz, nr, F, form):
    # BF16 (form 2) or FP16 (form 3) hi/lo split on tcgen05 against the FP64
    # oracle's direct sum, element by element, on the GPU's path list; shapes
    # cover one tile, ragged tiles (Nt=100, Nr=10), two M and N tiles (Nr=70,
    # Nt=300) and an odd row length (Nt=63: rows of H start on odd elements,
    # Nr=13: a partial group of 8 receive elements)
    sc = scenes.config3(N=60, K=3, F=F, ny_tx=ny, nz_tx=nz, n_rx=nr)
    r = sbr.run_scene(sc)
    d = r["dev"]
    assert r["paths"].n > 20
    ex = to_numpy(r["export"])
    Ho = _oracle_H_of(sc, ex)
    Htc = sbr.synthesize_H(r["paths"], r["g"], d["freqs"], d["tx_elem"], d["rx_elem"], 0, form).cpu().numpy()
    assert Htc.shape == Ho.shape == (F, nr, ny * nz)
    e_max, e_med = _h_errors(Htc, Ho)
    print("tcgen05 form", form, (ny * nz, nr, F), "vs oracle: max|dH|/max|H| =", e_max, "median rel =", e_med)
    tol_max, tol_med = TC_TOL[form]
    assert e_max < tol_max
    assert e_med < tol_med
    # every frequency on its own (none dropped or shifted)
    per_f = np.abs(Htc - Ho).reshape(F, -1).max(1) / np.abs(Ho).reshape(F, -1).max(1)
    assert per_f.max() < 1e-4
    # the CUDA-core FP64 form agrees with the oracle too (the tests above compare
    # the tensor-core forms against the oracle itself, not against it)
    H64 = sbr.synthesize_H(r["paths"], r["g"], d["freqs"], d["tx_elem"], d["rx_elem"], 0, 0).cpu().numpy()
    assert _h_errors(H64, Ho)[0] < 5e-6


@pytest.mark.parametrize("form", [2, 3])
def test_tensor_core_synthesis_with_many_paths(sbr, form):
    # a closed room at K = 5 gives one receiver well over a hundred reflected
    # paths: many K-chunks of 32 paths, the two operand stages alternating
    # within a tile and across tiles; element by element against the oracle
    lam = C0 / 60e9
    sc = scenes.shoebox(N=61, K=5, sub=3, n_rx=1)
    sc = dict(sc, tx_elem=scenes.upa_yz(sc["tx"], 6, 5, lam / 2), rx_elem=scenes.ula_y(sc["rx"][0], 11, lam / 2),
              freqs=np.array([59.5e9, 60e9, 60.5e9]), gamma_db_km=np.zeros(3, np.float32),
              disp_deg_km=np.zeros(3, np.float32))
    r = sbr.run_scene(sc)
    ex = to_numpy(r["export"])
    n_refl = int((ex["nb"] > 0).sum())
    assert n_refl > 128, n_refl      # at least five chunks
    Ho = _oracle_H_of(sc, ex)
    d = r["dev"]
    H = sbr.synthesize_H(r["paths"], r["g"], d["freqs"], d["tx_elem"], d["rx_elem"], 0, form).cpu().numpy()
    assert H.shape == Ho.shape == (3, 11, 30)
    e_max, e_med = _h_errors(H, Ho)
    print("tcgen05 form", form, "with", n_refl, "reflected paths: max", e_max, "median", e_med)
    tol_max, tol_med = TC_TOL[form]
    assert e_max < tol_max and e_med < tol_med


def test_synthesis_and_capacity_at_128x128_tx(sbr):
    # the largest Tx array of the capacity trend (128 x 128 UPA, Nt = 16384) on
    # four subcarriers: every form against the oracle on sampled transmit
    # elements (all receive elements and frequencies), and the capacity of the
    # FP16x3 H against the oracle's log-det of that same H
    sc = scenes.config3(N=60, K=3, F=4)
    lam = 299792458.0 / 100e9
    te = scenes.upa_yz(sc["tx"], 128, 128, lam / 2)
    sc = dict(sc, tx_elem=te)
    r = sbr.run_scene(sc)
    ex = to_numpy(r["export"])
    d = r["dev"]
    rng = np.random.default_rng(128)
    pi = np.unique(np.concatenate([[0, 127, 16383 - 127, 16383], rng.choice(16384, 60, replace=False)]))
    Ho = _oracle_H_of(sc, ex, tx_elem=te[pi])
    te_d = torch.as_tensor(te, dtype=torch.float64, device="cuda")
    for form, (tol_max, tol_med) in ((0, (5e-6, 1e-6)), (1, (2e-5, 1e-5)), (2, TC_TOL[2]), (3, TC_TOL[3])):
        H = sbr.synthesize_H(r["paths"], r["g"], d["freqs"], te_d, d["rx_elem"], 0, form)
        assert tuple(H.shape) == (4, 64, 16384)
        e_max, e_med = _h_errors(H.cpu().numpy()[:, :, pi], Ho)
        print("128x128 Tx, form", form, "max", e_max, "median", e_med)
        assert e_max < tol_max and e_med < tol_med, (form, e_max, e_med)
        if form == 3:
            snr = np.arange(0.0, 31.0, 5.0)
            C = sbr.capacity(H, snr).cpu().numpy()
            Co = oracle.capacity(H.cpu().numpy().astype(np.complex128), snr)
            assert np.abs(C - Co).max() < 1e-5 * np.abs(Co).max(), (C, Co)
            assert np.all(np.diff(C) > 0)


@pytest.mark.parametrize("form", [2, 3])
def test_tensor_core_synthesis_los_only(sbr, form):
    # no reflected path: the GEMM is empty and the epilogue writes the LoS term alone
    sc = dict(name="free", tri=np.zeros((0, 3, 3), np.float32), surface_id=np.zeros(0, np.int32),
              materials=np.zeros((0, 3)), tx=np.array([0.0, 0.0, 1.0]),
              rx=np.array([[3.0, 0.5, 1.2]]), rx_valid=np.ones(1, bool),
              freqs=np.array([27e9, 28e9]), gamma_db_km=np.zeros(2, np.float32),
              disp_deg_km=np.zeros(2, np.float32), N=30, K=1, pol="V",
              tx_elem=scenes.upa_yz([0.0, 0.0, 1.0], 4, 4, 0.05),
              rx_elem=scenes.ula_y([3.0, 0.5, 1.2], 6, 0.05))
    r = sbr.run_scene(sc)
    d = r["dev"]
    H64 = sbr.synthesize_H(r["paths"], r["g"], d["freqs"], d["tx_elem"], d["rx_elem"], 0, 0).cpu().numpy()
    Htc = sbr.synthesize_H(r["paths"], r["g"], d["freqs"], d["tx_elem"], d["rx_elem"], 0, form).cpu().numpy()
    # the LoS term is evaluated in the FP32 epilogue (phase ~1e-6 relative)
    assert np.abs(Htc - H64).max() < 1e-5 * np.abs(H64).max()


def test_export_into_pinned_host_buffers(sbr):
    # the path list copied straight into pinned host memory equals the device export
    sc = SCENES["urban_small"]()
    r = sbr.run_scene(sc)
    ex = r["paths"].export()
    pinned = {k: torch.empty(v.shape, dtype=v.dtype, pin_memory=True) for k, v in ex.items()}
    r["paths"].export(out=pinned)
    torch.cuda.synchronize()
    for k, v in ex.items():
        assert torch.equal(pinned[k], v.cpu()), k
    with pytest.raises(ValueError):
        r["paths"].export(out={k: torch.empty(v.shape, dtype=v.dtype) for k, v in ex.items()})


def _wide_rx_array(sc, n, spacing, extra=()):
    """Receivers = the elements of a wide ULA (traced one by one), plus extra points."""
    el = scenes.ula_y([8.5, 4.0, 2.5], n, spacing)   # above every furniture box (heights <= 2 m)
    if len(extra):
        el = np.concatenate([el, np.asarray(extra, np.float64).reshape(-1, 3)])
    sc = dict(sc, rx=el, rx_valid=np.ones(len(el), bool), rx_elem=el)
    return sc


@pytest.mark.parametrize("precision,tol", [(0, 5e-6), (1, 2e-5)])
def test_per_element_synthesis_matches_oracle(sbr, precision, tol):
    # a 24-element ULA of 5.75 m aperture, and one point outside the room (no paths)
    sc = _wide_rx_array(scenes.config3(N=40, K=3, F=8, ny_tx=3, nz_tx=2), 24, 0.25,
                        extra=[[12.0, 4.0, 1.5]])
    r = sbr.run_scene(sc)
    ex = to_numpy(r["export"])
    d = r["dev"]
    H = sbr.synthesize_H_elements(r["paths"], r["g"], d["freqs"], d["tx_elem"], precision).cpu().numpy()
    assert H.shape == (8, 25, 6)
    paths = dict(rx=ex["rx"], nb=ex["nb"], pts=ex["pts"], L=ex["L"])
    g_ref = oracle.gains(sc, dict(rx=ex["rx"], nb=ex["nb"], seq=ex["seq"], pts=ex["pts"], L=ex["L"]))
    Ho = oracle.synth_H_elements(paths, g_ref, sc["freqs"], sc["tx"], sc["tx_elem"], sc["rx_elem"])
    err = np.abs(H - Ho).max() / np.abs(Ho).max()
    print("per-element synthesis precision", precision, "max|dH|/max|H| =", err)
    assert err < tol
    # the receiver outside the room has no path and a zero row
    assert not np.any(ex["rx"] == 24) and np.all(H[:, 24, :] == 0)
    # the array is non-stationary: its elements do not all see the same surface sequences
    sets = [frozenset(tuple(s[:m]) for s, m in zip(ex["seq"][ex["rx"] == q], ex["nb"][ex["rx"] == q]))
            for q in range(24)]
    assert len(set(sets)) > 1


def test_per_element_synthesis_free_space_is_the_spherical_wave(sbr):
    tx = np.array([0.0, 0.0, 1.0])
    rx_el = scenes.ula_y([6.0, 0.5, 1.2], 9, 0.75)       # 6 m aperture: distinct path loss per element
    sc = dict(name="free", tri=np.zeros((0, 3, 3), np.float32), surface_id=np.zeros(0, np.int32),
              materials=np.zeros((0, 3)), tx=tx, rx=rx_el, rx_valid=np.ones(len(rx_el), bool),
              freqs=np.array([99e9, 100e9, 101e9]), gamma_db_km=np.zeros(3, np.float32),
              disp_deg_km=np.zeros(3, np.float32), N=30, K=1, pol="V",
              tx_elem=scenes.upa_yz(tx, 4, 4, 0.0015), rx_elem=rx_el)
    r = sbr.run_scene(sc)
    ex = to_numpy(r["export"])
    assert ex["nb"].tolist() == [0] * len(rx_el)
    d = r["dev"]
    f = sc["freqs"]
    d0 = np.linalg.norm(rx_el - tx, axis=1)
    dist = np.linalg.norm(rx_el[:, None, :] - sc["tx_elem"][None, :, :], axis=2)
    ref = (C0 / (4 * np.pi * f[:, None, None] * d0[None, :, None])) \
        * np.exp(-2j * np.pi * f[:, None, None] * dist[None] / C0)
    for prec, tol in ((0, 1e-6), (1, 1e-5)):
        H = sbr.synthesize_H_elements(r["paths"], r["g"], d["freqs"], d["tx_elem"], prec).cpu().numpy()
        assert np.abs(H - ref).max() < tol * np.abs(ref).max(), prec


def test_per_element_synthesis_reduces_to_reference_point_form(sbr):
    # one receive element at the traced receiver: both syntheses describe the same channel
    sc = scenes.config3(N=40, K=3, F=6, ny_tx=4, nz_tx=2)
    sc = dict(sc, rx_elem=sc["rx"][:1].copy())
    r = sbr.run_scene(sc)
    d = r["dev"]
    He = sbr.synthesize_H_elements(r["paths"], r["g"], d["freqs"], d["tx_elem"], 0).cpu().numpy()
    Hr = sbr.synthesize_H(r["paths"], r["g"], d["freqs"], d["tx_elem"], d["rx_elem"], 0, 0).cpu().numpy()
    assert He.shape == Hr.shape == (6, 1, 8)
    assert np.abs(He - Hr).max() <= 1e-6 * np.abs(Hr).max()
    for bad in (dict(precision=2), dict(precision=3)):
        with pytest.raises(sbr.SbrError):
            sbr.synthesize_H_elements(r["paths"], r["g"], d["freqs"], d["tx_elem"], **bad)


@pytest.mark.parametrize("name", ["urban_small", "urban_med", "shoebox_K5", "indoor_small"])
def test_path_list_is_in_key_order(sbr, name):
    # paths come out sorted by (receiver, reflections, surface sequence), each key once;
    # the per-receiver offsets follow that order
    r = sbr.run_scene(SCENES[name]())
    ex = to_numpy(r["export"])
    keys = [(int(q), int(m)) + tuple(int(x) for x in s[:m]) for q, m, s in zip(ex["rx"], ex["nb"], ex["seq"])]
    assert len(keys) > 10
    assert all(a < b for a, b in zip(keys, keys[1:]))


def test_large_path_list_is_in_key_order(sbr):
    # 4096 receivers: more keys than the single-block sort holds, so the key sort
    # runs as one cooperative launch; the order and uniqueness rules are the same
    sc = scenes.config2(N=150, K=4, nx=3, ny=3, sub=4, ground_sub=8, rx_grid=64)
    r = sbr.run_scene(sc)
    info = r["paths"].info()
    assert info["n_keys"] > 12288, info
    ex = to_numpy(r["export"])
    keys = [(int(q), int(m)) + tuple(int(x) for x in s[:m]) for q, m, s in zip(ex["rx"], ex["nb"], ex["seq"])]
    assert all(a < b for a, b in zip(keys, keys[1:]))
    # receiver offsets agree with the sorted receiver column
    n_rx = len(sc["rx"])
    counts = np.bincount(ex["rx"], minlength=n_rx)
    pdp, st = sbr.pdp_angles(r["paths"], r["g"], 0, float(sc["freqs"][0]), 1e-9, 64)
    st = st.cpu().numpy()
    assert np.all(np.isinf(st[counts == 0, 1]))
    assert np.mean(np.isfinite(st[counts > 0, 1])) > 0.9   # (gains below the FP32 range read as no power)


def test_sort_without_cooperative_launch_gives_the_same_paths(sbr, monkeypatch):
    # SBR_SORT_PHASES=1 keeps the radix sorts above the single-block size to their
    # per-phase launches (the path taken where no cooperative launch exists): the
    # BVH's Morton order and the key order, hence the whole path list, are identical
    sc = scenes.config2(N=150, K=4, rx_grid=64)
    assert len(sc["tri"]) > 12288
    ref = sbr.run_scene(sc)
    monkeypatch.setenv("SBR_SORT_PHASES", "1")
    alt = sbr.run_scene(sc)
    monkeypatch.delenv("SBR_SORT_PHASES")
    assert ref["paths"].info()["n_keys"] > 12288
    a, b = to_numpy(ref["export"]), to_numpy(alt["export"])
    assert a.keys() == b.keys()
    for k in a:
        assert np.array_equal(a[k], b[k]), k
    assert np.array_equal(ref["g"].cpu().numpy(), alt["g"].cpu().numpy())


@pytest.mark.parametrize("name", ["urban_small", "urban_med", "shoebox_K5", "indoor_small"])
def test_sah_top_bvh_gives_the_same_paths(sbr, name):
    # the SAH-rebuilt top changes the tree, not the closest hits: identical path lists
    sc = SCENES[name]()
    d = sbr.scene_to_device(sc)
    out = []
    for sah in (False, True):
        bvh = sbr.build_bvh(d["tri"], d["surface_id"], d["S"], sah_top=sah)
        info = bvh.info()
        assert info["n_nodes"] == max(1, len(sc["tri"]) - 1) and 1 <= info["depth"] <= 64
        tr = sbr.trace(bvh, d["tx"], d["rx"], sc["N"], sc["K"], table_log2=18)
        st = tr.stats()
        pl = sbr.paths(tr, bvh)
        out.append((st["ray_bounces"], to_numpy(pl.export())))
    assert out[0][0] == out[1][0]
    for k in out[0][1]:
        assert np.array_equal(out[0][1][k], out[1][1][k]), k


def test_sah_top_bvh_with_duplicated_faces(sbr):
    # every face three times (same surface): equal centroids exercise the SAH build's
    # split by position, and tied hits go to the lowest face id in both trees
    sc = scenes.shoebox(N=61, K=4, sub=3)
    tri = np.concatenate([sc["tri"]] * 3)
    sid = np.concatenate([sc["surface_id"]] * 3)
    sc = dict(sc, tri=tri, surface_id=sid)
    d = sbr.scene_to_device(sc)
    out = []
    for sah in (False, True):
        bvh = sbr.build_bvh(d["tri"], d["surface_id"], d["S"], sah_top=sah)
        tr = sbr.trace(bvh, d["tx"], d["rx"], sc["N"], sc["K"], table_log2=16)
        st = tr.stats()
        out.append((st["ray_bounces"], to_numpy(sbr.paths(tr, bvh).export())))
    assert out[0][0] == out[1][0]
    for k in out[0][1]:
        assert np.array_equal(out[0][1][k], out[1][1][k]), k
    # the faces reported are the lowest ids: the first copy
    assert np.all(out[0][1]["face"][out[0][1]["face"] >= 0] < len(tri) // 3)
