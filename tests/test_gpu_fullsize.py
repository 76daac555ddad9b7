"""Parity at the benchmark sizes, on outputs the FP64 oracle can compute one
by one (the full oracle trace of 10^7 rays against 51,600 faces is hours).

Urban workload (10,000,002 rays, 6 reflections, 1024 receivers, 51,600
triangles), in the launch configuration bench.py times:
  - kept rays of a random sample of GPU paths are retraced by the oracle, which
    must receive the same (rx, surface sequence) on that ray unless it flags
    the ray as edge-ambiguous;
  - a spread sample of rays is traced by the oracle; every reception of an
    unflagged ray whose key refines to a valid path must be in the GPU set;
  - sampled paths are refined and their gains computed by the oracle: faces
    exact, lengths 1e-9, gains 1e-4 relative.
Indoor MIMO workload (3,994,242 rays, H [1024, 64, 256]): sampled H entries
of every precision form against the oracle's direct sum over the GPU's paths.
"""
import numpy as np
import pytest

import oracle
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


@pytest.fixture(scope="module")
def urban(sbr):
    sc = scenes.config2()
    r = sbr.run_scene(sc)
    return sc, r, to_numpy(r["export"]), r["g"].cpu().numpy()


def _keys_of(cands):
    return {(int(c["rx"]), tuple(int(x) for x in c["seq"][: c["nb"]])) for c in cands}


def test_urban_kept_rays_retrace(urban):
    sc, r, ex, g = urban
    P = len(ex["rx"])
    assert P > 1000
    rng = np.random.default_rng(11)
    idx = rng.choice(P, size=40, replace=False)
    bad = []
    for i in idx:
        ray = int(ex["ray"][i])
        c, fl, _ = oracle.trace(sc, ray_begin=ray, ray_end=ray + 1)
        key = (int(ex["rx"][i]), tuple(int(x) for x in ex["seq"][i][: ex["nb"][i]]))
        if key not in _keys_of(c) and not fl[0]:
            bad.append((key, ray))
    assert not bad, bad


def test_urban_sampled_rays_are_all_found(urban):
    sc, r, ex, g = urban
    gpu_keys = {(int(ex["rx"][i]), tuple(int(x) for x in ex["seq"][i][: ex["nb"][i]]))
                for i in range(len(ex["rx"]))}
    R = 10 * sc["N"] ** 2 + 2
    cands = []
    flags_all = []
    for c in range(24):
        b0 = (R * c) // 24 + 12345
        cc, fl, _ = oracle.trace(sc, ray_begin=b0, ray_end=b0 + 100)
        cands.append(cc)
        flags_all.append((b0, fl))
    cc = np.concatenate(cands)
    assert len(cc) > 0
    unflagged = cc[cc["flags"] == 0]
    keys, nprod, allf = oracle.dedup(unflagged)
    ref = oracle.refine(sc, keys)
    missing = []
    for k in range(len(keys)):
        if not ref["valid"][k]:
            continue
        key = (int(keys["rx"][k]), tuple(int(x) for x in keys["seq"][k][: keys["nb"][k]]))
        if key not in gpu_keys:
            missing.append(key)
    assert not missing, missing[:10]


def test_urban_sampled_paths_refine_and_gains(urban):
    sc, r, ex, g = urban
    rng = np.random.default_rng(5)
    idx = np.sort(rng.choice(len(ex["rx"]), size=300, replace=False))
    keys = np.zeros(len(idx), oracle.CAND_DTYPE)
    keys["rx"] = ex["rx"][idx]
    keys["nb"] = ex["nb"][idx]
    keys["seq"] = ex["seq"][idx]
    ref = oracle.refine(sc, keys)
    assert ref["valid"].all()
    for j, i in enumerate(idx):
        m = ex["nb"][i]
        assert np.array_equal(ref["face"][j][:m], ex["face"][i][:m])
        assert abs(ref["L"][j] - ex["L"][i]) <= 1e-9 * ref["L"][j]
    paths = oracle.paths_of(sc, keys, ref)
    go = oracle.gains(sc, paths)
    err = np.abs(g[idx] - go) / np.abs(go)
    assert err.max() < 1e-4, err.max()


def test_indoor_full_H_sampled_entries(sbr):
    sc = scenes.config3()
    r = sbr.run_scene(sc)
    ex = to_numpy(r["export"])
    d = r["dev"]
    rng = np.random.default_rng(3)
    fi = np.sort(rng.choice(len(sc["freqs"]), 6, replace=False))
    qi = np.sort(rng.choice(len(sc["rx_elem"]), 5, replace=False))
    pi = np.sort(rng.choice(len(sc["tx_elem"]), 7, replace=False))
    paths = dict(rx=ex["rx"], nb=ex["nb"], seq=ex["seq"], pts=ex["pts"], L=ex["L"])
    g_ref = oracle.gains(sc, paths, freqs=sc["freqs"][fi], gamma=sc["gamma_db_km"][fi],
                         disp=sc["disp_deg_km"][fi])
    Ho = oracle.synth_H(paths, g_ref, sc["freqs"][fi], sc["tx"], sc["rx"][0], sc["tx_elem"][pi],
                        sc["rx_elem"][qi])
    for prec, tol in ((0, 5e-6), (1, 2e-5), (2, 5e-5), (3, 2e-5)):
        H = sbr.synthesize_H(r["paths"], r["g"], d["freqs"], d["tx_elem"], d["rx_elem"], 0, prec)
        Hs = H.cpu().numpy()[np.ix_(fi, qi, pi)]
        err = np.abs(Hs - Ho).max() / np.abs(Ho).max()
        print("full-size H, precision", prec, "sampled max|dH|/max|H| =", err, "paths", r["paths"].n)
        assert err < tol
