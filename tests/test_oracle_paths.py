"""Pins for the oracle's trace, dedup, refinement and path gains.

Independent references: the two-ray ground model in closed form, the corner
reflector's four paths, exhaustive image-method enumeration (tests/
im_bruteforce.py) on tiny scenes, Snell's law of reflection at every refined
point, Friis' law with the Eq. 9 absorption term, and Tx/Rx reciprocity.
"""
import numpy as np
import pytest

import oracle
import scenes
from im_bruteforce import enumerate_paths

C0 = 299792458.0


def _keyset(paths, rx=0):
    return {tuple(paths["seq"][i][: paths["nb"][i]]) for i in range(len(paths["rx"]))
            if paths["rx"][i] == rx}


@pytest.mark.parametrize("make", [scenes.config1, scenes.corner_reflector, scenes.two_ray,
                                  scenes.shoebox])
def test_path_set_equals_exhaustive_image_method(make):
    sc = make()
    r = oracle.run(sc)
    p = r["paths"]
    for rxi in range(len(sc["rx"])):
        im = enumerate_paths(sc, rx_index=rxi)
        sbr = _keyset(p, rxi)
        diff = sbr ^ set(im)
        # a difference is allowed only for keys whose every producing ray is edge-ambiguous
        for k in diff:
            sel = [i for i in range(len(p["rx"])) if p["rx"][i] == rxi
                   and tuple(p["seq"][i][: p["nb"][i]]) == k]
            assert sel and p["all_flagged"][sel[0]], (make.__name__, rxi, k)
        for k in set(im) & sbr:
            i = [i for i in range(len(p["rx"])) if p["rx"][i] == rxi
                 and tuple(p["seq"][i][: p["nb"][i]]) == k][0]
            assert abs(p["L"][i] - im[k]["L"]) <= 1e-12 * im[k]["L"]
            assert np.allclose(p["pts"][i][: len(k)], im[k]["pts"], rtol=0, atol=1e-9)


def test_corner_reflector_has_four_paths():
    r = oracle.run(scenes.corner_reflector())
    nb = sorted(r["paths"]["nb"].tolist())
    assert nb == [0, 1, 1, 2]


def _textbook_gamma(er, th, pol):
    n = np.sqrt(er)
    tt = np.arcsin(np.sin(th) / n)
    if pol == "H":   # E perpendicular to the plane of incidence
        return (np.cos(th) - n * np.cos(tt)) / (np.cos(th) + n * np.cos(tt))
    return (n * np.cos(th) - np.cos(tt)) / (n * np.cos(th) + np.cos(tt))


@pytest.mark.parametrize("pol", ["H", "V"])
@pytest.mark.parametrize("ht,hr,d", [(10.0, 2.0, 50.0), (25.0, 1.5, 300.0), (3.0, 3.0, 12.0)])
def test_two_ray_ground_model(pol, ht, hr, d):
    f = 28e9
    sc = scenes.two_ray(h_tx=ht, h_rx=hr, dist=d, f=f, eps_r=5.31, sigma=0.0, pol=pol, N=220)
    r = oracle.run(sc)
    p, g = r["paths"], r["g"][:, 0]
    assert sorted(p["nb"].tolist()) == [0, 1]
    los, gr = (0, 1) if p["nb"][0] == 0 else (1, 0)
    d1 = np.hypot(d, ht - hr)
    d2 = np.hypot(d, ht + hr)
    assert abs(p["L"][los] - d1) < 1e-12 * d1
    assert abs(p["L"][gr] - d2) < 1e-12 * d2
    # reflection point at x = d ht / (ht + hr) on the ground
    assert np.allclose(p["pts"][gr][0], [d * ht / (ht + hr), 0, 0], atol=1e-10)
    lam = C0 / f
    th = np.arctan2(d, ht + hr)  # incidence angle from the normal
    gam = _textbook_gamma(5.31, th, pol)
    assert abs(g[los] - lam / (4 * np.pi * d1)) < 1e-12 * abs(g[los])
    assert abs(g[gr] - gam * lam / (4 * np.pi * d2)) < 1e-10 * abs(g[gr])
    # total field: (lambda / 4 pi) [e^{-jk d1}/d1 + Gamma e^{-jk d2}/d2]
    k = 2 * np.pi * f / C0
    e_ref = lam / (4 * np.pi) * (np.exp(-1j * k * d1) / d1 + gam * np.exp(-1j * k * d2) / d2)
    e = sum(g[i] * np.exp(-2j * np.pi * ((f * p["L"][i] / C0) % 1.0)) for i in range(2))
    assert abs(e - e_ref) < 1e-9 * abs(e_ref)


def test_vpol_grazing_cancellation():
    # V-pol ground reflection tends to -1 at grazing: far Rx, low antennas
    sc = scenes.two_ray(h_tx=1.0, h_rx=1.0, dist=900.0, eps_r=5.31, sigma=0.48, pol="V", N=800)
    r = oracle.run(sc)
    p, g = r["paths"], r["g"][:, 0]
    los, gr = (0, 1) if p["nb"][0] == 0 else (1, 0)
    ratio = g[gr] / g[los] * p["L"][gr] / p["L"][los]
    assert abs(ratio + 1) < 0.05


@pytest.mark.parametrize("make", [scenes.config1, scenes.shoebox])
def test_snell_reflection_at_refined_points(make):
    sc = make()
    r = oracle.run(sc)
    p = r["paths"]
    tri = sc["tri"].astype(float)
    for i in range(len(p["rx"])):
        m = p["nb"][i]
        chain = [sc["tx"]] + [p["pts"][i][k] for k in range(m)] + [sc["rx"][p["rx"][i]]]
        for k in range(1, m + 1):
            t = tri[p["face"][i][k - 1]]
            n = np.cross(t[1] - t[0], t[2] - t[0]); n /= np.linalg.norm(n)
            din = chain[k] - chain[k - 1]; din /= np.linalg.norm(din)
            dout = chain[k + 1] - chain[k]; dout /= np.linalg.norm(dout)
            assert np.allclose(dout, din - 2 * (din @ n) * n, atol=1e-9)
            # reported face is the lowest-id triangle of the surface containing the point
            sid = sc["surface_id"]
            assert sid[p["face"][i][k - 1]] == p["seq"][i][k - 1]


def test_kept_ray_retrace_follows_the_path():
    sc = scenes.shoebox()
    r = oracle.run(sc)
    p = r["paths"]
    a = oracle.alpha(sc["N"])
    for i in range(len(p["rx"])):
        seg = oracle.trace_one(sc, int(p["ray"][i]))
        m = p["nb"][i]
        assert len(seg["face"]) >= m + 1
        faces = seg["face"][:m]
        assert [int(sc["surface_id"][f]) for f in faces] == list(p["seq"][i][:m])
        chain = [sc["tx"]] + [p["pts"][i][k] for k in range(m)]
        for k in range(m):
            hit = seg["o"][k + 1]
            s = seg["L"][k + 1]
            t = sc["tri"][faces[k]].astype(float)
            n = np.cross(t[1] - t[0], t[2] - t[0]); n /= np.linalg.norm(n)
            din = p["pts"][i][k] - chain[k]; din /= np.linalg.norm(din)
            # the ray's bounce point lies within a ray-tube width (alpha s across the
            # ray, stretched by 1/cos(theta_i) along the surface) of the exact point
            assert np.linalg.norm(hit - p["pts"][i][k]) <= a * s / abs(din @ n)


def test_k0_gives_los_only_and_tiny_sphere_gives_nothing():
    sc = scenes.config1(N=60, K=0)
    r = oracle.run(sc)
    assert r["paths"]["nb"].tolist() == [0]
    c, _, _ = oracle.trace(sc, alpha_=1e-12)
    assert len(c) == 0


def _empty_scene(d, gamma):
    return dict(name="free", tri=np.zeros((0, 3, 3), np.float32), surface_id=np.zeros(0, np.int32),
                materials=np.zeros((0, 3)), tx=np.array([0.0, 0.0, 0.0]),
                rx=np.array([[d, 0.3 * d, 0.1 * d]]), rx_valid=np.ones(1, bool),
                freqs=np.array([60e9]), gamma_db_km=np.array([gamma], np.float32),
                disp_deg_km=np.zeros(1, np.float32), tx_elem=np.zeros((1, 3)),
                rx_elem=np.array([[d, 0.3 * d, 0.1 * d]]), N=40, K=2, pol="V")


def test_friis_slope_and_absorption_linear_in_length():
    lam = C0 / 60e9
    vals = []
    for d in (10.0, 100.0, 1000.0):
        sc = _empty_scene(d, 15.0)
        r = oracle.run(sc)
        L = r["paths"]["L"][0]
        assert abs(L - d * np.sqrt(1.1)) < 1e-12 * L
        g = abs(r["g"][0, 0])
        ref_db = 20 * np.log10(lam / (4 * np.pi * L)) - 15.0 * L / 1000.0
        assert abs(20 * np.log10(g) - ref_db) < 1e-9
        vals.append(20 * np.log10(g) + 15.0 * L / 1000.0)
    assert abs((vals[1] - vals[0]) + 20) < 1e-9 and abs((vals[2] - vals[1]) + 20) < 1e-9


def test_dispersion_rotates_the_phase_by_phi_times_length():
    # specific dispersion phi (deg/km) over the path length L: a phase of -phi L / 1000 degrees,
    # magnitude unchanged; a quarter, half and full turn over the LoS length
    sc = _empty_scene(250.0, 15.0)
    r0 = oracle.run(sc)
    L = r0["paths"]["L"][0]
    g0 = r0["g"][0, 0]
    for turn, factor in ((0.25, -1j), (0.5, -1.0), (1.0, 1.0)):
        phi = 360.0 * turn / (L / 1000.0)
        sc["disp_deg_km"] = np.array([phi], np.float32)
        g = oracle.run(sc)["g"][0, 0]
        # phi is stored in float32: allow its rounding (2^-24 relative) in the phase
        assert abs(g - g0 * factor) <= abs(g0) * (1e-12 + 2 * np.pi * turn * 2.0 ** -23)
        assert abs(abs(g) - abs(g0)) <= 1e-12 * abs(g0)


@pytest.mark.parametrize("pol", ["V", "H"])
@pytest.mark.parametrize("make", [scenes.config1, scenes.corner_reflector])
def test_reciprocity(pol, make):
    sc = make()
    sc["pol"] = pol
    rs = dict(sc)
    rs["tx"], rs["rx"] = sc["rx"][0].copy(), sc["tx"][None, :].copy()
    a, b = oracle.run(sc), oracle.run(rs)
    ka = {tuple(a["paths"]["seq"][i][: a["paths"]["nb"][i]]): i for i in range(len(a["paths"]["rx"]))}
    kb = {tuple(b["paths"]["seq"][i][: b["paths"]["nb"][i]])[::-1]: i
          for i in range(len(b["paths"]["rx"]))}
    assert set(ka) == set(kb)
    for k in ka:
        i, j = ka[k], kb[k]
        assert abs(a["paths"]["L"][i] - b["paths"]["L"][j]) < 1e-12 * a["paths"]["L"][i]
        assert abs(a["g"][i, 0] - b["g"][j, 0]) < 1e-12 * abs(a["g"][i, 0])
