"""Pins for the oracle's H(f) synthesis (Eq. 11-14), PDP and statistics
(Eq. 2, 4, 5) and capacity (Eq. 15-17, Frobenius-normalised reading).

Independent references: the factorised form U diag(w) V^T evaluated with
numpy, the spherical-wave response of a single LoS path, the plane-wave
limit of a distant path, closed forms of the RMS delay spread and of the
capacity of scaled-identity and rank-1 channels, and numpy's slogdet.
"""
import numpy as np
import pytest

import oracle
import scenes

C0 = 299792458.0


def _small_mimo(N=40, F=16, nt=(4, 3), nr=5, seed=3):
    sc = scenes.config3(N=N, K=2, n_furniture=4, wall_sub=2, box_sub=1, F=F, ny_tx=nt[0],
                        nz_tx=nt[1], n_rx=nr, seed=seed)
    return sc


def test_synth_direct_loop_equals_factorised_form():
    sc = _small_mimo()
    r = oracle.run(sc)
    p, g = r["paths"], r["g"]
    assert len(p["rx"]) >= 5
    H = oracle.synth_H(p, g, sc["freqs"], sc["tx"], sc["rx"][0], sc["tx_elem"], sc["rx_elem"])
    T, R = sc["tx_elem"], sc["rx_elem"]
    ref = np.zeros_like(H)
    for n in range(len(p["rx"])):
        m = p["nb"][n]
        if m == 0:
            dist = np.linalg.norm(R[:, None, :] - T[None, :, :], axis=2)     # [Nr, Nt]
            ph = np.exp(-2j * np.pi * sc["freqs"][:, None, None] * dist[None] / C0)
            ref += g[n][:, None, None] * ph
            continue
        P1, Pm = p["pts"][n][0], p["pts"][n][m - 1]
        dt = np.linalg.norm(T - P1, axis=1) - np.linalg.norm(sc["tx"] - P1)
        dr = np.linalg.norm(R - Pm, axis=1) - np.linalg.norm(sc["rx"][0] - Pm)
        w = g[n] * np.exp(-2j * np.pi * sc["freqs"] * p["L"][n] / C0)         # [F]
        U = np.exp(-2j * np.pi * sc["freqs"][:, None] * dr[None, :] / C0)     # [F, Nr]
        V = np.exp(-2j * np.pi * sc["freqs"][:, None] * dt[None, :] / C0)     # [F, Nt]
        ref += w[:, None, None] * U[:, :, None] * V[:, None, :]
    err = np.abs(H - ref).max() / np.abs(ref).max()
    assert err < 1e-9


def test_single_los_path_is_spherical_wave_response():
    f = np.array([27e9, 28e9, 29e9])
    sc = dict(name="free", tri=np.zeros((0, 3, 3), np.float32), surface_id=np.zeros(0, np.int32),
              materials=np.zeros((0, 3)), tx=np.array([0.0, 0.0, 1.0]),
              rx=np.array([[3.0, 0.5, 1.2]]), rx_valid=np.ones(1, bool), freqs=f,
              gamma_db_km=np.zeros(3, np.float32), disp_deg_km=np.zeros(3, np.float32),
              N=30, K=1, pol="V")
    T = scenes.upa_yz(sc["tx"], 4, 4, 0.05)
    R = scenes.ula_y(sc["rx"][0], 6, 0.05)
    r = oracle.run(sc)
    p, g = r["paths"], r["g"]
    assert p["nb"].tolist() == [0]
    H = oracle.synth_H(p, g, f, sc["tx"], sc["rx"][0], T, R)
    d0 = np.linalg.norm(sc["tx"] - sc["rx"][0])
    dist = np.linalg.norm(R[:, None, :] - T[None, :, :], axis=2)
    ref = (C0 / (4 * np.pi * f * d0))[:, None, None] * np.exp(-2j * np.pi * f[:, None, None] * dist / C0)
    assert np.abs(H - ref).max() < 1e-12 * np.abs(ref).max()


def test_far_path_approaches_plane_wave_steering():
    # one ground bounce 1.8 km away: per-element delays -> -(T_p - T0).u
    sc = scenes.two_ray(h_tx=30.0, h_rx=30.0, dist=1800.0, f=10e9, N=500)
    sc["freqs"] = np.array([10e9])
    r = oracle.run(sc)
    p, g = r["paths"], r["g"]
    gr = int(np.nonzero(p["nb"] == 1)[0][0])
    T = scenes.upa_yz(sc["tx"], 3, 3, 0.015)
    R = scenes.ula_y(sc["rx"][0], 4, 0.015)
    H = oracle.synth_H({k: v[gr:gr + 1] for k, v in p.items()}, g[gr:gr + 1], sc["freqs"],
                       sc["tx"], sc["rx"][0], T, R)
    P1 = p["pts"][gr][0]
    u_t = (P1 - sc["tx"]) / np.linalg.norm(P1 - sc["tx"])
    u_r = (P1 - sc["rx"][0]) / np.linalg.norm(P1 - sc["rx"][0])
    k = 2 * np.pi * 10e9 / C0
    a_t = np.exp(1j * k * (T - sc["tx"]) @ u_t)
    a_r = np.exp(1j * k * (R - sc["rx"][0]) @ u_r)
    w = g[gr, 0] * np.exp(-2j * np.pi * 10e9 * p["L"][gr] / C0)
    ref = w * np.outer(a_r, a_t)
    assert np.abs(H[0] - ref).max() < 1e-3 * abs(w)


def _paths_dict(L, aod, aoa):
    n = len(L)
    return dict(rx=np.zeros(n, np.int32), L=np.asarray(L, float),
                aod=np.asarray(aod, float).reshape(n, 2), aoa=np.asarray(aoa, float).reshape(n, 2))


def test_pdp_single_path_and_two_equal_taps():
    L = [30.0]
    g = np.array([[1e-4 * np.exp(0.3j)]])
    pdp, st = oracle.pdp_stats(_paths_dict(L, [[10, -5]], [[170, 5]]), g, 0, 28e9, 1e-9, 400, 1)
    k = int(np.floor(L[0] / C0 / 1e-9))
    assert abs(pdp[0, k] - 20 * np.log10(1e-4)) < 1e-12
    assert np.isneginf(np.delete(pdp[0], k)).all()
    assert abs(st[0, 1] - 80.0) < 1e-12 and abs(st[0, 0] - 80.0) < 1e-12
    assert st[0, 2] == 0.0
    assert np.allclose(st[0, 3:], [10, -5, 170, 5])
    L2 = [30.0, 75.0]
    g2 = np.array([[2e-5], [2e-5 * 1j]])
    pdp, st = oracle.pdp_stats(_paths_dict(L2, [[0, 0], [40, 10]], [[0, 0], [-20, 30]]), g2, 0,
                               28e9, 1e-9, 400, 1)
    assert abs(st[0, 2] - abs(L2[1] - L2[0]) / C0 / 2) < 1e-20
    assert np.allclose(st[0, 3:], [20, 5, -10, 15])
    assert abs(st[0, 1] + 10 * np.log10(2 * 4e-10)) < 1e-12


def test_rms_delay_spread_matches_eq5_moments():
    rng = np.random.default_rng(5)
    L = rng.uniform(10, 300, 40)
    g = (rng.normal(size=40) + 1j * rng.normal(size=40))[:, None] * 1e-5
    _, st = oracle.pdp_stats(_paths_dict(L, np.zeros((40, 2)), np.zeros((40, 2))), g, 0, 60e9,
                             1e-9, 2000, 1)
    tau = L / C0
    pw = np.abs(g[:, 0]) ** 2
    m = np.average(tau, weights=pw)
    ref = np.sqrt(np.average((tau - m) ** 2, weights=pw))
    assert abs(st[0, 2] - ref) < 1e-9 * ref


@pytest.mark.parametrize("n", [1, 4, 8])
def test_capacity_scaled_identity(n):
    F = 3
    H = np.stack([(0.3 + 0.1j) * np.eye(n)] * F)
    snr_db = np.array([0.0, 10.0, 20.0])
    C = oracle.capacity(H, snr_db)
    # W = (n^2/||H||^2) H H^H = n I  ->  C = n log2(1 + SNR)
    ref = n * np.log2(1 + 10 ** (snr_db / 10))
    assert np.allclose(C, ref, rtol=1e-12, atol=1e-12)


def test_capacity_rank_one():
    rng = np.random.default_rng(1)
    a = rng.normal(size=6) + 1j * rng.normal(size=6)
    b = rng.normal(size=9) + 1j * rng.normal(size=9)
    H = np.outer(a, b.conj())[None]
    snr_db = np.array([-5.0, 0.0, 30.0])
    C = oracle.capacity(H, snr_db)
    # one nonzero eigenvalue: (Nr Nt / ||H||^2) ||H||^2 = Nr Nt -> log2(1 + SNR Nr)
    ref = np.log2(1 + 10 ** (snr_db / 10) * 6)
    assert np.allclose(C, ref, rtol=1e-11)


@pytest.mark.parametrize("nr,nt", [(4, 7), (7, 4), (5, 5)])
def test_capacity_matches_numpy_slogdet(nr, nt):
    rng = np.random.default_rng(nr * 10 + nt)
    F = 5
    H = rng.normal(size=(F, nr, nt)) + 1j * rng.normal(size=(F, nr, nt))
    snr_db = np.array([0.0, 12.0])
    C = oracle.capacity(H, snr_db)
    q = np.mean(np.sum(np.abs(H) ** 2, axis=(1, 2)))
    ref = np.zeros(2)
    for s, sd in enumerate(snr_db):
        for f in range(F):
            W = H[f] @ H[f].conj().T if nt >= nr else H[f].conj().T @ H[f]
            W = W * nr * nt / q
            sign, ld = np.linalg.slogdet(np.eye(W.shape[0]) + 10 ** (sd / 10) / nt * W)
            ref[s] += ld / np.log(2) / F
    assert np.allclose(C, ref, rtol=1e-12)


def _free_space(f):
    return dict(name="free", tri=np.zeros((0, 3, 3), np.float32), surface_id=np.zeros(0, np.int32),
                materials=np.zeros((0, 3)), tx=np.array([0.0, 0.0, 1.0]), rx_valid=None, freqs=f,
                gamma_db_km=np.zeros(len(f), np.float32), disp_deg_km=np.zeros(len(f), np.float32),
                N=30, K=1, pol="V")


def test_per_element_free_space_is_the_exact_spherical_wave():
    # every receive element traced as a receiver of its own: in free space each row is
    # the element's own Friis amplitude times the exact element-pair phasor
    f = np.array([27e9, 28e9, 29e9])
    sc = _free_space(f)
    T = scenes.upa_yz(sc["tx"], 4, 4, 0.05)
    R = scenes.ula_y([3.0, 0.5, 1.2], 6, 0.05)
    sc["rx"] = R
    sc["rx_valid"] = np.ones(len(R), bool)
    r = oracle.run(sc)
    p, g = r["paths"], r["g"]
    assert sorted(p["rx"].tolist()) == list(range(len(R))) and (p["nb"] == 0).all()
    H = oracle.synth_H_elements(p, g, f, sc["tx"], T, R)
    d0 = np.linalg.norm(R - sc["tx"], axis=1)                                  # [Nr]
    dist = np.linalg.norm(R[:, None, :] - T[None, :, :], axis=2)                # [Nr, Nt]
    ref = (C0 / (4 * np.pi * f[:, None, None] * d0[None, :, None])) * \
        np.exp(-2j * np.pi * f[:, None, None] * dist[None] / C0)
    assert np.abs(H - ref).max() < 1e-12 * np.abs(ref).max()


def test_per_element_with_one_element_at_the_reference_equals_reference_synthesis():
    # a single receive element at the receiver reference point: the per-element form and
    # the reference-point form (zero receive-side correction) coincide
    sc = _small_mimo(nr=1)
    sc["rx_elem"] = sc["rx"][:1].copy()
    r = oracle.run(sc)
    p, g = r["paths"], r["g"]
    sel = p["rx"] == 0
    assert sel.sum() >= 3
    H_ref = oracle.synth_H(p, g, sc["freqs"], sc["tx"], sc["rx"][0], sc["tx_elem"], sc["rx_elem"])
    sub = {k: v[sel] for k, v in p.items() if isinstance(v, np.ndarray) and len(v) == len(sel)}
    H_el = oracle.synth_H_elements(sub, g[sel], sc["freqs"], sc["tx"], sc["tx_elem"], sc["rx_elem"])
    # (phases of ~1e3-1e4 cycles: agreement to the rounding of the path length)
    assert np.abs(H_el - H_ref).max() <= 1e-11 * np.abs(H_ref).max()
