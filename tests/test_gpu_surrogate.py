"""The surrogate workflow end to end at test size: SBR-traced targets of a
receiver set on the urban grid (the library's trace, paths, gains and target
kernels), training of the tcgen05 MLP on them, and evaluation against full
SBR on held-out receivers."""
import numpy as np
import pytest

import scenes

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


def test_surrogate_workflow_learns_path_loss(sbr):
    from paper_2208_10006_gb300 import surrogate as S
    sc = scenes.config2(N=200, K=4, nx=3, ny=3, sub=4, ground_sub=8, rx_grid=1)
    freqs = np.linspace(290e9, 310e9, 4)
    rx = S.sample_receivers(sc, 6000, seed=5)
    rx_t = S.sample_receivers(sc, 500, seed=6)
    t, _ = S.sbr_targets(sc, rx, freqs, chunk=4096)
    tt, _ = S.sbr_targets(sc, rx_t, freqs, chunk=4096)
    X, Y = S.make_xy(rx, freqs, t)
    Xt, Yt = S.make_xy(rx_t, freqs, tt)
    assert X.shape == (24000, 4) and Y.shape == (24000, S.N_OUT)
    cov = float((Y[:, S.CH_COV] > 0.5).float().mean())
    assert 0.2 < cov <= 1.0
    lo, hi = S.x_box(sc, freqs)
    # a small training set: the coarser feature bandwidth of the 1M-sample sweeps
    m, hist, _ = S.train(X, Y, lo, hi, epochs=30, batch=2048, feat_log2_max=2.0)
    assert hist[-1] < 0.5 * hist[0], hist
    ev = S.evaluate(m, Xt, Yt)
    print(ev)
    # a trained model beats the constant predictor of the held-out path loss by a wide margin
    pl = Yt[Yt[:, S.CH_COV] > 0.5, S.CH_PL]
    assert ev["pl_rmse_db"] < 0.6 * float(pl.std())
    assert ev["coverage_accuracy"] > 0.8
    fb = ev["fallback"]["3_dB"]
    assert 0.0 <= fb["fraction"] <= 1.0
    assert fb["pl_rmse_db_with_fallback"] <= ev["pl_rmse_db"]
    # a looser threshold serves more queries
    assert ev["fallback"]["10_dB"]["fraction"] <= fb["fraction"]
