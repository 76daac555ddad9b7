"""The surrogate's CUDA kernels through the C ABI: the tcgen05 MLP forward,
gradients and Adam step against the CPU reference (tests/mlp_ref.py, itself
pinned to torch autograd), convergence on a smooth function, and the
per-receiver targets against numpy over the same path list."""
import numpy as np
import pytest

import mlp_ref
import scenes
from parity import to_numpy

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

LO, HI = [-20.0, -20.0, 0.0, 280e9], [500.0, 320.0, 10.0, 320e9]


@pytest.fixture(scope="module")
def sbr():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2208_10006_gb300 import build as b
    b.build()
    import paper_2208_10006_gb300 as m
    return m


def _inputs(B, n_out, seed):
    rng = np.random.default_rng(seed)
    x = np.column_stack([rng.uniform(LO[k], HI[k], B) for k in range(4)]).astype(np.float32)
    y = rng.normal(size=(B, n_out)).astype(np.float32) * 3.0 + 1.0
    y[rng.uniform(size=(B, n_out)) < 0.1] = np.nan
    return x, y


SHIFT = np.array([1.0, -0.5, 0.0, 2.0, 0.0, 0.0], np.float32)
SCALE = np.array([2.0, 1.0, 3.0, 0.5, 1.0, 2.0], np.float32)
LOSS_W = np.array([1.0, 0.5, 2.0, 1.0, 1.0, 0.3], np.float32)


@pytest.mark.parametrize("depth,width,B", [(2, 256, 300), (4, 256, 1024), (1, 128, 130)])
def test_forward_gradients_and_adam_match_reference(sbr, depth, width, B):
    n_out = 6
    m = sbr.MLP(n_out, LO, HI, width=width, depth=depth, max_batch=B, seed=7, lr=1e-3, err_channel=5,
                err_of=0, loss_w=LOSS_W, y_shift=SHIFT, y_scale=SCALE)
    x, y = _inputs(B, n_out, depth)
    xd, yd = torch.tensor(x, device="cuda"), torch.tensor(y, device="cuda")
    p0 = m.params(0).cpu().numpy()
    layers = mlp_ref.unpack(p0, width, depth)
    feat = mlp_ref.features(x, LO, HI)
    hs, p = mlp_ref.forward(layers, feat)
    # forward, in target units: the fused kernel, and the per-layer GEMMs bit for bit
    got = m.predict(xd).cpu().numpy()
    want = p[:, :n_out] * SCALE + SHIFT
    err = np.abs(got - want).max() / np.abs(want).max()
    assert err < 1e-2, err
    assert np.array_equal(got, m.predict(xd, layered=True).cpu().numpy())
    # one training step: loss, gradients, Adam update
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    m.train_step(xd, yd, loss)
    m.status()
    shift = np.zeros(mlp_ref.OUT_W)
    shift[:n_out] = SHIFT
    scale = np.ones(mlp_ref.OUT_W)
    scale[:n_out] = SCALE
    w = np.zeros(mlp_ref.OUT_W)
    w[:n_out] = LOSS_W
    L, g = mlp_ref.loss_grad(p, y.astype(np.float64), w, shift, scale, 5, 0)
    assert abs(loss.item() - L) <= 1e-2 * L
    ref = mlp_ref.backward(layers, hs, g)
    grads = m.params(2).cpu().numpy()
    o = 0
    worst = []
    for li, (dW, db) in enumerate(ref):
        for name, r in (("W", dW.ravel()), ("b", db)):
            gg = grads[o:o + r.size].astype(np.float64)
            o += r.size
            nrm = np.linalg.norm(r)
            if nrm == 0:
                assert np.abs(gg).max() == 0
                continue
            # per tensor, element by element: every entry within 5% of the
            # tensor's largest entry (BF16 operands carry 2^-9 relative each,
            # and a ReLU whose input rounds across zero moves a whole row), and
            # the tensor as a whole within 2% in norm
            e_max = np.abs(gg - r).max() / np.abs(r).max()
            e_nrm = np.linalg.norm(gg - r) / nrm
            worst.append((li, name, e_max, e_nrm))
            assert e_max <= 5e-2, (li, name, e_max)
            assert e_nrm <= 2e-2, (li, name, e_nrm)
    print("gradient errors per tensor (layer, W/b, max|dg|/max|g|, |dg|/|g|):", worst)
    assert o == len(grads)
    # Adam, first step: m = (1 - b1) g, v = (1 - b2) g^2, bias-corrected
    gg = grads.astype(np.float32)
    mh = ((1 - 0.9) * gg) / np.float32(1 - 0.9)
    vh = ((1 - 0.999) * gg * gg) / np.float32(1 - 0.999)
    want_p = p0 - 1e-3 * mh / (np.sqrt(vh) + 1e-8)
    assert np.abs(m.params(0).cpu().numpy() - want_p).max() <= 1e-6


def test_training_fits_a_smooth_function(sbr):
    rng = np.random.default_rng(3)
    n = 8192
    x = np.column_stack([rng.uniform(LO[k], HI[k], n) for k in range(4)]).astype(np.float32)
    u = (x - np.array(LO, np.float32)) / (np.array(HI, np.float32) - np.array(LO, np.float32))
    y = np.column_stack([np.sin(2 * np.pi * u[:, 0]) + np.cos(np.pi * u[:, 1]) * u[:, 2],
                         u[:, 3] ** 2 - u[:, 0] * u[:, 1]]).astype(np.float32)
    m = sbr.MLP(2, LO, HI, width=256, depth=4, max_batch=1024, seed=1, lr=2e-3)
    xd, yd = torch.tensor(x, device="cuda"), torch.tensor(y, device="cuda")
    losses = []
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    for step in range(400):
        i = (step % 8) * 1024
        loss.zero_()
        m.train_step(xd[i:i + 1024], yd[i:i + 1024], loss)
        losses.append(loss.item())
    m.status()
    assert np.mean(losses[-8:]) < 0.05 * np.mean(losses[:8]), (losses[:8], losses[-8:])


def test_surrogate_targets_match_numpy(sbr):
    sc = scenes.config2(N=60, K=3, nx=2, ny=2, sub=3, ground_sub=6, rx_grid=6)
    sc["freqs"] = np.array([290e9, 300e9, 310e9])
    sc["gamma_db_km"] = np.full(3, 5.0, np.float32)
    sc["disp_deg_km"] = np.zeros(3, np.float32)
    r = sbr.run_scene(sc)
    ex = to_numpy(r["export"])
    g = r["g"].cpu().numpy().astype(np.complex128)
    F, n_taps, tap_s, floor_db = 3, 16, 5e-9, -40.0
    t = sbr.surrogate_targets(r["paths"], r["g"], F, n_taps, tap_s, floor_db).cpu().numpy()
    assert t.shape == (len(sc["rx"]), F, 2 + n_taps)
    c0 = 299792458.0
    n_cov = 0
    for q in range(len(sc["rx"])):
        sel = np.where(ex["rx"] == q)[0]
        if len(sel) == 0:
            assert np.isnan(t[q]).all()
            continue
        n_cov += 1
        tau = ex["L"][sel] / c0
        tau = tau - tau.min()
        for f in range(F):
            pw = np.abs(g[sel, f]) ** 2
            s = pw.sum()
            assert abs(t[q, f, 0] + 10 * np.log10(s)) <= 1e-4
            mean = (pw * tau).sum() / s
            rms = np.sqrt(max((pw * tau * tau).sum() / s - mean ** 2, 0.0))
            assert abs(t[q, f, 1] - rms) <= 1e-6 * max(rms, 1e-12) + 1e-15
            b = np.floor(tau / tap_s)
            for k in range(n_taps):
                tk = pw[b == k].sum()
                want = max(10 * np.log10(tk / s), floor_db) if tk > 0 else floor_db
                assert abs(t[q, f, 2 + k] - want) <= 1e-3
    assert n_cov >= 3


def test_mlp_rejects_bad_configs(sbr):
    for kw in (dict(width=100), dict(depth=0), dict(err_channel=1, err_of=1), dict(err_channel=2, err_of=-1),
               dict(lr=0.0)):
        args = dict(width=256, depth=2, max_batch=128)
        args.update(kw)
        with pytest.raises(sbr.SbrError) as e:
            sbr.MLP(4, LO, HI, **args)
        assert e.value.status == 1
    with pytest.raises(sbr.SbrError):
        sbr.MLP(4, LO, HI, y_scale=[1.0, 0.0, 1.0, 1.0])
