"""The CPU reference of the surrogate MLP (tests/mlp_ref.py) against torch
autograd in float64 (no BF16 rounding): forward, loss and every gradient,
including the error head's stop-gradient; and the BF16 rounding helper
against torch's bfloat16 conversion."""
import numpy as np
import pytest

import mlp_ref

torch = pytest.importorskip("torch")


def test_bf16_rounding_matches_torch():
    rng = np.random.default_rng(0)
    a = (rng.normal(size=10000) * 10.0 ** rng.uniform(-6, 6, 10000)).astype(np.float32)
    a[:4] = [0.0, -0.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8]   # ties to even
    want = torch.tensor(a).to(torch.bfloat16).to(torch.float32).numpy()
    assert np.array_equal(mlp_ref.bf16(a), want)


@pytest.mark.parametrize("depth,width", [(1, 128), (3, 256)])
def test_reference_backprop_equals_autograd(depth, width):
    rng = np.random.default_rng(depth)
    B, n_out = 37, 6
    widths = [mlp_ref.N_FEAT] + [width] * depth + [mlp_ref.OUT_W]
    params = np.concatenate([np.concatenate([rng.normal(size=widths[l] * widths[l + 1]) / np.sqrt(widths[l]),
                                             rng.normal(size=widths[l + 1]) * 0.1])
                             for l in range(len(widths) - 1)])
    layers = mlp_ref.unpack(params, width, depth)
    x = rng.uniform(0, 1, (B, 4))
    feat = mlp_ref.features(x, [0] * 4, [1] * 4, rnd=False).astype(np.float64)
    y = rng.normal(size=(B, n_out))
    y[3, 1] = np.nan
    y[5, 0] = np.nan
    w = np.array([1.0, 0.5, 2.0, 1.0, 1.0, 0.3])
    shift = np.zeros(mlp_ref.OUT_W)
    shift[:n_out] = rng.normal(size=n_out)
    scale = np.ones(mlp_ref.OUT_W)
    scale[:n_out] = rng.uniform(0.5, 2.0, n_out)
    e_ch, e_of = 5, 0
    hs, p = mlp_ref.forward(layers, feat, rnd=False)
    L, g = mlp_ref.loss_grad(p, y, w, shift, scale, e_ch, e_of)
    grads = mlp_ref.backward(layers, hs, g, rnd=False)
    # autograd
    tl = [(torch.tensor(W, requires_grad=True), torch.tensor(b, requires_grad=True)) for W, b in layers]
    h = torch.tensor(feat)
    for W, b in tl[:-1]:
        h = torch.relu(h @ W.T + b)
    pt = h @ tl[-1][0].T + tl[-1][1]
    yt = (torch.tensor(y) - torch.tensor(shift[:n_out])) / torch.tensor(scale[:n_out])
    loss = torch.zeros((), dtype=torch.float64)
    for o in range(n_out):
        if o == e_ch:
            ok = torch.isfinite(yt[:, e_of])
            tgt = (pt[:, e_of].detach() - yt[:, e_of]).abs()
            d = pt[:, o][ok] - tgt[ok]
        else:
            ok = torch.isfinite(yt[:, o])
            d = pt[:, o][ok] - yt[:, o][ok]
        loss = loss + w[o] * (d * d).sum() / B
    loss.backward()
    assert abs(L - loss.item()) <= 1e-12 * max(1.0, abs(L))
    for (dW, db), (W, b) in zip(grads, tl):
        assert np.allclose(dW, W.grad.numpy(), rtol=1e-10, atol=1e-14)
        assert np.allclose(db, b.grad.numpy(), rtol=1e-10, atol=1e-14)
