"""CPU reference of the surrogate MLP (test infrastructure): the network of
sbr_mlp_create written out in numpy, forward and backward, with optional BF16
rounding at the points where the CUDA path stores BF16 (features, weights,
hidden activations, output and hidden gradients). Accumulation in float64.
"""
from __future__ import annotations

import numpy as np

N_OCT = 16
N_FEAT = 128
OUT_W = 128


def bf16(a):
    """Round float32 values to the nearest bfloat16 (ties to even), as float32."""
    a = np.ascontiguousarray(a, dtype=np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return (r & 0xFFFFFFFF).astype(np.uint32).view(np.float32)


def features(x, lo, hi, rnd=True, lmax=9.0):
    """[B, 4] -> [B, 128]: coordinate c, octave k: sin, cos of pi 2^(k lmax/15) u_c."""
    x = np.asarray(x, np.float32)
    lo = np.asarray(lo, np.float32)
    inv = (np.float32(1.0) / (np.asarray(hi, np.float32) - lo)).astype(np.float32)
    u = ((x - lo) * inv).astype(np.float32)
    B = len(x)
    f = np.zeros((B, N_FEAT), np.float32)
    for c in range(4):
        for k in range(N_OCT):
            w = np.exp2(np.float32(np.float32(lmax) * np.float32(k) / np.float32(15.0))).astype(np.float32)
            arg = (w * u[:, c]).astype(np.float64)
            f[:, c * 2 * N_OCT + 2 * k] = np.sin(np.pi * arg)
            f[:, c * 2 * N_OCT + 2 * k + 1] = np.cos(np.pi * arg)
    return bf16(f) if rnd else f


def unpack(params, width, depth):
    """Flat parameter vector -> [(W [n_out, n_in], b [n_out])] per layer."""
    widths = [N_FEAT] + [width] * depth + [OUT_W]
    layers, o = [], 0
    for l in range(len(widths) - 1):
        n_in, n_out = widths[l], widths[l + 1]
        W = params[o:o + n_in * n_out].reshape(n_out, n_in)
        o += n_in * n_out
        b = params[o:o + n_out]
        o += n_out
        layers.append((W.astype(np.float64), b.astype(np.float64)))
    assert o == len(params)
    return layers


def forward(layers, feat, rnd=True):
    """Hidden activations (list, the input first) and outputs [B, 128]."""
    def wr(W):   # the weights as the GEMM sees them
        return np.asarray(bf16(W.astype(np.float32)), np.float64) if rnd else W

    hs = [np.asarray(feat, np.float64)]
    for W, b in layers[:-1]:
        h = np.maximum(hs[-1] @ wr(W).T + b, 0.0)
        hs.append(np.asarray(bf16(h.astype(np.float32)), np.float64) if rnd else h)
    W, b = layers[-1]
    p = hs[-1] @ wr(W).T + b
    return hs, p


def loss_grad(p, y, w, shift, scale, e_ch=-1, e_of=-1):
    """Loss and dL/dp of the sbr_mlp_train_step objective (p normalised, y in units)."""
    B, n_out = y.shape
    g = np.zeros_like(p)
    L = 0.0
    yn = (y - shift[:n_out]) / scale[:n_out]
    for o in range(n_out):
        if o == e_ch and e_of >= 0:
            ok = np.isfinite(yn[:, e_of])
            t = np.abs(p[:, e_of] - yn[:, e_of])
            d = np.where(ok, p[:, o] - np.where(ok, t, 0.0), 0.0)
        else:
            ok = np.isfinite(yn[:, o])
            d = np.where(ok, p[:, o] - np.where(ok, yn[:, o], 0.0), 0.0)
        L += w[o] * np.sum(d * d) / B
        g[:, o] = 2.0 * w[o] * d / B
    return L, g


def backward(layers, hs, g_out, rnd=True):
    """Gradients [(dW, db)] per layer for dL/dp = g_out."""
    def r(a):    # a gradient or weight as stored for the GEMMs
        return np.asarray(bf16(a.astype(np.float32)), np.float64) if rnd else a

    grads = [None] * len(layers)
    d = r(g_out)
    for l in range(len(layers) - 1, -1, -1):
        W, _ = layers[l]
        grads[l] = (d.T @ hs[l], d.sum(axis=0))
        if l > 0:
            d = r(np.where(hs[l] > 0, d @ r(W), 0.0))
    return grads
