"""Learned surrogate workflow: SBR-traced training data on a scene, the BF16
MLP of sbr_mlp_create, and its evaluation against full SBR with fallback.

Every number here comes from the library's kernels: the trace, paths and
gains of a receiver set (Sec. II-A, Eq. 1, 3, 6-10), the per-receiver targets
(sbr_surrogate_targets: path loss, RMS delay spread and a 16-tap PDP, Eq. 2,
4, 5), and the MLP's training and inference. This module only moves tensors
between those calls and computes the evaluation statistics.

Outputs of the network (target units):
  0        path loss (dB, incoherent sum)
  1        RMS delay spread (ns)
  2 .. 17  PDP taps relative to the total power (dB, 5 ns taps from the first
           arrival, floor -40 dB)
  18       coverage (1 when the receiver has a path loss of at most
           PL_MAX_DB, else 0)
  19       error head: the expected |path-loss error| (dB)
A receiver out of coverage has no path-loss, delay or tap target. At 300 GHz
the Kirchhoff factor of a rough facade removes tens of dB per reflection, so
receivers reached only by high-order paths sit at 200-500 dB: far below any
link budget, and read here as out of coverage.
"""
from __future__ import annotations

import time

import numpy as np
import torch

from . import MLP, POL_H, POL_V, build_bvh, path_gains, paths, scene_to_device, surrogate_targets, trace

N_TAPS, TAP_S, FLOOR_DB = 16, 5e-9, -40.0
CH_PL, CH_TAU, CH_TAP0, CH_COV, CH_ERR = 0, 1, 2, 18, 19
N_OUT = 20
PL_MAX_DB = 200.0
# highest Fourier-feature octave (log2 of the top frequency per unit of the
# input box): held-out sweeps on the urban scene chose 2.5 at 8.4M training
# samples (2.0 at 1M; finer features overfit)
FEAT_LOG2_MAX = 2.5
SHIFT = np.array([120.0, 20.0] + [-20.0] * N_TAPS + [0.0, 0.0], np.float32)
SCALE = np.array([20.0, 20.0] + [20.0] * N_TAPS + [1.0, 20.0], np.float32)
LOSS_W = np.array([1.0, 0.5] + [0.25] * N_TAPS + [1.0, 0.5], np.float32)


def sample_receivers(sc: dict, n: int, seed: int, z_range=(1.0, 5.0)) -> np.ndarray:
    """n receiver points uniform over the ground rectangle of an urban-grid scene
    (outside every building footprint) with z uniform in z_range."""
    rng = np.random.default_rng(seed)
    tri = sc["tri"].reshape(-1, 9)
    sid = sc["surface_id"]
    g = tri[sid == 0].reshape(-1, 3, 3)
    lo, hi = g.reshape(-1, 3).min(0), g.reshape(-1, 3).max(0)
    # building footprints from the roofs (the z+ face of each building: surfaces 5, 10, ...)
    boxes = []
    for s in range(5, int(sid.max()) + 1, 5):
        v = tri[sid == s].reshape(-1, 3)
        boxes.append((v[:, 0].min(), v[:, 0].max(), v[:, 1].min(), v[:, 1].max()))
    out = np.zeros((0, 3))
    while len(out) < n:
        m = 2 * (n - len(out)) + 16
        p = np.column_stack([rng.uniform(lo[0], hi[0], m), rng.uniform(lo[1], hi[1], m),
                             rng.uniform(z_range[0], z_range[1], m)])
        ok = np.ones(m, bool)
        for (x0, x1, y0, y1) in boxes:
            ok &= ~((p[:, 0] >= x0) & (p[:, 0] <= x1) & (p[:, 1] >= y0) & (p[:, 1] <= y1))
        out = np.concatenate([out, p[ok]])
    return out[:n]


def sbr_targets(sc: dict, rx: np.ndarray, freqs: np.ndarray, alpha: float = 0.0, chunk: int = 16384,
                dev=None, bvh=None):
    """Full SBR at every receiver: [n, F, 2 + N_TAPS] targets (float32, CUDA),
    chunk receivers per trace. Returns (targets, seconds of GPU time)."""
    d = dev if dev is not None else scene_to_device(sc)
    if bvh is None:
        bvh = build_bvh(d["tri"], d["surface_id"], d["S"])
    fr = torch.as_tensor(np.asarray(freqs, np.float64), device="cuda")
    gam = torch.as_tensor(np.interp(freqs, sc["freqs"], sc["gamma_db_km"]).astype(np.float32), device="cuda") \
        if len(sc["freqs"]) > 1 else torch.full((len(freqs),), float(sc["gamma_db_km"][0]), device="cuda")
    pol = POL_V if sc.get("pol", "V") == "V" else POL_H
    out = torch.empty((len(rx), len(freqs), 2 + N_TAPS), dtype=torch.float32, device="cuda")
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    lg = 0
    for c0 in range(0, len(rx), chunk):
        r = torch.as_tensor(np.ascontiguousarray(rx[c0:c0 + chunk], np.float64), device="cuda")
        for _ in range(4):
            tr = trace(bvh, d["tx"], r, d["N"], d["K"], alpha=alpha, table_log2=lg)
            st = tr.stats(check=False)
            if st["status"] != 3:
                break
            lg = st["table_log2"] + 1
        pl = paths(tr, bvh)
        g = path_gains(pl, d["mats"], fr, gam, None, pol) if pl.n else None
        out[c0:c0 + len(r)] = surrogate_targets(pl, g, len(freqs), N_TAPS, TAP_S, FLOOR_DB)
    e1.record()
    e1.synchronize()
    return out, e0.elapsed_time(e1) / 1e3


def make_xy(rx: np.ndarray, freqs: np.ndarray, t: torch.Tensor, pl_max_db: float = PL_MAX_DB):
    """Inputs [n F, 4] (x, y, z, f) and targets [n F, N_OUT] from sbr_targets."""
    n, F = len(rx), len(freqs)
    X = np.empty((n, F, 4), np.float32)
    X[:, :, :3] = rx[:, None, :]
    X[:, :, 3] = np.asarray(freqs)[None, :]
    cov = torch.isfinite(t[:, :, 0]) & (t[:, :, 0] <= pl_max_db)
    Y = torch.full((n, F, N_OUT), float("nan"), dtype=torch.float32, device="cuda")
    Y[:, :, :2 + N_TAPS] = torch.where(cov[:, :, None], t, torch.full_like(t, float("nan")))
    Y[:, :, CH_TAU] *= 1e9
    Y[:, :, CH_COV] = cov.float()
    return torch.as_tensor(X.reshape(-1, 4), device="cuda"), Y.reshape(-1, N_OUT)


def x_box(sc: dict, freqs) -> tuple:
    v = sc["tri"].reshape(-1, 3)
    lo = [float(v[:, 0].min()), float(v[:, 1].min()), 0.0, float(np.min(freqs))]
    hi = [float(v[:, 0].max()), float(v[:, 1].max()), 10.0, float(np.max(freqs))]
    if hi[3] <= lo[3]:
        hi[3] = lo[3] + 1.0
    return lo, hi


def train(X: torch.Tensor, Y: torch.Tensor, lo, hi, epochs: int = 20, batch: int = 8192, lr: float = 2e-3,
          seed: int = 5, width: int = 256, depth: int = 4, lr_min: float = 5e-5,
          feat_log2_max: float = FEAT_LOG2_MAX):
    """Adam on shuffled batches, learning rate on a cosine from lr to lr_min
    over the epochs; returns (model, per-epoch mean loss, seconds)."""
    m = MLP(N_OUT, lo, hi, width=width, depth=depth, max_batch=batch, seed=seed, lr=lr,
            err_channel=CH_ERR, err_of=CH_PL, loss_w=LOSS_W, y_shift=SHIFT, y_scale=SCALE,
            feat_log2_max=feat_log2_max)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(seed)
    n = X.shape[0]
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    hist = []
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for ep in range(epochs):
        m.set_lr(lr_min + 0.5 * (lr - lr_min) * (1.0 + np.cos(np.pi * ep / max(epochs, 1))))
        perm = torch.randperm(n, device="cuda", generator=gen)
        loss.zero_()
        steps = 0
        for i in range(0, n - batch + 1, batch):
            idx = perm[i:i + batch]
            m.train_step(X[idx].contiguous(), Y[idx].contiguous(), loss)
            steps += 1
        hist.append(loss.item() / max(steps, 1))
    torch.cuda.synchronize()
    m.status()
    return m, hist, time.perf_counter() - t0


def predict(m: MLP, X: torch.Tensor, batch: int = 8192) -> torch.Tensor:
    out = torch.empty((X.shape[0], N_OUT), dtype=torch.float32, device="cuda")
    for i in range(0, X.shape[0], batch):
        m.predict(X[i:i + batch].contiguous(), out=out[i:i + batch])
    return out


def evaluate(m: MLP, X: torch.Tensor, Y: torch.Tensor, threshold_db: float = 3.0,
             thresholds=(3.0, 6.0, 10.0)) -> dict:
    """Errors against full SBR on (X, Y), and the effect of the fallback rule:
    a query goes to full SBR when the error head predicts more than the
    threshold of path-loss error or the coverage output is in (0.2, 0.8); per
    threshold, the fraction of queries that fall back, the path-loss RMSE of
    the served ones and the RMSE over all (fallback answers exact)."""
    P = predict(m, X)
    cov = Y[:, CH_COV] > 0.5
    pc = P[:, CH_COV]
    e_pl = (P[:, CH_PL] - Y[:, CH_PL])[cov]
    e_tau = (P[:, CH_TAU] - Y[:, CH_TAU])[cov]
    e_tap = (P[:, CH_TAP0:CH_TAP0 + N_TAPS] - Y[:, CH_TAP0:CH_TAP0 + N_TAPS])[cov]
    rms = lambda e: float(torch.sqrt((e.double() ** 2).mean())) if e.numel() else float("nan")
    cov_ok = ((pc > 0.5) == cov).float().mean()
    out = dict(n=int(X.shape[0]), covered=float(cov.float().mean()),
               pl_rmse_db=rms(e_pl), tau_rmse_ns=rms(e_tau), taps_rmse_db=rms(e_tap),
               coverage_accuracy=float(cov_ok), fallback={})
    for th in sorted(set(thresholds) | {threshold_db}):
        fb = (P[:, CH_ERR] > th) | ((pc > 0.2) & (pc < 0.8))
        kept = ~fb[cov]
        out["fallback"]["%g_dB" % th] = dict(
            fraction=float(fb.float().mean()), pl_rmse_db_served=rms(e_pl[kept]),
            pl_rmse_db_with_fallback=rms(torch.where(kept, e_pl, torch.zeros_like(e_pl))))
    return out
