"""Helpers that compare the CUDA path with the FP64 oracle (test infrastructure).

Path-set rule: the sets of (rx, surface sequence) of valid paths must be
equal, except for keys produced only by rays the oracle flags as
edge-ambiguous (within 1e-6 relative of a triangle edge, of a t tie between
surfaces, of the reception-sphere boundary or of a segment end). Every such
exemption is counted and returned. On common keys the face sequences must be
identical, lengths agree within 1e-9 relative, gains within 1e-4 relative.
"""
from __future__ import annotations

import numpy as np

L_RTOL = 1e-9
G_RTOL = 1e-4


def keymap(rx, nb, seq):
    return {(int(rx[i]), tuple(int(x) for x in seq[i][: nb[i]])): i for i in range(len(rx))}


def compare_paths(gpu: dict, g_gpu: np.ndarray, orc: dict, L_rtol=L_RTOL, g_rtol=G_RTOL):
    """gpu: exported path arrays (numpy); orc: oracle.run(...) result."""
    op = orc["paths"]
    gk = keymap(gpu["rx"], gpu["nb"], gpu["seq"])
    ok = keymap(op["rx"], op["nb"], op["seq"])
    only_gpu = sorted(set(gk) - set(ok))
    only_orc = sorted(set(ok) - set(gk))
    flags = orc["flags"]
    bad = []
    exempt = 0
    for k in only_orc:
        if op["all_flagged"][ok[k]]:
            exempt += 1
        else:
            bad.append(("missing on GPU", k))
    for k in only_gpu:
        ray = int(gpu["ray"][gk[k]]) & 0xffffffff
        if ray < len(flags) and flags[ray]:
            exempt += 1
        else:
            bad.append(("extra on GPU", k, ray))
    common = sorted(set(gk) & set(ok))
    face_bad = L_err = pts_err = ang_err = g_err = 0.0
    n_face_bad = 0
    for k in common:
        i, j = gk[k], ok[k]
        m = int(gpu["nb"][i])
        if not np.array_equal(gpu["face"][i][:m], op["face"][j][:m]):
            n_face_bad += 1
        L_err = max(L_err, abs(gpu["L"][i] - op["L"][j]) / op["L"][j])
        if m:
            pts_err = max(pts_err, float(np.abs(gpu["pts"][i][:m] - op["pts"][j][:m]).max()))
        da = np.abs(np.concatenate([gpu["aod"][i] - op["aod"][j], gpu["aoa"][i] - op["aoa"][j]]))
        da = np.minimum(da, 360.0 - da)
        ang_err = max(ang_err, float(da.max()))
        if g_gpu is not None:
            ref = orc["g"][j]
            g_err = max(g_err, float(np.max(np.abs(g_gpu[i] - ref) / np.maximum(np.abs(ref), 1e-300))))
    return dict(n_gpu=len(gk), n_orc=len(ok), n_common=len(common), only_gpu=only_gpu,
                only_orc=only_orc, exempt=exempt, bad=bad, n_face_bad=n_face_bad, L_err=L_err,
                pts_err=pts_err, ang_err=ang_err, g_err=g_err)


def assert_parity(rep: dict, L_rtol=L_RTOL, g_rtol=G_RTOL):
    assert not rep["bad"], rep["bad"][:10]
    assert rep["n_face_bad"] == 0, rep
    assert rep["L_err"] <= L_rtol, rep
    assert rep["pts_err"] <= 1e-7, rep
    assert rep["ang_err"] <= 1e-7, rep
    assert rep["g_err"] <= g_rtol, rep


def to_numpy(export: dict) -> dict:
    out = {k: v.cpu().numpy() for k, v in export.items()}
    out["ray"] = out["ray"].astype(np.int64) & 0xffffffff
    return out
