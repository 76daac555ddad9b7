"""Exhaustive image-method path enumeration for tiny scenes (test helper).

An independent route to the exact specular path set: every surface sequence
up to K reflections (no surface twice in a row) is mirrored, back-traced and
kept if every reflection point lies on its surface and no segment is
blocked. It shares no code with the oracle or the CUDA path and exists only
to pin the SBR oracle's path set (image method, Sec. I of the paper).
"""
from __future__ import annotations

import itertools
import numpy as np


def _planes(tri, sid, S):
    planes = []
    for s in range(S):
        idx = np.nonzero(sid == s)[0]
        t = tri[idx[0]]
        n = np.cross(t[1] - t[0], t[2] - t[0])
        n = n / np.linalg.norm(n)
        planes.append((n, float(n @ t[0]), idx))
    return planes


def _inside(tris, p, tol=1e-9):
    """Barycentric containment of p (on the plane) in any of tris [k,3,3]."""
    a, b, c = tris[:, 0], tris[:, 1], tris[:, 2]
    v0, v1, v2 = b - a, c - a, p[None, :] - a
    d00 = np.einsum("ij,ij->i", v0, v0)
    d01 = np.einsum("ij,ij->i", v0, v1)
    d11 = np.einsum("ij,ij->i", v1, v1)
    d20 = np.einsum("ij,ij->i", v2, v0)
    d21 = np.einsum("ij,ij->i", v2, v1)
    den = d00 * d11 - d01 * d01
    l1 = (d11 * d20 - d01 * d21) / den
    l2 = (d00 * d21 - d01 * d20) / den
    l0 = 1 - l1 - l2
    return np.nonzero((l0 >= -tol) & (l1 >= -tol) & (l2 >= -tol))[0]


def _blocked(tri, allowed_mask, p, q, tol=1e-9):
    """True if the open segment p->q crosses any triangle not in allowed_mask."""
    d = q - p
    e1 = tri[:, 1] - tri[:, 0]
    e2 = tri[:, 2] - tri[:, 0]
    h = np.cross(d[None, :], e2)
    det = np.einsum("ij,ij->i", e1, h)
    ok = np.abs(det) > 1e-300
    inv = np.where(ok, 1.0 / np.where(ok, det, 1.0), 0.0)
    s = p[None, :] - tri[:, 0]
    u = np.einsum("ij,ij->i", s, h) * inv
    qv = np.cross(s, e1)
    v = np.einsum("ij,j->i", qv, d) * inv
    t = np.einsum("ij,ij->i", e2, qv) * inv
    hit = ok & (u >= 0) & (v >= 0) & (u + v <= 1) & (t > tol) & (t < 1 - tol) & ~allowed_mask
    return bool(hit.any())


def enumerate_paths(sc, K=None, rx_index=0):
    """Returns {seq tuple: dict(L, pts)} of the valid, unblocked specular paths."""
    tri = sc["tri"].astype(np.float64)
    sid = sc["surface_id"]
    S = len(sc["materials"])
    K = sc["K"] if K is None else K
    tx = np.asarray(sc["tx"], float)
    rx = np.asarray(sc["rx"][rx_index], float)
    planes = _planes(tri, sid, S)
    out = {}
    for m in range(K + 1):
        for seq in itertools.product(range(S), repeat=m):
            if any(seq[i] == seq[i + 1] for i in range(m - 1)):
                continue
            imgs = [tx]
            for s in seq:
                n, c, _ = planes[s]
                imgs.append(imgs[-1] - 2 * (n @ imgs[-1] - c) * n)
            pts = [None] * m
            target = rx
            ok = True
            for i in range(m, 0, -1):
                n, c, idx = planes[seq[i - 1]]
                dv = target - imgs[i]
                den = n @ dv
                if den == 0:
                    ok = False
                    break
                u = (c - n @ imgs[i]) / den
                if not (0 < u < 1):
                    ok = False
                    break
                p = imgs[i] + u * dv
                if len(_inside(tri[idx], p)) == 0:
                    ok = False
                    break
                pts[i - 1] = p
                target = p
            if not ok:
                continue
            chain = [tx] + pts + [rx]
            surf_at = [None] + list(seq) + [None]
            for i in range(len(chain) - 1):
                allowed = np.zeros(len(tri), bool)
                for s in (surf_at[i], surf_at[i + 1]):
                    if s is not None:
                        allowed |= sid == s
                if _blocked(tri, allowed, chain[i], chain[i + 1]):
                    ok = False
                    break
            if ok:
                out[tuple(seq)] = dict(L=float(np.linalg.norm(imgs[-1] - rx)),
                                       pts=np.array(pts).reshape(m, 3))
    return out
