"""Plain FP64 CPU oracle for the SBR hot path (arXiv 2208.10006).

TEST INFRASTRUCTURE ONLY: tests/, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of bench.py may import this package; the product library
never does. The arithmetic lives in ``oracle.c`` (plain C, FP64, brute force);
this module compiles it with gcc, loads it with ctypes and marshals numpy
arrays. It shares no code with the CUDA path; only the seeded scene
generators in ``scenes`` serve both.

Pipeline (paper section / equation, see ``oracle.c`` for the readings):
  geodesic_dirs / alpha   Sec. II-A.1       trace        Sec. II-A.2-3
  dedup                   Sec. II-A.2       refine       image method, Sec. I
  gains                   Eq. 1, 3, 6-10    synth_H      Eq. 11-14
  pdp_stats               Eq. 2, 4, 5       capacity     Eq. 15-17

Parity unpinned: the alpha definition, which candidate a duplicate key keeps,
the capacity normalisation reading and the arithmetic-mean angles.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
KMAX = 8
C0 = 299792458.0

CAND_DTYPE = np.dtype([("rx", "<i4"), ("nb", "<i4"), ("seq", "<i4", (KMAX,)), ("ray", "<i8"),
                       ("dist", "<f8"), ("flags", "<i4"), ("pad", "<i4")])
assert CAND_DTYPE.itemsize == 64

FLAG_NEAR_EDGE, FLAG_T_TIE, FLAG_RADIUS, FLAG_TSTAR, FLAG_GRAZING = 1, 2, 4, 8, 16


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so beside it (gcc, -O2, no fast-math)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-pthread",
                               "-fno-fast-math", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB)
        p = C.c_void_p
        i32, i64, f64 = C.c_int32, C.c_int64, C.c_double
        L.orc_geodesic_count.restype = i64
        L.orc_geodesic_count.argtypes = [i32]
        L.orc_geodesic_dirs.restype = i64
        L.orc_geodesic_dirs.argtypes = [i32, p]
        L.orc_geodesic_alpha.restype = f64
        L.orc_geodesic_alpha.argtypes = [i32]
        L.orc_trace.restype = i64
        L.orc_trace.argtypes = [p, p, i64, i32, p, p, i32, i32, i32, f64, i64, i64, f64, i32,
                                C.POINTER(p), p, p]
        L.orc_trace_one.restype = i32
        L.orc_trace_one.argtypes = [p, p, i64, i32, p, i32, i32, i64, p, p, p, p, p]
        L.orc_free.argtypes = [p]
        L.orc_dedup.restype = i64
        L.orc_dedup.argtypes = [p, i64, p, p, p]
        L.orc_refine.restype = i64
        L.orc_refine.argtypes = [p, p, i64, i32, p, p, p, i64, p, p, p, p, p, p]
        L.orc_fresnel.argtypes = [f64, f64, f64, f64, p, p, p, p]
        L.orc_roughness.restype = f64
        L.orc_roughness.argtypes = [f64, f64, f64]
        L.orc_gains.restype = i32
        L.orc_gains.argtypes = [p, p, i64, i32, p, p, p, i64, p, p, p, p, p, p, i32, p, p, i32, p]
        L.orc_synth_H.restype = i32
        L.orc_synth_H.argtypes = [i64, p, p, p, p, p, i32, p, p, p, i32, p, i32, i32, p]
        L.orc_synth_H_elements.restype = i32
        L.orc_synth_H_elements.argtypes = [i64, p, p, p, p, p, p, i32, p, p, i32, p, i32, p]
        L.orc_pdp_stats.restype = i32
        L.orc_pdp_stats.argtypes = [i64, p, p, p, p, f64, f64, i32, p, p]
        L.orc_capacity.restype = i32
        L.orc_capacity.argtypes = [p, i32, i32, i32, p, i32, p]
        _lib = L
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def nthreads_default() -> int:
    return max(1, len(os.sched_getaffinity(0)))


# ---------------------------------------------------------------- O1
def geodesic_count(N: int) -> int:
    return int(lib().orc_geodesic_count(N))


def geodesic_dirs(N: int) -> np.ndarray:
    R = geodesic_count(N)
    out = np.empty((R, 3), np.float64)
    n = lib().orc_geodesic_dirs(N, _ptr(out))
    if n != R:
        raise ValueError("bad subdivision N=%r" % N)
    return out


def alpha(N: int) -> float:
    return float(lib().orc_geodesic_alpha(N))


# ---------------------------------------------------------------- scene marshalling
def _scene_args(sc):
    tri = _c(sc["tri"], np.float32).reshape(-1, 9)
    sid = _c(sc["surface_id"], np.int32)
    S = int(len(sc["materials"]))
    return tri, sid, len(sid), S


# ---------------------------------------------------------------- O2
def trace(sc, N=None, K=None, alpha_=None, ray_begin=0, ray_end=None, eps=1e-6,
          nthreads=None, rx=None):
    """Trace rays [ray_begin, ray_end). Returns (candidates, ray_flags, counters)."""
    N = sc["N"] if N is None else N
    K = sc["K"] if K is None else K
    R = geodesic_count(N)
    ray_end = R if ray_end is None else ray_end
    tri, sid, T, S = _scene_args(sc)
    tx = _c(sc["tx"], np.float64)
    rxa = _c(sc["rx"] if rx is None else rx, np.float64).reshape(-1, 3)
    flags = np.zeros(max(ray_end - ray_begin, 1), np.uint8)
    cnt = np.zeros(3, np.int64)
    out = C.c_void_p()
    n = lib().orc_trace(_ptr(tri), _ptr(sid), T, S, _ptr(tx), _ptr(rxa), len(rxa), N, K,
                        0.0 if alpha_ is None else float(alpha_), ray_begin, ray_end, eps,
                        nthreads or nthreads_default(), C.byref(out), _ptr(flags), _ptr(cnt))
    if n < 0:
        raise RuntimeError("orc_trace failed: %d" % n)
    cands = np.empty(n, CAND_DTYPE)
    if n:
        C.memmove(cands.ctypes.data, out.value, n * CAND_DTYPE.itemsize)
    lib().orc_free(out)
    counters = dict(rays=int(cnt[0]), segments=int(cnt[1]), flagged_rays=int(cnt[2]))
    return cands, flags[: ray_end - ray_begin], counters


def trace_one(sc, ray: int, N=None, K=None):
    """Per-segment record of one ray: origins, directions, hit faces, t_hit, L."""
    N = sc["N"] if N is None else N
    K = sc["K"] if K is None else K
    tri, sid, T, S = _scene_args(sc)
    tx = _c(sc["tx"], np.float64)
    o = np.zeros((K + 1, 3)); d = np.zeros((K + 1, 3))
    fc = np.full(K + 1, -1, np.int64); t = np.full(K + 1, np.inf); Ls = np.zeros(K + 1)
    ns = lib().orc_trace_one(_ptr(tri), _ptr(sid), T, S, _ptr(tx), N, K, int(ray), _ptr(o),
                             _ptr(d), _ptr(fc), _ptr(t), _ptr(Ls))
    if ns < 0:
        raise ValueError("orc_trace_one failed")
    return dict(o=o[:ns], d=d[:ns], face=fc[:ns], t=t[:ns], L=Ls[:ns])


# ---------------------------------------------------------------- O3
def dedup(cands: np.ndarray):
    """Returns (keys, n_producers, all_flagged); keys sorted by (rx, nb, seq)."""
    c = np.ascontiguousarray(cands.copy())
    n = len(c)
    keys = np.empty(max(n, 1), CAND_DTYPE)
    nprod = np.zeros(max(n, 1), np.int64)
    allf = np.zeros(max(n, 1), np.int32)
    nk = lib().orc_dedup(_ptr(c), n, _ptr(keys), _ptr(nprod), _ptr(allf))
    return keys[:nk], nprod[:nk], allf[:nk].astype(bool)


# ---------------------------------------------------------------- O4
def refine(sc, keys: np.ndarray):
    tri, sid, T, S = _scene_args(sc)
    n = len(keys)
    k = np.ascontiguousarray(keys)
    valid = np.zeros(max(n, 1), np.int32)
    face = np.full((max(n, 1), KMAX), -1, np.int32)
    pts = np.zeros((max(n, 1), KMAX, 3))
    L = np.zeros(max(n, 1)); aod = np.zeros((max(n, 1), 2)); aoa = np.zeros((max(n, 1), 2))
    lib().orc_refine(_ptr(tri), _ptr(sid), T, S, _ptr(_c(sc["tx"], np.float64)),
                     _ptr(_c(sc["rx"], np.float64)), _ptr(k), n, _ptr(valid), _ptr(face),
                     _ptr(pts), _ptr(L), _ptr(aod), _ptr(aoa))
    return dict(valid=valid[:n].astype(bool), face=face[:n], pts=pts[:n], L=L[:n],
                aod=aod[:n], aoa=aoa[:n])


def fresnel(eps_r, sigma, f, cos_i):
    a = np.zeros(4)
    vals = [C.c_double() for _ in range(4)]
    lib().orc_fresnel(eps_r, sigma, f, cos_i, *[C.byref(v) for v in vals])
    return complex(vals[0].value, vals[1].value), complex(vals[2].value, vals[3].value)


def roughness(rough_m, f, cos_i):
    return float(lib().orc_roughness(rough_m, f, cos_i))


# ---------------------------------------------------------------- O5/O6
def gains(sc, paths: dict, freqs=None, gamma=None, disp=None, pol=None):
    """g[P, F] complex128 for the paths dict produced by `run`/`paths_of`."""
    tri, sid, T, S = _scene_args(sc)
    freqs = _c(sc["freqs"] if freqs is None else freqs, np.float64)
    F = len(freqs)
    gamma = _c(sc["gamma_db_km"] if gamma is None else gamma, np.float64)
    disp = _c(sc["disp_deg_km"] if disp is None else disp, np.float64)
    pol = sc["pol"] if pol is None else pol
    P = len(paths["rx"])
    g = np.zeros((max(P, 1), F), np.complex128)
    rc = lib().orc_gains(_ptr(tri), _ptr(sid), T, S, _ptr(_c(sc["materials"], np.float64)),
                         _ptr(_c(sc["tx"], np.float64)), _ptr(_c(sc["rx"], np.float64)), P,
                         _ptr(_c(paths["rx"], np.int32)), _ptr(_c(paths["nb"], np.int32)),
                         _ptr(_c(paths["seq"], np.int32)), _ptr(_c(paths["pts"], np.float64)),
                         _ptr(_c(paths["L"], np.float64)), _ptr(freqs), F, _ptr(gamma),
                         _ptr(disp), 0 if pol == "V" else 1, _ptr(g))
    if rc != 0:
        raise RuntimeError("orc_gains failed")
    return g[:P]


# ---------------------------------------------------------------- O7
def synth_H(paths: dict, g: np.ndarray, freqs, tx_ref, rx_ref, tx_elem, rx_elem,
            rx_index: int = 0, nthreads=None):
    sel = np.nonzero(np.asarray(paths["rx"]) == rx_index)[0]
    freqs = _c(freqs, np.float64)
    F = len(freqs)
    txe = _c(tx_elem, np.float64).reshape(-1, 3)
    rxe = _c(rx_elem, np.float64).reshape(-1, 3)
    H = np.zeros((F, len(rxe), len(txe)), np.complex128)
    gg = _c(g[sel], np.complex128)
    lib().orc_synth_H(len(sel), _ptr(_c(paths["nb"][sel], np.int32)),
                      _ptr(_c(paths["pts"][sel], np.float64)), _ptr(_c(paths["L"][sel], np.float64)),
                      _ptr(gg), _ptr(freqs), F, _ptr(_c(tx_ref, np.float64)),
                      _ptr(_c(rx_ref, np.float64)), _ptr(txe), len(txe), _ptr(rxe), len(rxe),
                      nthreads or nthreads_default(), _ptr(H))
    return H


def synth_H_elements(paths: dict, g: np.ndarray, freqs, tx_ref, tx_elem, rx_elem):
    """Per-element reception: paths of every receive element (paths["rx"] is the
    element index), H [F, Nr, Nt] complex128, each row from its element's own paths."""
    freqs = _c(freqs, np.float64)
    F = len(freqs)
    txe = _c(tx_elem, np.float64).reshape(-1, 3)
    rxe = _c(rx_elem, np.float64).reshape(-1, 3)
    H = np.zeros((F, len(rxe), len(txe)), np.complex128)
    P = len(paths["L"])
    rc = lib().orc_synth_H_elements(P, _ptr(_c(paths["rx"], np.int32)), _ptr(_c(paths["nb"], np.int32)),
                                    _ptr(_c(paths["pts"], np.float64)), _ptr(_c(paths["L"], np.float64)),
                                    _ptr(_c(g, np.complex128)), _ptr(freqs), F, _ptr(_c(tx_ref, np.float64)),
                                    _ptr(txe), len(txe), _ptr(rxe), len(rxe), _ptr(H))
    if rc != 0:
        raise ValueError("path receiver index out of range")
    return H


# ---------------------------------------------------------------- O8
def pdp_stats(paths: dict, g: np.ndarray, f_index: int, fc: float, bin_s: float, n_bins: int,
              n_rx: int):
    pdp = np.full((n_rx, n_bins), -np.inf)
    stats = np.zeros((n_rx, 7))
    for r in range(n_rx):
        sel = np.nonzero(np.asarray(paths["rx"]) == r)[0]
        gc = _c(g[sel, f_index], np.complex128)
        row = np.zeros(n_bins); st = np.zeros(7)
        lib().orc_pdp_stats(len(sel), _ptr(_c(paths["L"][sel], np.float64)), _ptr(gc),
                            _ptr(_c(paths["aod"][sel], np.float64)),
                            _ptr(_c(paths["aoa"][sel], np.float64)), fc, bin_s, n_bins,
                            _ptr(row), _ptr(st))
        pdp[r] = row
        stats[r] = st
    return pdp, stats


# ---------------------------------------------------------------- O9
def capacity(H: np.ndarray, snr_db) -> np.ndarray:
    H = _c(H, np.complex128)
    F, Nr, Nt = H.shape
    snr = _c(snr_db, np.float64)
    out = np.zeros(len(snr))
    rc = lib().orc_capacity(_ptr(H), F, Nr, Nt, _ptr(snr), len(snr), _ptr(out))
    if rc != 0:
        raise RuntimeError("orc_capacity failed")
    return out


# ---------------------------------------------------------------- whole pipeline
def paths_of(sc, keys: np.ndarray, ref: dict, nprod=None, allf=None):
    """Valid refined paths as a dict of arrays (sorted by rx, nb, seq)."""
    v = ref["valid"]
    out = dict(rx=keys["rx"][v].astype(np.int32), nb=keys["nb"][v].astype(np.int32),
               seq=keys["seq"][v].astype(np.int32), face=ref["face"][v], pts=ref["pts"][v],
               L=ref["L"][v], aod=ref["aod"][v], aoa=ref["aoa"][v],
               ray=keys["ray"][v], dist=keys["dist"][v])
    if nprod is not None:
        out["n_prod"] = nprod[v]
    if allf is not None:
        out["all_flagged"] = allf[v]
    return out


def run(sc, N=None, K=None, eps=1e-6, nthreads=None, ray_begin=0, ray_end=None):
    """Trace + dedup + refine + gains for a scene. Returns a dict."""
    cands, flags, cnt = trace(sc, N=N, K=K, eps=eps, nthreads=nthreads, ray_begin=ray_begin,
                              ray_end=ray_end)
    keys, nprod, allf = dedup(cands)
    ref = refine(sc, keys)
    paths = paths_of(sc, keys, ref, nprod, allf)
    g = gains(sc, paths)
    return dict(cands=cands, flags=flags, counters=cnt, keys=keys, n_prod=nprod,
                all_flagged=allf, refine=ref, paths=paths, g=g,
                n_invalid=int((~ref["valid"]).sum()))
