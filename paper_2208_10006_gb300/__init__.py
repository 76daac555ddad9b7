"""GB300-native SBR channel modelling (arXiv 2208.10006): Python binding.

Every call marshals arguments to the C ABI of libsbr.so (include/sbr.h);
every step of the path runs in the library's CUDA kernels. PyTorch provides
device memory and the current stream only. There is no CPU fallback: the
functions raise if the library is missing or no CUDA device is present.

Pipeline (paper section / equation):
    build_bvh                       scene acceleration structure (Sec. III-C)
    trace                           Sec. II-A.1 launch, II-A.2 trace, II-A.3 reception, dedup
    paths                           effective paths, image-method refinement (Sec. I)
    path_gains                      Eq. 1, 3, 6-10
    synthesize_H                    Eq. 11-14, near-field wavefront
    pdp_angles                      Eq. 2, 4, 5
    capacity                        Eq. 15-17
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import _lib
from ._lib import (KMAX, NSTATS, POL_H, POL_V, SYNTH_BF16X3, SYNTH_FP16X3, SYNTH_FP32, SYNTH_FP64,
                   STATUS_NAMES)

__all__ = ["SbrError", "BVH", "TraceResult", "PathList", "launch_dirs", "build_bvh", "trace",
           "paths", "path_gains", "synthesize_H", "synthesize_H_elements", "pdp_angles", "capacity", "version",
           "POL_V", "POL_H", "SYNTH_FP64", "SYNTH_FP32", "SYNTH_BF16X3", "SYNTH_FP16X3", "KMAX", "NSTATS",
           "scene_to_device", "run_scene", "Batch", "batch_create", "batch_tune", "surrogate_targets", "MLP"]


class SbrError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, str(status)), msg))
        self.status = status


def _L():
    return _lib.load()


def _check(st: int):
    if st != 0:
        raise SbrError(st, _L().sbr_last_error().decode(errors="replace"))


def _stream(stream=None):
    s = torch.cuda.current_stream() if stream is None else stream
    return C.c_void_p(s.cuda_stream)


def _ptr(t):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return C.c_void_p(t.data_ptr())


def _ptr_or_pinned(t):
    """A CUDA tensor or a pinned host tensor (copy destinations)."""
    if t is not None and not t.is_cuda:
        if not t.is_pinned() or not t.is_contiguous():
            raise ValueError("expected a CUDA tensor or a contiguous pinned host tensor")
        return C.c_void_p(t.data_ptr())
    return _ptr(t)


def _dev():
    if not torch.cuda.is_available():
        raise RuntimeError("no CUDA device: the SBR library has no CPU path")
    return torch.device("cuda", torch.cuda.current_device())


def version() -> str:
    return _L().sbr_version().decode()


def launch_count() -> int:
    """Kernels launched by the library so far in this process."""
    return int(_L().sbr_launch_count())


def launch_dirs(N: int, with_alpha: bool = True, with_dirs: bool = True, stream=None):
    """Geodesic launch directions [R, 3] (float64) and alpha (Sec. II-A.1)."""
    dev = _dev()
    R = 10 * N * N + 2
    d = torch.empty((R, 3), dtype=torch.float64, device=dev) if with_dirs else None
    a = torch.empty(1, dtype=torch.float64, device=dev) if with_alpha else None
    _check(_L().sbr_launch_dirs(N, _ptr(d), _ptr(a), _stream(stream)))
    return d, a


class BVH:
    def __init__(self, handle, T, S):
        self._h = handle
        self.T, self.S = T, S

    @property
    def handle(self):
        return self._h

    def info(self) -> dict:
        i = _lib.BvhInfo()
        _check(_L().sbr_bvh_query(self._h, C.byref(i)))
        return dict(T=i.T, S=i.S, n_nodes=i.n_nodes, depth=i.depth)

    def free(self):
        if self._h is not None:
            _L().sbr_bvh_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def build_bvh(tri: torch.Tensor, surface_id: torch.Tensor, S: int, sah_top: bool = False,
              stream=None) -> BVH:
    """tri: float32 [T,3,3] (or [T,9]); surface_id: int32 [T]; both CUDA.
    sah_top: rebuild the top levels with the surface-area heuristic (slower
    build, faster traversal: for scenes traced many times)."""
    T = int(surface_id.numel())
    tri = tri.reshape(T, 9) if T else tri
    if T:
        assert tri.dtype == torch.float32 and surface_id.dtype == torch.int32
    h = C.c_void_p()
    _check(_L().sbr_build_bvh_ex(_ptr(tri) if T else None, _ptr(surface_id) if T else None, T, int(S),
                                 _lib.BVH_SAH_TOP if sah_top else 0, C.byref(h), _stream(stream)))
    return BVH(h, T, int(S))


class TraceResult:
    def __init__(self, handle, params):
        self._h = handle
        self.params = params

    @property
    def handle(self):
        return self._h

    def stats(self, check: bool = True) -> dict:
        c = _lib.TraceCounters()
        st = _L().sbr_trace_stats(self._h, C.byref(c))
        if check:
            _check(st)
        return dict(rays=c.rays, ray_bounces=c.ray_bounces, candidates=c.candidates, keys=c.keys,
                    fp64_segments=c.fp64_segments, fp64_tests=c.fp64_tests,
                    node_visits=c.node_visits, tri_tests=c.tri_tests, rx_visits=c.rx_visits,
                    near_edge_hits=c.near_edge_hits,
                    queue=list(c.queue), alpha=c.alpha,
                    status=c.status, table_log2=c.table_log2, bounce_ms=list(c.bounce_ms))

    def entries(self, stream=None):
        """The deduplicated receptions as records (sbr_trace_entries): keys
        int32 [n, 10] (receiver, reflections, 8 surface ids, -1 padded) and
        vals int64 [n] (FP32 distance bits << 32 | ray id), CUDA tensors."""
        n = C.c_int64(0)
        st = _L().sbr_trace_entries(self._h, None, None, 0, C.byref(n), _stream(stream))
        if st not in (0, 3):
            _check(st)
        keys = torch.empty((max(n.value, 1), 10), dtype=torch.int32, device=_dev())
        vals = torch.empty(max(n.value, 1), dtype=torch.int64, device=_dev())
        _check(_L().sbr_trace_entries(self._h, _ptr(keys), _ptr(vals), n.value, C.byref(n), _stream(stream)))
        return keys[:n.value], vals[:n.value]

    def free(self):
        if self._h is not None:
            _L().sbr_trace_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def _trace_params(tx, rx, N, K, alpha, table_log2):
    p = _lib.TraceParams()
    for k in range(3):
        p.tx[k] = float(tx[k])
    n_rx = int(rx.shape[0]) if rx is not None else 0
    p.rx_xyz = rx.data_ptr() if n_rx else None
    if n_rx:
        assert rx.dtype == torch.float64 and rx.is_cuda and rx.is_contiguous()
    p.n_rx = n_rx
    p.subdiv_N = int(N)
    p.max_bounces = int(K)
    p.table_log2 = int(table_log2)
    p.alpha = float(alpha)
    return p


def trace_merge(tx, rx: torch.Tensor, N: int, K: int, keys: torch.Tensor, vals: torch.Tensor, alpha: float = 0.0,
                table_log2: int = 0, stream=None) -> TraceResult:
    """A trace result from the records of traces of disjoint ray ranges
    (sbr_trace_merge); sbr_paths on it gives the path list of the union."""
    p = _trace_params(tx, rx, N, K, alpha, table_log2)
    keys = keys.contiguous()
    vals = vals.contiguous()
    assert keys.dtype == torch.int32 and vals.dtype == torch.int64 and keys.shape[0] == vals.shape[0]
    h = C.c_void_p()
    _check(_L().sbr_trace_merge(C.byref(p), _ptr(keys), _ptr(vals), int(vals.shape[0]), C.byref(h),
                                _stream(stream)))
    return TraceResult(h, p)


def trace(bvh: BVH, tx, rx: torch.Tensor, N: int, K: int, alpha: float = 0.0, table_log2: int = 0,
          timing: bool = False, count_visits: bool = False, depth_first_from: int = 0,
          ray_range=None, stream=None) -> TraceResult:
    """Shoot and bounce. tx: 3 floats; rx: float64 [n_rx, 3] CUDA. Bounces from
    depth_first_from on are traced depth first (K + 1: all breadth first).
    ray_range = (begin, end): trace only those geodesic ids (end 0 = all)."""
    p = _trace_params(tx, rx, N, K, alpha, table_log2)
    if ray_range is not None:
        p.ray_begin, p.ray_end = int(ray_range[0]), int(ray_range[1])
    p.flags = (_lib.TRACE_TIMING if timing else 0) | (_lib.TRACE_COUNT_VISITS if count_visits else 0)
    p.depth_first_from = int(depth_first_from)
    h = C.c_void_p()
    _check(_L().sbr_trace(bvh.handle, C.byref(p), C.byref(h), _stream(stream)))
    return TraceResult(h, p)


class PathList:
    def __init__(self, handle, n, n_rx):
        self._h = handle
        self.n = n          # paths
        self.n_rx = n_rx    # receivers of the trace (known without a query, which waits for the stream)

    @property
    def handle(self):
        return self._h

    def info(self) -> dict:
        i = _lib.PathInfo()
        _check(_L().sbr_path_query(self._h, C.byref(i)))
        return dict(n_paths=i.n_paths, n_keys=i.n_keys, n_invalid=i.n_invalid, n_rx=i.n_rx,
                    max_bounces=i.max_bounces, status=i.status)

    def export(self, stream=None, out: dict = None) -> dict:
        """The path list as tensors; `out` may hold preallocated CUDA or pinned
        host tensors of the same shapes (then the copies land there directly)."""
        dev = _dev()
        P = self.n
        if out is not None:
            o = out
            _check(_L().sbr_path_export(self._h, *[_ptr_or_pinned(o[k]) for k in
                                                   ("rx", "nb", "seq", "face", "pts", "L", "aod", "aoa", "ray",
                                                    "dist")], _stream(stream)))
            return out
        out = dict(
            rx=torch.empty(P, dtype=torch.int32, device=dev),
            nb=torch.empty(P, dtype=torch.int32, device=dev),
            seq=torch.empty((P, KMAX), dtype=torch.int32, device=dev),
            face=torch.empty((P, KMAX), dtype=torch.int32, device=dev),
            pts=torch.empty((P, KMAX, 3), dtype=torch.float64, device=dev),
            L=torch.empty(P, dtype=torch.float64, device=dev),
            aod=torch.empty((P, 2), dtype=torch.float64, device=dev),
            aoa=torch.empty((P, 2), dtype=torch.float64, device=dev),
            ray=torch.empty(P, dtype=torch.int32, device=dev),
            dist=torch.empty(P, dtype=torch.float32, device=dev),
        )
        o = out
        _check(_L().sbr_path_export(self._h, _ptr(o["rx"]), _ptr(o["nb"]), _ptr(o["seq"]),
                                    _ptr(o["face"]), _ptr(o["pts"]), _ptr(o["L"]), _ptr(o["aod"]),
                                    _ptr(o["aoa"]), _ptr(o["ray"]), _ptr(o["dist"]),
                                    _stream(stream)))
        return out

    def free(self):
        if self._h is not None:
            _L().sbr_path_list_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def paths(tr: TraceResult, bvh: BVH, stream=None) -> PathList:
    h = C.c_void_p()
    n = C.c_int64()
    _check(_L().sbr_paths(tr.handle, bvh.handle, C.byref(h), C.byref(n), _stream(stream)))
    return PathList(h, int(n.value), int(tr.params.n_rx))


def path_gains(pl: PathList, mats: torch.Tensor, freqs: torch.Tensor, gamma_db_km=None,
               disp_deg_km=None, pol: int = POL_V, out=None, stream=None) -> torch.Tensor:
    """Complex path gains [P, F] (complex64). mats: float64 [S, 3] CUDA."""
    F = int(freqs.numel())
    g = out if out is not None else torch.empty((pl.n, F), dtype=torch.complex64, device=_dev())
    _check(_L().sbr_path_gains(pl.handle, _ptr(mats), int(mats.shape[0]), _ptr(freqs), F,
                               _ptr(gamma_db_km), _ptr(disp_deg_km), int(pol), _ptr(g),
                               _stream(stream)))
    return g


def synthesize_H(pl: PathList, gains: torch.Tensor, freqs: torch.Tensor, tx_elem: torch.Tensor,
                 rx_elem: torch.Tensor, rx_index: int = 0, precision: int = SYNTH_FP32, out=None,
                 stream=None) -> torch.Tensor:
    """H(f) [F, Nr, Nt] complex64 for receiver rx_index (Eq. 13-14)."""
    F, Nt, Nr = int(freqs.numel()), int(tx_elem.shape[0]), int(rx_elem.shape[0])
    H = out if out is not None else torch.empty((F, Nr, Nt), dtype=torch.complex64, device=_dev())
    g = gains if gains.numel() else torch.empty(1, dtype=torch.complex64, device=_dev())
    _check(_L().sbr_synthesize_H(pl.handle, _ptr(g), _ptr(freqs), F, _ptr(tx_elem), Nt,
                                 _ptr(rx_elem), Nr, int(rx_index), int(precision), _ptr(H),
                                 _stream(stream)))
    return H


def synthesize_H_elements(pl: PathList, gains: torch.Tensor, freqs: torch.Tensor, tx_elem: torch.Tensor,
                          precision: int = SYNTH_FP32, out=None, stream=None) -> torch.Tensor:
    """H(f) [F, n_rx, Nt] complex64 with per-element reception: every receiver
    of the trace is one receive element and its row sums its own paths."""
    F, Nt, Nr = int(freqs.numel()), int(tx_elem.shape[0]), pl.n_rx
    H = out if out is not None else torch.empty((F, Nr, Nt), dtype=torch.complex64, device=_dev())
    g = gains if gains.numel() else torch.empty(1, dtype=torch.complex64, device=_dev())
    _check(_L().sbr_synthesize_H_elements(pl.handle, _ptr(g), _ptr(freqs), F, _ptr(tx_elem), Nt,
                                          int(precision), _ptr(H), _stream(stream)))
    return H


def pdp_angles(pl: PathList, gains: torch.Tensor, f_index: int, fc_hz: float, bin_s: float = 1e-9,
               n_bins: int = 1024, stream=None, out=None):
    """PDP in dB [n_rx, n_bins] (float32) and stats [n_rx, 7] (float64). `out`
    may be a (pdp, stats) pair of preallocated CUDA or pinned host tensors of
    shapes [max(n_rx, 1), n_bins] and [max(n_rx, 1), 7]: the kernel then writes
    them directly (pinned host memory is device-accessible under unified
    addressing), complete once the stream has passed the call."""
    n_rx = pl.n_rx
    F = int(gains.shape[1]) if gains.dim() == 2 else 1
    if out is None:
        pdp = torch.empty((max(n_rx, 1), n_bins), dtype=torch.float32, device=_dev())
        stats = torch.empty((max(n_rx, 1), NSTATS), dtype=torch.float64, device=_dev())
    else:
        pdp, stats = out
        if (tuple(pdp.shape) != (max(n_rx, 1), n_bins) or pdp.dtype != torch.float32 or
                tuple(stats.shape) != (max(n_rx, 1), NSTATS) or stats.dtype != torch.float64):
            raise ValueError("out: float32 [max(n_rx, 1), n_bins] and float64 [max(n_rx, 1), %d]" % NSTATS)
    g = gains if gains.numel() else torch.empty(1, dtype=torch.complex64, device=_dev())
    _check(_L().sbr_pdp_angles(pl.handle, _ptr(g), F, int(f_index), float(fc_hz), float(bin_s),
                               int(n_bins), _ptr_or_pinned(pdp), _ptr_or_pinned(stats), _stream(stream)))
    return pdp[:n_rx], stats[:n_rx]


def capacity(H: torch.Tensor, snr_db, stream=None) -> torch.Tensor:
    """Mean capacity over frequency (bit/s/Hz) per SNR (Eq. 15-17)."""
    F, Nr, Nt = H.shape
    snr = np.ascontiguousarray(np.asarray(snr_db, dtype=np.float64))
    C_out = torch.empty(len(snr), dtype=torch.float64, device=_dev())
    _check(_L().sbr_capacity(_ptr(H), F, Nr, Nt, snr.ctypes.data_as(C.c_void_p), len(snr),
                             _ptr(C_out), _stream(stream)))
    return C_out


# ---------------------------------------------------------------- convenience
def scene_to_device(sc: dict) -> dict:
    """Move a scene dict of numpy arrays (see the `scenes` module) to the GPU."""
    dev = _dev()
    t = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device=dev)
    return dict(
        tri=t(sc["tri"].reshape(-1, 9), torch.float32),
        surface_id=t(sc["surface_id"], torch.int32),
        S=int(len(sc["materials"])),
        mats=t(sc["materials"].reshape(-1, 3), torch.float64),
        rx=t(sc["rx"].reshape(-1, 3), torch.float64),
        freqs=t(sc["freqs"], torch.float64),
        gamma=t(sc["gamma_db_km"], torch.float32),
        disp=t(sc["disp_deg_km"], torch.float32),
        tx_elem=t(sc["tx_elem"].reshape(-1, 3), torch.float64),
        rx_elem=t(sc["rx_elem"].reshape(-1, 3), torch.float64),
        tx=[float(x) for x in sc["tx"]], N=int(sc["N"]), K=int(sc["K"]),
        pol=POL_V if sc.get("pol", "V") == "V" else POL_H,
    )


def run_scene(sc: dict, alpha: float = 0.0, table_log2: int = 0, stream=None):
    """build_bvh + trace + paths + gains for a scene dict. Returns a dict."""
    d = scene_to_device(sc)
    bvh = build_bvh(d["tri"], d["surface_id"], d["S"], stream=stream)
    lg = table_log2
    for _ in range(3):
        tr = trace(bvh, d["tx"], d["rx"], d["N"], d["K"], alpha=alpha, table_log2=lg, stream=stream)
        st = tr.stats(check=False)
        if st["status"] != 3:  # SBR_ERR_CAPACITY: retry with a larger table
            break
        lg = st["table_log2"] + 2
    _check(st["status"])
    pl = paths(tr, bvh, stream=stream)
    g = path_gains(pl, d["mats"], d["freqs"], d["gamma"], d["disp"], d["pol"], stream=stream)
    return dict(dev=d, bvh=bvh, trace=tr, stats=st, paths=pl, export=pl.export(stream=stream), g=g)


# ---------------------------------------------------------------- batched jobs
class Batch:
    """Handle of sbr_batch_create: many Tx-Rx jobs over several scenes."""

    def __init__(self, handle, jobs, keep):
        self._h = handle
        self.jobs = jobs
        self._keep = keep   # device tensors the batch reads (scenes' materials, job inputs, H)

    @property
    def handle(self):
        return self._h

    def run(self, stream=None):
        _check(_L().sbr_batch_run(self._h, _stream(stream)))

    def query(self):
        """(paths per job, sbr_status per job, summary dict); synchronous."""
        n = len(self.jobs)
        np_ = np.zeros(n, np.int32)
        st = np.zeros(n, np.int32)
        info = _lib.BatchInfo()
        _L().sbr_batch_query(self._h, np_.ctypes.data_as(C.c_void_p), st.ctypes.data_as(C.c_void_p),
                             C.byref(info))
        c = info.config
        summary = dict(n_jobs=info.n_jobs, n_waves=info.n_waves, graph_kernels=info.graph_kernels,
                       status=info.status, max_keys=info.max_keys, rays=info.rays,
                       ray_bounces=info.ray_bounces, paths=info.paths,
                       config=dict(wave_rays=c.wave_rays, path_cap=c.path_cap, table_log2=c.table_log2,
                                   tile_n=c.tile_n, trace_blocks_per_sm=c.trace_blocks_per_sm,
                                   precision=c.precision, use_graph=c.use_graph,
                                   breadth_first=c.breadth_first))
        return np_, st, summary

    def export(self, job: int, n: int, stream=None) -> dict:
        """First n paths of a job (n <= its path count) and their gains [n, F]."""
        dev = _dev()
        K = KMAX
        F = int(self.jobs[job]["F"])
        out = dict(nb=torch.empty(n, dtype=torch.int32, device=dev),
                   seq=torch.empty((n, K), dtype=torch.int32, device=dev),
                   face=torch.empty((n, K), dtype=torch.int32, device=dev),
                   pts=torch.empty((n, K, 3), dtype=torch.float64, device=dev),
                   L=torch.empty(n, dtype=torch.float64, device=dev),
                   aod=torch.empty((n, 2), dtype=torch.float64, device=dev),
                   aoa=torch.empty((n, 2), dtype=torch.float64, device=dev),
                   ray=torch.empty(n, dtype=torch.int32, device=dev),
                   dist=torch.empty(n, dtype=torch.float32, device=dev),
                   g=torch.empty((n, F), dtype=torch.complex64, device=dev))
        _check(_L().sbr_batch_export(self._h, int(job), int(n), _ptr(out["nb"]), _ptr(out["seq"]),
                                     _ptr(out["face"]), _ptr(out["pts"]), _ptr(out["L"]), _ptr(out["aod"]),
                                     _ptr(out["aoa"]), _ptr(out["ray"]),
                                     _ptr(out["dist"]), _ptr(out["g"]), _stream(stream)))
        return out

    def free(self):
        if self._h:
            _L().sbr_batch_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def _batch_args(scenes, jobs):
    """ctypes arrays for a list of (BVH, materials tensor) scenes and job dicts.

    Job keys: scene, N, K, tx, rx, freqs (float64 CUDA [F]), tx_elem / rx_elem
    (float64 CUDA [n, 3]); optional: pol, alpha, gamma / disp (float32 CUDA [F]),
    H (complex64 CUDA [F, Nr, Nt], allocated when absent)."""
    dev = _dev()
    ns = len(scenes)
    sc_arr = (C.c_void_p * ns)(*[s[0].handle.value for s in scenes])
    mat_arr = (C.c_void_p * ns)(*[s[1].data_ptr() for s in scenes])
    keep = [s[1] for s in scenes]
    jarr = (_lib.BatchJob * len(jobs))()
    for i, j in enumerate(jobs):
        F, Nt, Nr = int(j["freqs"].shape[0]), int(j["tx_elem"].shape[0]), int(j["rx_elem"].shape[0])
        for key in ("freqs", "tx_elem", "rx_elem"):
            assert j[key].is_cuda and j[key].dtype == torch.float64 and j[key].is_contiguous(), key
        if j.get("H") is None:
            j["H"] = torch.empty((F, Nr, Nt), dtype=torch.complex64, device=dev)
        j["F"] = F
        b = jarr[i]
        b.scene = int(j["scene"])
        b.subdiv_N = int(j["N"])
        b.max_bounces = int(j["K"])
        b.pol = POL_V if j.get("pol", "V") in ("V", POL_V) else POL_H
        for k in range(3):
            b.tx[k] = float(j["tx"][k])
            b.rx[k] = float(j["rx"][k])
        b.alpha = float(j.get("alpha", 0.0))
        b.F, b.Nt, b.Nr = F, Nt, Nr
        b.freqs_hz = j["freqs"].data_ptr()
        b.gamma_db_km = j["gamma"].data_ptr() if j.get("gamma") is not None else None
        b.disp_deg_km = j["disp"].data_ptr() if j.get("disp") is not None else None
        b.tx_elem = j["tx_elem"].data_ptr()
        b.rx_elem = j["rx_elem"].data_ptr()
        b.H = j["H"].data_ptr()
        keep += [j[k] for k in ("freqs", "tx_elem", "rx_elem", "H", "gamma", "disp") if j.get(k) is not None]
    return sc_arr, mat_arr, jarr, keep


def _batch_config(config):
    c = _lib.BatchConfig()
    c.use_graph = 1
    for k, v in (config or {}).items():
        setattr(c, k, int(v))
    return c


def batch_create(scenes, jobs, config=None, stream=None) -> Batch:
    """sbr_batch_create. scenes: list of (BVH, materials float64 CUDA [S, 3])."""
    sc_arr, mat_arr, jarr, keep = _batch_args(scenes, jobs)
    c = _batch_config(config)
    h = C.c_void_p()
    _check(_L().sbr_batch_create(sc_arr, mat_arr, len(scenes), jarr, len(jobs), C.byref(c), C.byref(h),
                                 _stream(stream)))
    return Batch(h, jobs, keep + [s[0] for s in scenes])


def batch_tune(scenes, jobs, config=None, stream=None):
    """sbr_batch_tune on these jobs; returns (config dict, ms per run)."""
    sc_arr, mat_arr, jarr, keep = _batch_args(scenes, jobs)
    c = _batch_config(config)
    ms = C.c_double()
    _check(_L().sbr_batch_tune(sc_arr, mat_arr, len(scenes), jarr, len(jobs), C.byref(c), C.byref(ms),
                               _stream(stream)))
    del keep
    return dict(wave_rays=c.wave_rays, path_cap=c.path_cap, table_log2=c.table_log2, tile_n=c.tile_n,
                trace_blocks_per_sm=c.trace_blocks_per_sm, precision=c.precision,
                use_graph=c.use_graph, breadth_first=c.breadth_first), ms.value


# ---------------------------------------------------------------- surrogate
def surrogate_targets(pl: PathList, gains: torch.Tensor, F: int, n_taps: int = 16, tap_s: float = 5e-9,
                      floor_db: float = -40.0, stream=None) -> torch.Tensor:
    """[n_rx, F, 2 + n_taps] float32: path loss (dB), RMS delay spread (s), PDP taps (dB)."""
    n_rx = pl.n_rx
    out = torch.empty((max(n_rx, 1), F, 2 + n_taps), dtype=torch.float32, device=_dev())
    _check(_L().sbr_surrogate_targets(pl.handle, _ptr(gains) if pl.n else None, int(F), int(n_taps),
                                      float(tap_s), float(floor_db), _ptr(out), _stream(stream)))
    return out[:n_rx]


class MLP:
    """Handle of sbr_mlp_create (BF16 MLP on Fourier features of (x, y, z, f))."""

    def __init__(self, n_out: int, x_lo, x_hi, width: int = 256, depth: int = 4, max_batch: int = 8192,
                 seed: int = 0, lr: float = 1e-3, betas=(0.9, 0.999), eps: float = 1e-8, err_channel: int = -1,
                 err_of: int = -1, loss_w=None, y_shift=None, y_scale=None, feat_log2_max: float = 9.0,
                 stream=None):
        c = _lib.MlpConfig()
        c.n_out, c.width, c.depth, c.max_batch, c.seed = n_out, width, depth, max_batch, seed
        for k in range(4):
            c.x_lo[k] = float(x_lo[k])
            c.x_hi[k] = float(x_hi[k])
        c.lr, c.beta1, c.beta2, c.eps = lr, betas[0], betas[1], eps
        c.err_channel, c.err_of = err_channel, err_of
        c.feat_log2_max = feat_log2_max
        self.n_out, self.max_batch = n_out, max_batch
        arr = lambda v: None if v is None else np.ascontiguousarray(v, dtype=np.float32)
        lw, sh, sc = arr(loss_w), arr(y_shift), arr(y_scale)
        p = lambda a: None if a is None else a.ctypes.data_as(C.c_void_p)
        h = C.c_void_p()
        _check(_L().sbr_mlp_create(C.byref(c), p(lw), p(sh), p(sc), C.byref(h), _stream(stream)))
        self._h = h

    def train_step(self, x: torch.Tensor, y: torch.Tensor, loss: torch.Tensor = None, stream=None):
        assert x.dtype == torch.float32 and y.dtype == torch.float32
        _check(_L().sbr_mlp_train_step(self._h, _ptr(x), _ptr(y), int(x.shape[0]), _ptr(loss), _stream(stream)))

    def predict(self, x: torch.Tensor, out: torch.Tensor = None, layered: bool = False,
                stream=None) -> torch.Tensor:
        """Outputs for x [B, 4]: one fused launch, or (layered) the per-layer GEMMs."""
        B = int(x.shape[0])
        y = out if out is not None else torch.empty((B, self.n_out), dtype=torch.float32, device=_dev())
        fn = _L().sbr_mlp_predict_layered if layered else _L().sbr_mlp_predict
        _check(fn(self._h, _ptr(x), B, _ptr(y), _stream(stream)))
        return y

    def params(self, mode: int = 0, values: torch.Tensor = None, stream=None) -> torch.Tensor:
        """mode 0: parameters, 2: last gradients (flat float32); mode 1 loads `values`."""
        n = int(_L().sbr_mlp_param_count(self._h))
        buf = values if mode == 1 else torch.empty(n, dtype=torch.float32, device=_dev())
        _check(_L().sbr_mlp_params(self._h, _ptr(buf), int(mode), _stream(stream)))
        return buf

    def status(self):
        _check(_L().sbr_mlp_status(self._h))

    def set_lr(self, lr: float):
        _check(_L().sbr_mlp_set_lr(self._h, float(lr)))

    def free(self):
        if self._h:
            _L().sbr_mlp_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass
