"""ctypes declarations of the C ABI in include/sbr.h (libsbr.so, in-tree)."""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libsbr.so")

SBR_OK = 0
STATUS_NAMES = {0: "SBR_OK", 1: "SBR_ERR_INVALID_ARG", 2: "SBR_ERR_CUDA", 3: "SBR_ERR_CAPACITY",
                4: "SBR_ERR_STACK_OVERFLOW", 5: "SBR_ERR_TIMEOUT", 6: "SBR_ERR_NUMERIC",
                7: "SBR_ERR_UNSUPPORTED", 8: "SBR_ERR_ALLOC"}
KMAX = 8
NSTATS = 7
POL_V, POL_H = 0, 1
SYNTH_FP64, SYNTH_FP32, SYNTH_BF16X3, SYNTH_FP16X3 = 0, 1, 2, 3
TRACE_TIMING = 1
TRACE_COUNT_VISITS = 2

BVH_SAH_TOP = 1   # sbr_build_bvh_ex flag

EXPORTS = ["sbr_last_error", "sbr_version", "sbr_launch_count", "sbr_launch_dirs", "sbr_build_bvh", "sbr_build_bvh_ex", "sbr_bvh_free",
           "sbr_bvh_query", "sbr_trace", "sbr_trace_stats", "sbr_trace_free", "sbr_trace_entries",
           "sbr_trace_merge", "sbr_paths",
           "sbr_path_query", "sbr_path_export", "sbr_path_list_free", "sbr_path_gains",
           "sbr_synthesize_H", "sbr_synthesize_H_elements", "sbr_pdp_angles", "sbr_capacity", "sbr_capacity_noalloc",
           "sbr_batch_create", "sbr_batch_run", "sbr_batch_query", "sbr_batch_export", "sbr_batch_free",
           "sbr_batch_tune", "sbr_surrogate_targets", "sbr_mlp_create", "sbr_mlp_train_step",
           "sbr_mlp_predict", "sbr_mlp_param_count", "sbr_mlp_params", "sbr_mlp_status", "sbr_mlp_free",
           "sbr_mlp_set_lr", "sbr_mlp_predict_layered"]


class TraceParams(C.Structure):
    _fields_ = [("tx", C.c_double * 3), ("rx_xyz", C.c_void_p), ("n_rx", C.c_int32),
                ("subdiv_N", C.c_int32), ("max_bounces", C.c_int32), ("table_log2", C.c_int32),
                ("alpha", C.c_double), ("flags", C.c_uint32), ("depth_first_from", C.c_int32),
                ("ray_begin", C.c_int64), ("ray_end", C.c_int64)]


class TraceCounters(C.Structure):
    _fields_ = [("rays", C.c_int64), ("ray_bounces", C.c_int64), ("candidates", C.c_int64),
                ("keys", C.c_int64), ("fp64_segments", C.c_int64), ("fp64_tests", C.c_int64),
                ("node_visits", C.c_int64), ("tri_tests", C.c_int64), ("rx_visits", C.c_int64),
                ("near_edge_hits", C.c_int64),
                ("queue", C.c_int64 * (KMAX + 2)),
                ("alpha", C.c_double), ("status", C.c_int32), ("table_log2", C.c_int32),
                ("bounce_ms", C.c_float * (KMAX + 1)), ("reserved", C.c_int32)]


class BvhInfo(C.Structure):
    _fields_ = [("T", C.c_int64), ("S", C.c_int32), ("n_nodes", C.c_int32), ("depth", C.c_int32),
                ("reserved", C.c_int32)]


class PathInfo(C.Structure):
    _fields_ = [("n_paths", C.c_int64), ("n_keys", C.c_int64), ("n_invalid", C.c_int64),
                ("n_rx", C.c_int32), ("max_bounces", C.c_int32), ("status", C.c_int32),
                ("reserved", C.c_int32)]


class BatchJob(C.Structure):
    _fields_ = [("scene", C.c_int32), ("subdiv_N", C.c_int32), ("max_bounces", C.c_int32),
                ("pol", C.c_int32), ("tx", C.c_double * 3), ("rx", C.c_double * 3), ("alpha", C.c_double),
                ("F", C.c_int32), ("Nt", C.c_int32), ("Nr", C.c_int32), ("reserved", C.c_int32),
                ("freqs_hz", C.c_void_p), ("gamma_db_km", C.c_void_p), ("disp_deg_km", C.c_void_p),
                ("tx_elem", C.c_void_p), ("rx_elem", C.c_void_p), ("H", C.c_void_p)]


class BatchConfig(C.Structure):
    _fields_ = [("wave_rays", C.c_int64), ("path_cap", C.c_int32), ("table_log2", C.c_int32),
                ("tile_n", C.c_int32), ("trace_blocks_per_sm", C.c_int32), ("precision", C.c_int32),
                ("use_graph", C.c_int32), ("breadth_first", C.c_int32), ("reserved", C.c_int32)]


class BatchInfo(C.Structure):
    _fields_ = [("n_jobs", C.c_int32), ("n_waves", C.c_int32), ("graph_kernels", C.c_int32),
                ("status", C.c_int32), ("max_keys", C.c_int32), ("reserved", C.c_int32),
                ("rays", C.c_int64), ("ray_bounces", C.c_int64), ("paths", C.c_int64),
                ("config", BatchConfig)]


class MlpConfig(C.Structure):
    _fields_ = [("n_out", C.c_int32), ("width", C.c_int32), ("depth", C.c_int32), ("max_batch", C.c_int32),
                ("seed", C.c_uint64), ("x_lo", C.c_float * 4), ("x_hi", C.c_float * 4), ("lr", C.c_float),
                ("beta1", C.c_float), ("beta2", C.c_float), ("eps", C.c_float), ("err_channel", C.c_int32),
                ("err_of", C.c_int32), ("feat_log2_max", C.c_float), ("reserved", C.c_int32)]


assert C.sizeof(TraceParams) == 80
assert C.sizeof(BatchJob) == 136
assert C.sizeof(BatchConfig) == 40
assert C.sizeof(BatchInfo) == 88

_lib = None


def load() -> C.CDLL:
    """Load libsbr.so; raises if it has not been built (no fallback exists)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError("libsbr.so is not built: run __graft_entry__.build() or "
                          "python paper_2208_10006_gb300/build.py")
    L = C.CDLL(LIB_PATH)
    p, i32, i64, f64, st = C.c_void_p, C.c_int32, C.c_int64, C.c_double, C.c_int
    pp = C.POINTER(C.c_void_p)
    L.sbr_last_error.restype = C.c_char_p
    L.sbr_last_error.argtypes = []
    L.sbr_version.restype = C.c_char_p
    L.sbr_version.argtypes = []
    L.sbr_launch_count.restype = i64
    L.sbr_launch_count.argtypes = []
    L.sbr_launch_dirs.restype = st
    L.sbr_launch_dirs.argtypes = [i32, p, p, p]
    L.sbr_build_bvh.restype = st
    L.sbr_build_bvh.argtypes = [p, p, i64, i32, pp, p]
    L.sbr_build_bvh_ex.restype = st
    L.sbr_build_bvh_ex.argtypes = [p, p, i64, i32, C.c_uint32, pp, p]
    L.sbr_bvh_free.restype = None
    L.sbr_bvh_free.argtypes = [p]
    L.sbr_bvh_query.restype = st
    L.sbr_bvh_query.argtypes = [p, C.POINTER(BvhInfo)]
    L.sbr_trace.restype = st
    L.sbr_trace.argtypes = [p, C.POINTER(TraceParams), pp, p]
    L.sbr_trace_stats.restype = st
    L.sbr_trace_stats.argtypes = [p, C.POINTER(TraceCounters)]
    L.sbr_trace_free.restype = None
    L.sbr_trace_free.argtypes = [p]
    L.sbr_trace_entries.restype = st
    L.sbr_trace_entries.argtypes = [p, p, p, i64, C.POINTER(C.c_int64), p]
    L.sbr_trace_merge.restype = st
    L.sbr_trace_merge.argtypes = [C.POINTER(TraceParams), p, p, i64, pp, p]
    L.sbr_paths.restype = st
    L.sbr_paths.argtypes = [p, p, pp, C.POINTER(C.c_int64), p]
    L.sbr_path_query.restype = st
    L.sbr_path_query.argtypes = [p, C.POINTER(PathInfo)]
    L.sbr_path_export.restype = st
    L.sbr_path_export.argtypes = [p] + [p] * 10 + [p]
    L.sbr_path_list_free.restype = None
    L.sbr_path_list_free.argtypes = [p]
    L.sbr_path_gains.restype = st
    L.sbr_path_gains.argtypes = [p, p, i32, p, i32, p, p, i32, p, p]
    L.sbr_synthesize_H.restype = st
    L.sbr_synthesize_H.argtypes = [p, p, p, i32, p, i32, p, i32, i32, i32, p, p]
    L.sbr_synthesize_H_elements.restype = st
    L.sbr_synthesize_H_elements.argtypes = [p, p, p, i32, p, i32, i32, p, p]
    L.sbr_pdp_angles.restype = st
    L.sbr_pdp_angles.argtypes = [p, p, i32, i32, f64, f64, i32, p, p, p]
    L.sbr_capacity.restype = st
    L.sbr_capacity.argtypes = [p, i32, i32, i32, p, i32, p, p]
    L.sbr_capacity_noalloc.restype = st
    L.sbr_capacity_noalloc.argtypes = [p, i32, i32, i32, p, i32, p, p]
    L.sbr_batch_create.restype = st
    L.sbr_batch_create.argtypes = [p, p, i32, C.POINTER(BatchJob), i32, C.POINTER(BatchConfig), pp, p]
    L.sbr_batch_run.restype = st
    L.sbr_batch_run.argtypes = [p, p]
    L.sbr_batch_query.restype = st
    L.sbr_batch_query.argtypes = [p, p, p, C.POINTER(BatchInfo)]
    L.sbr_batch_export.restype = st
    L.sbr_batch_export.argtypes = [p, i32, i32] + [p] * 10 + [p]
    L.sbr_batch_free.restype = None
    L.sbr_batch_free.argtypes = [p]
    L.sbr_batch_tune.restype = st
    L.sbr_batch_tune.argtypes = [p, p, i32, C.POINTER(BatchJob), i32, C.POINTER(BatchConfig),
                                 C.POINTER(C.c_double), p]
    L.sbr_surrogate_targets.restype = st
    L.sbr_surrogate_targets.argtypes = [p, p, i32, i32, f64, f64, p, p]
    L.sbr_mlp_create.restype = st
    L.sbr_mlp_create.argtypes = [C.POINTER(MlpConfig), p, p, p, pp, p]
    L.sbr_mlp_train_step.restype = st
    L.sbr_mlp_train_step.argtypes = [p, p, p, i32, p, p]
    L.sbr_mlp_predict.restype = st
    L.sbr_mlp_predict.argtypes = [p, p, i32, p, p]
    L.sbr_mlp_predict_layered.restype = st
    L.sbr_mlp_predict_layered.argtypes = [p, p, i32, p, p]
    L.sbr_mlp_param_count.restype = i64
    L.sbr_mlp_param_count.argtypes = [p]
    L.sbr_mlp_params.restype = st
    L.sbr_mlp_params.argtypes = [p, p, i32, p]
    L.sbr_mlp_status.restype = st
    L.sbr_mlp_status.argtypes = [p]
    L.sbr_mlp_set_lr.restype = st
    L.sbr_mlp_set_lr.argtypes = [p, C.c_float]
    L.sbr_mlp_free.restype = None
    L.sbr_mlp_free.argtypes = [p]
    _lib = L
    return L
