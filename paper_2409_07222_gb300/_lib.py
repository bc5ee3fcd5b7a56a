"""ctypes loader for liblabs.so (the C ABI declared in include/labs.h).

There is no fallback: if the library is missing or fails to load, every call raises.
"""
import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "liblabs.so")

LABS_OK = 0
LABS_ERR_INVALID_ARG = 1
LABS_ERR_CAPACITY = 2
LABS_ERR_TIMEOUT = 3
LABS_ERR_CUDA = 4
LABS_ERR_NOMEM = 5
LABS_MAX_L = 576
LABS_MAX_W = 9
LABS_AUTO_THRESHOLD = -(2**31)
INT32_MIN = -(2**31)
INT32_MAX = 2**31 - 1

# Every symbol include/labs.h declares, with its ctypes signature.
_P = ctypes.c_void_p
_i32, _i64, _u64, _ci = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_int
SIGNATURES = {
    "labs_ctx_create": (_ci, [ctypes.POINTER(_P), _ci]),
    "labs_ctx_destroy": (None, [_P]),
    "labs_status_string": (ctypes.c_char_p, [_ci]),
    "labs_abi_version": (_ci, []),
    "labs_energy_batch": (_ci, [_P, _P, _ci, _i64, _P, _P, _P]),
    "labs_flip_deltas": (_ci, [_P, _P, _P, _ci, _i64, _ci, _ci, _P, _P]),
    "labs_skew_search": (_ci, [_P, _P, _P, _ci, _P, _P, _P, _P]),
    "labs_sample_threshold": (_ci, [_P, _ci, _ci, _ci, _P, _ci, _u64, _i64, _i64, _P, _P, _P]),
    "labs_skew_exhaustive": (_ci, [_P, _ci, _ci, _u64, _P, _P, _P, _P, _P]),
    "labs_sample_threshold_noalloc": (_ci, [_ci, _ci, _ci, _P, _ci, _u64, _i64, _i64, _P, _P]),
    "labs_batched_search": (_ci, [_P, _P, _P, _P, _P, _ci, _P, _P, _P, _P, _P]),
    "labs_sequence_operators": (_ci, [_P, _P, _ci, _i64, _P, _P, _P, _P, _P]),
    "labs_legendre_family": (_ci, [_ci, ctypes.c_double, ctypes.c_double, ctypes.c_double, _P, _i64, _P]),
    "labs_legendre_construct": (_ci, [_P, _ci, _P, _i64, _P, _P, _P]),
    "labs_pq_independent": (_ci, [_P, _P, _P, _ci, _P, _P, _P, _P]),
    "labs_pq_refine": (_ci, [_P, _P, _P, _ci, _P, _P, _P, _P]),
    "labs_chunked_search": (_ci, [_P, _P, _P, ctypes.c_float, _ci, _P, _ci, _P, _P, _P, _P, _P, _P, _P]),
    "labs_policy_param_count": (_ci, [_ci, _P]),
    "labs_policy_create": (_ci, [_P, _ci, _u64, ctypes.POINTER(_P)]),
    "labs_policy_destroy": (None, [_P]),
    "labs_policy_set_params": (_ci, [_P, _P, _P]),
    "labs_policy_get_params": (_ci, [_P, _P, _P]),
    "labs_policy_forward": (_ci, [_P, _P, _i64, _P, _P]),
    "labs_policy_sync_status": (_ci, [_P, _P]),
    "labs_policy_train_step": (_ci, [_P, _P, _P, _P, _i64, _ci, _ci, ctypes.c_float, _P, _P, _P]),
    "labs_seq_to_hex": (_ci, [_P, _ci, ctypes.c_char_p, ctypes.c_size_t]),
    "labs_hex_to_seq": (_ci, [ctypes.c_char_p, _ci, _P]),
    "labs_measure_issue_rates": (_ci, [_ci, _P, _ci]),
}


class WalkCfg(ctypes.Structure):
    """labs_walk_cfg (include/labs.h)."""

    _fields_ = [
        ("L", _i32), ("skew", _i32), ("p", _i32), ("T_i", _i32),
        ("n_walks", _i64), ("walk_begin", _i64), ("flip_budget", _i64),
        ("seed", _u64),
        ("R", _i32), ("bloom_log2", _i32), ("bloom_k", _i32), ("E_thr", _i32),
        ("n_thresh_samples", _i64), ("thresh_rank", _i64),
        ("E_target", _i32), ("tile_m", _i32), ("warps_per_cta", _i32), ("lanes_per_walk", _i32),
        ("E_thr_dev", _P),
    ]


class BatchCfg(ctypes.Structure):
    """labs_batch_cfg (include/labs.h)."""

    _fields_ = [
        ("n_len", _i32), ("p", _i32), ("flip_budget", _i64), ("seed", _u64),
        ("R", _i32), ("bloom_log2", _i32), ("bloom_k", _i32), ("T_i", _i32),
        ("n_thresh_samples", _i64), ("thresh_rank", _i64),
        ("E_target", _i32), ("tile_m", _i32), ("warps_per_cta", _i32), ("use_graph", _i32),
    ]


class PqCfg(ctypes.Structure):
    """labs_pq_cfg (include/labs.h)."""

    _fields_ = [
        ("L", _i32), ("B", _i32), ("cap", _i64), ("H_log2", _i32), ("T_r", _i32),
        ("max_expansions", _i64), ("T_u", _i64),
    ]


class PqIndepCfg(ctypes.Structure):
    """labs_pq_indep_cfg (include/labs.h)."""

    _fields_ = [
        ("L", _i32), ("T_r", _i32), ("H_log2", _i32), ("reserved", _i32), ("max_expansions", _i64),
        ("T_u", _i64), ("max_workspace_bytes", _i64),
    ]


WALK_STATS_BYTES = 48  # labs_walk_stats
PQ_STATS_BYTES = 72    # labs_pq_stats
CANDIDATE_BYTES = 96   # labs_candidate

_lib = None


class LabsError(RuntimeError):
    def __init__(self, status, what):
        super().__init__("%s failed: %s (status %d)" % (what, status_string(status), status))
        self.status = status


def load():
    """Loads liblabs.so; raises if it has not been built (no CPU fallback exists)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("liblabs.so is not built (run __graft_entry__.build() or "
                              "python paper_2409_07222_gb300/build.py)")
        lib = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
    return _lib


def status_string(status):
    return load().labs_status_string(status).decode()


def check(status, what):
    if status != LABS_OK:
        raise LabsError(status, what)
