"""ctypes view of the C ABI declared in include/snsolve.h and include/snsolve_debug.h.

Names, structs and argument orders are the C ones.  This module only loads
libsnsolve.so and declares argument types: it does no arithmetic.  If the
library is missing it raises (there is no fallback).
"""
import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libsnsolve.so")

# enums
SNS_OK, SNS_EINVAL, SNS_ENOMEM, SNS_ERANK, SNS_ENOTCONV, SNS_EAGAIN, SNS_ETIMEOUT, SNS_ECUDA, SNS_EBUDGET = range(9)
SNS_COUNTSKETCH, SNS_GAUSSIAN, SNS_SRHT, SNS_SPARSE_SIGN = range(4)
SNS_DENSE_F32, SNS_DENSE_F64, SNS_CSR_F32 = range(3)
SNS_CS_AUTO, SNS_CS_SORTED, SNS_CS_STREAM = range(3)
SNS_SAP, SNS_SAA = range(2)

STATUS_NAMES = {0: "SNS_OK", 1: "SNS_EINVAL", 2: "SNS_ENOMEM", 3: "SNS_ERANK", 4: "SNS_ENOTCONV",
                5: "SNS_EAGAIN", 6: "SNS_ETIMEOUT", 7: "SNS_ECUDA", 8: "SNS_EBUDGET"}


class sns_sketch_desc(C.Structure):
    _fields_ = [("kind", C.c_int32), ("variant", C.c_int32), ("d", C.c_int64), ("seed", C.c_uint64)]


class sns_problem(C.Structure):
    _fields_ = [("m", C.c_int64), ("n", C.c_int64), ("fmt", C.c_int32), ("reserved", C.c_int32),
                ("A", C.c_void_p), ("lda", C.c_int64), ("rowptr", C.c_void_p), ("col", C.c_void_p),
                ("val", C.c_void_p), ("nnz", C.c_int64), ("b", C.c_void_p)]


class sns_opts(C.Structure):
    _fields_ = [("sk", sns_sketch_desc), ("tol", C.c_double), ("max_iter", C.c_int32), ("inner", C.c_int32),
                ("precondition", C.c_int32), ("method", C.c_int32)]


class sns_info(C.Structure):
    _fields_ = [("status", C.c_int32), ("iters", C.c_int32), ("outer", C.c_int32), ("reserved", C.c_int32),
                ("eta", C.c_double), ("resid_norm", C.c_double), ("sketch_resid", C.c_double),
                ("ms_sketch", C.c_float), ("ms_qr", C.c_float), ("ms_iter", C.c_float), ("reserved2", C.c_int32)]


P = C.POINTER
vp = C.c_void_p
i64 = C.c_int64
sz = C.c_size_t

# (name, restype, argtypes) of every exported function
SIGNATURES = [
    ("snsolve_create", C.c_int, [P(vp), C.c_int]),
    ("snsolve_destroy", None, [vp]),
    ("snsolve_status_string", C.c_char_p, [C.c_int]),
    ("snsolve_last_cuda_error", C.c_char_p, []),
    ("snsolve_version", C.c_int, []),
    ("snsolve_sketch_workspace_size", C.c_int, [P(sns_problem), P(sns_sketch_desc), P(sz)]),
    ("snsolve_sketch", C.c_int, [vp, P(sns_problem), P(sns_sketch_desc), vp, i64, vp, vp, sz, vp]),
    ("snsolve_sketch_status", C.c_int, [P(sns_problem), P(sns_sketch_desc), vp, sz, vp]),
    ("snsolve_sketch_rows", C.c_int, [vp, P(sns_problem), P(sns_sketch_desc), i64, vp, i64, vp, vp, sz, vp]),
    ("snsolve_solve_sketched_workspace_size", C.c_int, [i64, i64, P(sz)]),
    ("snsolve_solve_sketched", C.c_int, [vp, vp, i64, C.c_int32, i64, i64, vp, P(sns_info), vp, sz, vp]),
    ("snsolve_lstsq_workspace_size", C.c_int, [P(sns_problem), P(sns_opts), P(sz)]),
    ("snsolve_lstsq", C.c_int, [vp, P(sns_problem), P(sns_opts), vp, P(sns_info), vp, sz, vp]),
    ("snsolve_lstsq_batched_workspace_size", C.c_int, [P(sns_problem), P(sns_opts), C.c_int, P(sz)]),
    ("snsolve_lstsq_batched", C.c_int, [vp, P(sns_problem), P(sns_opts), C.c_int, P(vp), P(sns_info), vp, sz, vp]),
    ("snsolve_server_create", C.c_int, [P(vp), vp, sz, C.c_int]),
    ("snsolve_server_destroy", None, [vp]),
    ("snsolve_submit", C.c_int, [vp, P(sns_problem), P(sns_opts), vp, P(C.c_uint64)]),
    ("snsolve_poll", C.c_int, [vp, C.c_uint64, i64, P(sns_info)]),
    ("snsolve_server_stats", C.c_int, [vp, P(C.c_int), P(C.c_int), P(sz)]),
    ("snsolve_sketch_countsketch_static", C.c_int, [P(sns_problem), i64, C.c_uint64, vp, i64, vp, vp]),
    # debug ABI
    ("snsolve_debug_countsketch_hash", C.c_int, [i64, i64, C.c_uint64, vp, vp, vp]),
    ("snsolve_debug_stream_keys", C.c_int, [C.c_uint64, C.c_int, i64, i64, vp, vp]),
    ("snsolve_debug_srht_sample_ws", C.c_int, [i64, i64, P(sz)]),
    ("snsolve_debug_srht_sample", C.c_int, [i64, i64, C.c_uint64, vp, vp, sz, vp]),
    ("snsolve_debug_gaussian_table", C.c_int, [P(C.c_uint16)]),
    ("snsolve_launch_count", C.c_uint64, []),
    ("snsolve_profile", C.c_int, [C.c_int]),
    ("snsolve_profile_num_kernels", C.c_int, []),
    ("snsolve_profile_kernel_name", C.c_char_p, [C.c_int]),
    ("snsolve_profile_read", C.c_int, [P(C.c_double), P(C.c_uint64), C.c_int]),
    ("snsolve_tune_reset", None, []),
    ("snsolve_debug_set_qr_wait_limit", None, [i64]),
    ("snsolve_debug_form_y", C.c_int, [P(sns_problem), vp, vp, i64, vp]),
    ("snsolve_debug_set_fault", C.c_int, [C.c_char_p]),
    ("snsolve_debug_fault_armed", C.c_int, [P(i64)]),
]

_lib = None


def lib():
    """The loaded library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "`python -c 'import __graft_entry__ as g; g.build()'` (no CPU fallback exists)")
        L = C.CDLL(LIB_PATH)
        for name, res, args in SIGNATURES:
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def status_name(code):
    return STATUS_NAMES.get(int(code), f"status {code}")
