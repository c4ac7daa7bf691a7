"""GB300 (sm_103a) sketch-and-solve least squares: a thin torch-facing binding of
the C ABI in include/snsolve.h.

Every arithmetic step runs in libsnsolve.so's CUDA kernels; this module only
marshals torch tensors (device memory) and the current torch CUDA stream into
the C calls, and allocates the caller-side workspace with torch.
"""
import ctypes as C

import numpy as np
import torch

from . import abi
from .abi import (SNS_COUNTSKETCH, SNS_GAUSSIAN, SNS_SRHT, SNS_SPARSE_SIGN, SNS_CS_AUTO, SNS_CS_SORTED, SNS_CS_STREAM,
                  SNS_DENSE_F32, SNS_DENSE_F64, SNS_CSR_F32, status_name)

KIND = {"countsketch": SNS_COUNTSKETCH, "gaussian": SNS_GAUSSIAN, "srht": SNS_SRHT, "sparse_sign": SNS_SPARSE_SIGN}
VARIANT = {"auto": SNS_CS_AUTO, "sorted": SNS_CS_SORTED, "stream": SNS_CS_STREAM}


class SnsError(RuntimeError):
    def __init__(self, code, where):
        self.code = int(code)
        msg = f"{where}: {status_name(code)}"
        if self.code == abi.SNS_ECUDA:
            msg += f" ({abi.lib().snsolve_last_cuda_error().decode()})"
        super().__init__(msg)


def _check(code, where):
    if int(code) != abi.SNS_OK:
        raise SnsError(code, where)


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None else C.c_void_p(0)


def dense_problem(A, b):
    """sns_problem for a dense row-major CUDA matrix A (float32/float64, unit column stride)."""
    assert A.is_cuda and A.dim() == 2 and A.stride(1) == 1
    assert b.is_cuda and b.dim() == 1 and b.is_contiguous() and b.dtype == A.dtype
    fmt = SNS_DENSE_F64 if A.dtype == torch.float64 else SNS_DENSE_F32
    if A.dtype not in (torch.float32, torch.float64):
        raise TypeError("A must be float32 or float64")
    p = abi.sns_problem(m=A.shape[0], n=A.shape[1], fmt=fmt, A=A.data_ptr(), lda=A.stride(0), b=b.data_ptr())
    return p


def csr_problem(rowptr, col, val, b, n):
    """sns_problem for a CSR CUDA matrix (rowptr int64, col int32, val float32)."""
    assert rowptr.dtype == torch.int64 and col.dtype == torch.int32 and val.dtype == torch.float32
    assert b.dtype == torch.float32
    m = rowptr.numel() - 1
    return abi.sns_problem(m=m, n=n, fmt=SNS_CSR_F32, rowptr=rowptr.data_ptr(), col=col.data_ptr(),
                           val=val.data_ptr(), nnz=col.numel(), b=b.data_ptr(), lda=0)


def sketch_desc(d, kind="countsketch", seed=0, variant="auto"):
    """Sketch descriptor.  For CountSketch `variant` is "auto", "sorted" or
    "stream"; for the sparse sign embedding it is zeta, the nonzeros per column
    (an int 1..8; "auto" means 4); for the Gaussian sketch it is the number of
    BF16 terms of [A | b] in the tensor-core product (1, 2 or 3; "auto": 1 for
    a sketch, 3 inside a solve)."""
    if kind == "sparse_sign":
        v = 4 if variant == "auto" else int(variant)
    elif kind == "gaussian":
        v = 0 if variant == "auto" else int(variant)
    else:
        v = VARIANT[variant]
    return abi.sns_sketch_desc(kind=KIND[kind], variant=v, d=int(d), seed=int(seed) & (2**64 - 1))


METHOD = {"sap": abi.SNS_SAP, "saa": abi.SNS_SAA}


def opts(d, kind="countsketch", seed=0, variant="auto", tol=0.0, max_iter=0, inner=0, precondition=True,
         method="sap"):
    """Solve options; method "sap" (sketch-and-precondition) or "saa"
    (sketch-and-apply: explicit Y = A R^-1) for the iterative phase."""
    return abi.sns_opts(sk=sketch_desc(d, kind, seed, variant), tol=float(tol), max_iter=int(max_iter),
                        inner=int(inner), precondition=1 if precondition else 0, method=METHOD[method])


def _workspace(nbytes, device):
    return torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=device)


class Context:
    """Owns an sns_ctx on one CUDA device."""

    def __init__(self, device=0):
        self._L = abi.lib()
        h = C.c_void_p()
        _check(self._L.snsolve_create(C.byref(h), int(device)), "snsolve_create")
        self.h = h
        self.device = torch.device("cuda", int(device))

    def close(self):
        if getattr(self, "h", None):
            self._L.snsolve_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -------------------------------------------------------------- sketch
    def sketch_workspace(self, prob, sk):
        n = C.c_size_t()
        _check(self._L.snsolve_sketch_workspace_size(C.byref(prob), C.byref(sk), C.byref(n)),
               "snsolve_sketch_workspace_size")
        return n.value

    def sketch_problem(self, prob, sk, out_dtype, ws=None, stream=None):
        """SA (d x n) and Sb (d) for an sns_problem."""
        SA = torch.empty((sk.d, prob.n), dtype=out_dtype, device=self.device)
        Sb = torch.empty((sk.d,), dtype=out_dtype, device=self.device)
        need = self.sketch_workspace(prob, sk)
        if ws is None or ws.numel() < need:
            ws = _workspace(need, self.device)
        _check(self._L.snsolve_sketch(self.h, C.byref(prob), C.byref(sk), _ptr(SA), SA.stride(0), _ptr(Sb),
                                      _ptr(ws), ws.numel(), _stream(stream)), "snsolve_sketch")
        return SA, Sb

    def sketch(self, A, b, d, kind="countsketch", seed=0, variant="auto", ws=None, stream=None):
        """SA = S A and Sb = S b for a dense CUDA matrix."""
        return self.sketch_problem(dense_problem(A, b), sketch_desc(d, kind, seed, variant), A.dtype, ws, stream)

    def sketch_rows(self, A, b, row0, d, kind="countsketch", seed=0, variant="auto", ws=None, stream=None):
        """Partial sketch of rows row0.. of a larger dense matrix (global row
        indices); the sketch of the whole matrix is the sum of the parts'."""
        prob, sk = dense_problem(A, b), sketch_desc(d, kind, seed, variant)
        SA = torch.empty((sk.d, prob.n), dtype=A.dtype, device=self.device)
        Sb = torch.empty((sk.d,), dtype=A.dtype, device=self.device)
        need = self.sketch_workspace(prob, sk)
        if ws is None or ws.numel() < need:
            ws = _workspace(need, self.device)
        _check(self._L.snsolve_sketch_rows(self.h, C.byref(prob), C.byref(sk), int(row0), _ptr(SA), SA.stride(0),
                                           _ptr(Sb), _ptr(ws), ws.numel(), _stream(stream)), "snsolve_sketch_rows")
        return SA, Sb

    def solve_sketched(self, SAaug, ws=None, stream=None, check=True):
        """x^ = argmin ||SA x - Sb|| from a d x (n+1) augmented [SA | Sb] on the
        device (FP32 or FP64): FP64 Householder QR and back substitution."""
        assert SAaug.is_cuda and SAaug.dim() == 2 and SAaug.stride(1) == 1
        d, q = SAaug.shape
        n = q - 1
        sz = C.c_size_t()
        _check(self._L.snsolve_solve_sketched_workspace_size(d, n, C.byref(sz)),
               "snsolve_solve_sketched_workspace_size")
        if ws is None or ws.numel() < sz.value:
            ws = _workspace(sz.value, self.device)
        x = torch.empty(n, dtype=torch.float64, device=self.device)
        info = abi.sns_info()
        code = self._L.snsolve_solve_sketched(self.h, _ptr(SAaug), SAaug.stride(0),
                                              1 if SAaug.dtype == torch.float64 else 0, d, n, _ptr(x),
                                              C.byref(info), _ptr(ws), ws.numel(), _stream(stream))
        if check and code not in (abi.SNS_OK, abi.SNS_ERANK):
            raise SnsError(code, "snsolve_solve_sketched")
        return x, info

    def sketch_csr(self, rowptr, col, val, b, n, d, seed=0, variant="auto", ws=None, stream=None):
        return self.sketch_problem(csr_problem(rowptr, col, val, b, n), sketch_desc(d, "countsketch", seed, variant),
                                   torch.float32, ws, stream)

    # -------------------------------------------------------------- solve
    def lstsq_workspace(self, prob, op):
        n = C.c_size_t()
        _check(self._L.snsolve_lstsq_workspace_size(C.byref(prob), C.byref(op), C.byref(n)),
               "snsolve_lstsq_workspace_size")
        return n.value

    def lstsq_problem(self, prob, op, x=None, ws=None, stream=None, check=True):
        if x is None:
            x = torch.empty(prob.n, dtype=torch.float64, device=self.device)
        need = self.lstsq_workspace(prob, op)
        if ws is None or ws.numel() < need:
            ws = _workspace(need, self.device)
        info = abi.sns_info()
        code = self._L.snsolve_lstsq(self.h, C.byref(prob), C.byref(op), _ptr(x), C.byref(info), _ptr(ws),
                                     ws.numel(), _stream(stream))
        if check and code not in (abi.SNS_OK, abi.SNS_ERANK, abi.SNS_ENOTCONV):
            raise SnsError(code, "snsolve_lstsq")
        return x, info

    def lstsq(self, A, b, d, kind="countsketch", seed=0, tol=0.0, max_iter=0, inner=0, precondition=True,
              variant="auto", ws=None, stream=None, method="sap"):
        """Sketch-and-solve (tol <= 0), or sketch-and-precondition ("sap") /
        sketch-and-apply ("saa") to eta <= tol."""
        return self.lstsq_problem(dense_problem(A, b),
                                  opts(d, kind, seed, variant, tol, max_iter, inner, precondition, method), ws=ws,
                                  stream=stream)

    def lstsq_csr(self, rowptr, col, val, b, n, d, seed=0, tol=0.0, max_iter=0, inner=0, precondition=True,
                  variant="auto", ws=None, stream=None):
        """variant="sorted" makes the whole CSR solve bitwise reproducible
        (n <= 1422), at about 2.5x the time of the default."""
        return self.lstsq_problem(csr_problem(rowptr, col, val, b, n),
                                  opts(d, "countsketch", seed, variant, tol, max_iter, inner, precondition),
                                  ws=ws, stream=stream)

    # -------------------------------------------------------------- batched
    def lstsq_batched(self, As, bs, ds, seeds, ws=None, stream=None, check=True):
        """Sketch-and-solve of many dense FP32 problems in one persistent launch.
        As, bs: lists of CUDA tensors; ds, seeds: ints per problem.  Returns
        (list of x tensors, list of sns_info).  The problem and option tables
        are filled column-wise (numpy arrays laid out as the C structs) and the
        x vectors are views of one allocation, so marshalling stays a small
        fraction of a batch."""
        k = len(As)
        for A, b in zip(As, bs):
            if not (A.is_cuda and b.is_cuda and A.dtype == torch.float32 and b.dtype == torch.float32
                    and A.dim() == 2 and A.stride(1) == 1 and b.dim() == 1 and b.is_contiguous()):
                raise TypeError("lstsq_batched: every A must be a row-major float32 CUDA matrix, b float32")
        ns = [A.shape[1] for A in As]
        probs = np.zeros(k, dtype=np.dtype(abi.sns_problem))
        probs["m"] = [A.shape[0] for A in As]
        probs["n"] = ns
        probs["fmt"] = SNS_DENSE_F32
        probs["A"] = [A.data_ptr() for A in As]
        probs["lda"] = [A.stride(0) for A in As]
        probs["b"] = [b.data_ptr() for b in bs]
        ops = np.zeros(k, dtype=np.dtype(abi.sns_opts))
        ops["sk"]["kind"] = abi.SNS_COUNTSKETCH
        ops["sk"]["d"] = ds
        ops["sk"]["seed"] = [int(sd) & (2**64 - 1) for sd in seeds]
        ops["precondition"] = 1
        xflat = torch.empty(sum(ns), dtype=torch.float64, device=self.device)
        xs = list(torch.split(xflat, ns))
        xp = np.empty(k, dtype=np.uint64)
        xp[0] = xflat.data_ptr()
        if k > 1:
            xp[1:] = xflat.data_ptr() + 8 * np.cumsum(np.asarray(ns[:-1], dtype=np.uint64))
        pp = probs.ctypes.data_as(C.POINTER(abi.sns_problem))
        op = ops.ctypes.data_as(C.POINTER(abi.sns_opts))
        xpp = xp.ctypes.data_as(C.POINTER(C.c_void_p))
        n = C.c_size_t()
        _check(self._L.snsolve_lstsq_batched_workspace_size(pp, op, k, C.byref(n)),
               "snsolve_lstsq_batched_workspace_size")
        if ws is None or ws.numel() < n.value:
            ws = _workspace(n.value, self.device)
        infos = (abi.sns_info * k)()
        code = self._L.snsolve_lstsq_batched(self.h, pp, op, k, xpp, infos, _ptr(ws), ws.numel(), _stream(stream))
        if check and code not in (abi.SNS_OK, abi.SNS_ERANK):
            raise SnsError(code, "snsolve_lstsq_batched")
        return xs, list(infos)

    # -------------------------------------------------------------- debug
    def countsketch_hash(self, m, d, seed, stream=None):
        h = torch.empty(m, dtype=torch.int32, device=self.device)
        s = torch.empty(m, dtype=torch.int8, device=self.device)
        _check(self._L.snsolve_debug_countsketch_hash(m, d, seed & (2**64 - 1), _ptr(h), _ptr(s), _stream(stream)),
               "snsolve_debug_countsketch_hash")
        return h, s

    def stream_keys(self, seed, stream_id, start, count, stream=None):
        k = torch.empty(count, dtype=torch.int64, device=self.device)
        _check(self._L.snsolve_debug_stream_keys(seed & (2**64 - 1), stream_id, start, count, _ptr(k),
                                                 _stream(stream)), "snsolve_debug_stream_keys")
        return k

    def srht_sample(self, mp, d, seed, stream=None):
        n = C.c_size_t()
        _check(self._L.snsolve_debug_srht_sample_ws(mp, d, C.byref(n)), "snsolve_debug_srht_sample_ws")
        ws = _workspace(n.value, self.device)
        idx = torch.empty(d, dtype=torch.int64, device=self.device)
        _check(self._L.snsolve_debug_srht_sample(mp, d, seed & (2**64 - 1), _ptr(idx), _ptr(ws), ws.numel(),
                                                 _stream(stream)), "snsolve_debug_srht_sample")
        return idx


class Server:
    """Continuous-batching request server over one Context (snsolve_server_*)."""

    def __init__(self, ctx, hbm_budget_bytes, max_slots):
        self.ctx = ctx
        self._L = ctx._L
        h = C.c_void_p()
        _check(self._L.snsolve_server_create(C.byref(h), ctx.h, int(hbm_budget_bytes), int(max_slots)),
               "snsolve_server_create")
        self.h = h
        self._keep = {}

    def submit_problem(self, prob, op, x, keep=()):
        rid = C.c_uint64()
        code = self._L.snsolve_submit(self.h, C.byref(prob), C.byref(op), _ptr(x), C.byref(rid))
        if code != abi.SNS_OK:
            raise SnsError(code, "snsolve_submit")
        self._keep[rid.value] = (x,) + tuple(keep)       # tensors must outlive the request
        return rid.value

    def submit(self, A, b, d, seed=0, tol=0.0, kind="countsketch", max_iter=0, inner=0):
        x = torch.empty(A.shape[1], dtype=torch.float64, device=self.ctx.device)
        return self.submit_problem(dense_problem(A, b), opts(d, kind, seed, "auto", tol, max_iter, inner), x,
                                   keep=(A, b)), x

    def submit_csr(self, rowptr, col, val, b, n, d, seed=0, tol=0.0, max_iter=0, variant="auto"):
        x = torch.empty(n, dtype=torch.float64, device=self.ctx.device)
        return self.submit_problem(csr_problem(rowptr, col, val, b, n),
                                   opts(d, "countsketch", seed, variant, tol, max_iter), x,
                                   keep=(rowptr, col, val, b)), x

    def poll(self, rid, timeout_us=0):
        """(status code of the poll, sns_info or None)."""
        info = abi.sns_info()
        code = self._L.snsolve_poll(self.h, rid, int(timeout_us), C.byref(info))
        if code == abi.SNS_OK:
            self._keep.pop(rid, None)
            return code, info
        return code, None

    def stats(self):
        r, p, u = C.c_int(), C.c_int(), C.c_size_t()
        _check(self._L.snsolve_server_stats(self.h, C.byref(r), C.byref(p), C.byref(u)), "snsolve_server_stats")
        return r.value, p.value, u.value

    def close(self):
        if getattr(self, "h", None):
            self._L.snsolve_server_destroy(self.h)
            self.h = None
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def gaussian_table_bits():
    """The library's BF16 normal-quantile table as 256 raw uint16 values (host call)."""
    buf = (C.c_uint16 * 256)()
    _check(abi.lib().snsolve_debug_gaussian_table(buf), "snsolve_debug_gaussian_table")
    return list(buf)
