"""CPU-side checks of the C ABI: the library loads, exports every function the
headers declare, and its host-only logic (status strings, argument validation,
workspace queries, the Gaussian table) behaves as documented.  No kernel runs."""
import ctypes as C
import glob
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        txt = open(h).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        for m in re.finditer(r"\b(snsolve_\w+)\s*\(", txt):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_2409_14309_gb300 import abi
    if not os.path.exists(abi.LIB_PATH):
        from paper_2409_14309_gb300 import build
        build.build()
    return abi.lib()


def test_every_declared_symbol_is_exported(lib):
    from paper_2409_14309_gb300 import abi
    names = _declared()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n
    assert names == {s[0] for s in abi.SIGNATURES}


def test_status_strings(lib):
    for code in range(9):
        assert lib.snsolve_status_string(code).decode().startswith("SNS_")
    assert lib.snsolve_status_string(99) == b"SNS_UNKNOWN"
    assert lib.snsolve_version() >= 100


def test_create_without_gpu_fails_loudly(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = C.c_void_p()
    code = lib.snsolve_create(C.byref(h), 0)
    assert code in (2, 1, 7) and not h.value


def _prob(m=1000, n=10, fmt=0, lda=None):
    from paper_2409_14309_gb300 import abi
    return abi.sns_problem(m=m, n=n, fmt=fmt, A=0x1000, lda=lda or n, b=0x2000)


def test_workspace_queries_and_validation(lib):
    from paper_2409_14309_gb300 import abi
    sz = C.c_size_t()
    sk = abi.sns_sketch_desc(kind=0, variant=0, d=40, seed=1)
    assert lib.snsolve_sketch_workspace_size(C.byref(_prob()), C.byref(sk), C.byref(sz)) == 0
    assert sz.value > 0
    # stream variant needs no workspace
    sk2 = abi.sns_sketch_desc(kind=0, variant=2, d=40, seed=1)
    assert lib.snsolve_sketch_workspace_size(C.byref(_prob()), C.byref(sk2), C.byref(sz)) == 0
    assert sz.value == 0
    bad = [
        (_prob(), abi.sns_sketch_desc(kind=0, d=5)),          # d < n
        (_prob(m=5, n=10), sk),                                # m < n
        (_prob(lda=5), sk),                                    # lda < n
        (_prob(fmt=7), sk),                                    # bad format
        (_prob(), abi.sns_sketch_desc(kind=9, d=40)),          # bad kind
        (_prob(fmt=1), abi.sns_sketch_desc(kind=1, d=40)),     # Gaussian needs FP32
        (_prob(m=100), abi.sns_sketch_desc(kind=2, d=200)),    # SRHT d > m'
        (_prob(), abi.sns_sketch_desc(kind=3, variant=9, d=40)),   # sparse sign: zeta > 8
        (_prob(), abi.sns_sketch_desc(kind=3, variant=0, d=40)),   # sparse sign: zeta < 1
        (_prob(n=4), abi.sns_sketch_desc(kind=3, variant=6, d=5)),  # sparse sign: zeta > d
        (_prob(fmt=1), abi.sns_sketch_desc(kind=3, variant=2, d=40)),  # sparse sign needs FP32 dense
    ]
    for p, s in bad:
        assert lib.snsolve_sketch_workspace_size(C.byref(p), C.byref(s), C.byref(sz)) == 1
    # the sparse sign embedding streams: no workspace
    sse = abi.sns_sketch_desc(kind=3, variant=8, d=40, seed=1)
    assert lib.snsolve_sketch_workspace_size(C.byref(_prob()), C.byref(sse), C.byref(sz)) == 0
    assert sz.value == 0
    op = abi.sns_opts(sk=sk, tol=1e-8)
    assert lib.snsolve_lstsq_workspace_size(C.byref(_prob()), C.byref(op), C.byref(sz)) == 0
    with_iter = sz.value
    op0 = abi.sns_opts(sk=sk, tol=0.0)
    assert lib.snsolve_lstsq_workspace_size(C.byref(_prob()), C.byref(op0), C.byref(sz)) == 0
    assert sz.value < with_iter
    # sketch-and-apply: needs room for Y; dense input with a preconditioner only
    op_saa = abi.sns_opts(sk=sk, tol=1e-8, method=abi.SNS_SAA, precondition=1)
    assert lib.snsolve_lstsq_workspace_size(C.byref(_prob()), C.byref(op_saa), C.byref(sz)) == 0
    assert sz.value >= with_iter + 1000 * 12 * 4
    assert lib.snsolve_lstsq_workspace_size(C.byref(_prob()), C.byref(abi.sns_opts(sk=sk, tol=1e-8, method=7)),
                                            C.byref(sz)) == 1
    assert lib.snsolve_lstsq_workspace_size(
        C.byref(_prob()), C.byref(abi.sns_opts(sk=sk, tol=1e-8, method=abi.SNS_SAA, precondition=0)),
        C.byref(sz)) == 1
    csr = abi.sns_problem(m=1000, n=10, fmt=abi.SNS_CSR_F32, rowptr=0x1000, col=0x2000, val=0x3000, nnz=5, b=0x4000)
    assert lib.snsolve_lstsq_workspace_size(C.byref(csr), C.byref(op_saa), C.byref(sz)) == 1
    # null pointers are rejected before anything runs
    assert lib.snsolve_sketch(None, C.byref(_prob()), C.byref(sk), None, 10, None, None, 0, None) == 1
    assert lib.snsolve_lstsq(None, C.byref(_prob()), C.byref(op), None, None, None, 0, None) == 1


def test_gaussian_table_matches_oracle(lib):
    from oracle import sketch as OS
    import paper_2409_14309_gb300 as sns
    bits = np.array(sns.gaussian_table_bits(), dtype=np.uint32)
    lib_vals = (bits << 16).astype(np.uint32).view(np.float32).astype(np.float64)
    assert np.array_equal(lib_vals, OS.gaussian_table())


def test_gaussian_terms_and_solve_defaults(lib):
    """Gaussian variant = BF16 terms of [A | b] (0 = auto, 1..3): out-of-range
    values are refused; split tiles need more workspace; a solve resolves auto
    to three terms, a sketch to one."""
    from paper_2409_14309_gb300 import abi
    sz = C.c_size_t()
    p = _prob(m=100000, n=64)
    ws = {}
    for v in (0, 1, 2, 3):
        sk = abi.sns_sketch_desc(kind=abi.SNS_GAUSSIAN, variant=v, d=256, seed=1)
        assert lib.snsolve_sketch_workspace_size(C.byref(p), C.byref(sk), C.byref(sz)) == 0
        ws[v] = sz.value
    assert ws[0] == ws[1] < ws[2] < ws[3]
    for v in (-1, 4):
        sk = abi.sns_sketch_desc(kind=abi.SNS_GAUSSIAN, variant=v, d=256, seed=1)
        assert lib.snsolve_sketch_workspace_size(C.byref(p), C.byref(sk), C.byref(sz)) == 1
    ls = {}
    for v in (0, 1, 3):
        op = abi.sns_opts(sk=abi.sns_sketch_desc(kind=abi.SNS_GAUSSIAN, variant=v, d=256, seed=1), tol=1e-6)
        assert lib.snsolve_lstsq_workspace_size(C.byref(p), C.byref(op), C.byref(sz)) == 0
        ls[v] = sz.value
    assert ls[0] == ls[3] > ls[1]


def test_csr_reproducible_solve_size_limit(lib):
    """CountSketch variant SORTED on CSR asks for the reproducible solve, whose
    passes keep per-warp rows of n doubles: n up to 1422 is accepted, larger n
    refused; the default variant has no such limit."""
    from paper_2409_14309_gb300 import abi
    sz = C.c_size_t()

    def csr(n):
        return abi.sns_problem(m=100000, n=n, fmt=abi.SNS_CSR_F32, rowptr=0x1000, col=0x2000, val=0x3000,
                               nnz=10, b=0x4000)

    def op(variant, n):
        return abi.sns_opts(sk=abi.sns_sketch_desc(kind=abi.SNS_COUNTSKETCH, variant=variant, d=2 * n, seed=1),
                            tol=1e-8)
    assert lib.snsolve_lstsq_workspace_size(C.byref(csr(1422)), C.byref(op(abi.SNS_CS_SORTED, 1422)),
                                            C.byref(sz)) == 0
    assert lib.snsolve_lstsq_workspace_size(C.byref(csr(1423)), C.byref(op(abi.SNS_CS_SORTED, 1423)),
                                            C.byref(sz)) == 1
    assert lib.snsolve_lstsq_workspace_size(C.byref(csr(1500)), C.byref(op(abi.SNS_CS_AUTO, 1500)),
                                            C.byref(sz)) == 0


def test_srht_workspace_one_pass_form_needs_no_y(lib):
    """FP32 SRHT with m' >= 1024 and d <= 1024 runs in one pass: its workspace
    holds per-CTA partials and sign bits, far less than the transformed copy Y
    (m' x (n + 1) floats) that the two-pass form (d > 1024, FP64) needs."""
    from paper_2409_14309_gb300 import abi
    sz = C.c_size_t()
    m, n = 100000, 64
    mp = 1 << 17
    y_bytes = mp * (n + 4) * 4
    p32 = _prob(m=m, n=n)
    sk = abi.sns_sketch_desc(kind=abi.SNS_SRHT, d=512, seed=1)
    assert lib.snsolve_sketch_workspace_size(C.byref(p32), C.byref(sk), C.byref(sz)) == 0
    assert sz.value < y_bytes
    sk_big = abi.sns_sketch_desc(kind=abi.SNS_SRHT, d=2048, seed=1)
    assert lib.snsolve_sketch_workspace_size(C.byref(p32), C.byref(sk_big), C.byref(sz)) == 0
    assert sz.value >= y_bytes
    p64 = _prob(m=m, n=n, fmt=abi.SNS_DENSE_F64)
    assert lib.snsolve_sketch_workspace_size(C.byref(p64), C.byref(sk), C.byref(sz)) == 0
    assert sz.value >= 2 * y_bytes
