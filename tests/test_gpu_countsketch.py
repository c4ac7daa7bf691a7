"""CountSketch apply on the GPU vs the FP64 oracle (Sec. 1.2.2 sketch; the
paper's default operator).  Bucket ids and signs must match bit for bit; SA and
Sb within ||SA_gpu - SA_ref||_F / ||[A | b]||_F <= 1e-6 for FP32 data (1e-13
for FP64 data); the sorted variant must be bitwise reproducible."""
import numpy as np
import pytest
import torch

from gpu_util import ctx, dev, rel_fro
from oracle import hashing as OH
from oracle import sketch as OS
from synth import csr_problem, gaussian_problem, ill_conditioned_problem

pytestmark = pytest.mark.gpu

TOL32 = 1e-6


@pytest.mark.parametrize("m,d", [(1, 1), (33, 7), (5000, 1024), (100003, 2048), (70000, 8192)])
def test_hash_bit_exact(m, d):
    c = ctx()
    for seed in (0, 1, 2**63 + 5):
        h, s = c.countsketch_hash(m, d, seed)
        hr, sr = OH.countsketch_hash(seed, m, d)
        assert np.array_equal(h.cpu().numpy().astype(np.int64), hr)
        assert np.array_equal(s.cpu().numpy().astype(np.float64), sr)


def test_stream_keys_bit_exact():
    c = ctx()
    for stream in (0, 1, 2, 3):
        k = c.stream_keys(1234567, stream, 10, 1000).cpu().numpy().view(np.uint64)
        kr = OH.splitmix64_at(OH.stream_state(1234567, stream), np.arange(10, 1010, dtype=np.uint64))
        assert np.array_equal(k, kr)


CASES = [  # m, n, d, lda_pad
    (1, 1, 1, 0), (31, 7, 7, 0), (33, 7, 28, 3), (4097, 64, 256, 0), (12305, 257, 1028, 0),
    (9000, 128, 512, 4), (20000, 300, 1200, 0), (4096, 3, 5, 1), (50000, 16, 64, 0), (6000, 64, 1500, 0),
    (300001, 36, 144, 0),
]


@pytest.mark.parametrize("variant", ["sorted", "stream"])
@pytest.mark.parametrize("m,n,d,pad", CASES)
def test_countsketch_dense_f32(variant, m, n, d, pad):
    c = ctx()
    rng = np.random.default_rng(m * 7 + n)
    Afull = rng.standard_normal((m, n + pad)).astype(np.float32)
    b = rng.standard_normal(m).astype(np.float32)
    Ad = dev(Afull)[:, :n]
    SA, Sb = c.sketch(Ad, dev(b), d, seed=m, variant=variant)
    A = Afull[:, :n]
    scale = np.sqrt(np.linalg.norm(A.astype(np.float64)) ** 2 + np.linalg.norm(b.astype(np.float64)) ** 2)
    assert rel_fro(SA.cpu().numpy(), OS.countsketch_apply(A, d, m), scale) <= TOL32
    assert rel_fro(Sb.cpu().numpy(), OS.countsketch_apply(b, d, m), scale) <= TOL32


@pytest.mark.parametrize("m,n,d", [(1, 1, 1), (4097, 64, 256), (9001, 33, 100)])
def test_countsketch_dense_f64(m, n, d):
    c = ctx()
    A, b, _ = gaussian_problem(m, n, seed=m)
    SA, Sb = c.sketch(dev(A), dev(b), d, seed=3)
    scale = np.linalg.norm(np.column_stack([A, b]))
    assert rel_fro(SA.cpu().numpy(), OS.countsketch_apply(A, d, 3), scale) <= 1e-14
    assert rel_fro(Sb.cpu().numpy(), OS.countsketch_apply(b, d, 3), scale) <= 1e-14


@pytest.mark.parametrize("m,n,d", [(5, 4, 4), (4096, 64, 256), (1048577, 256, 1024), (300001, 36, 8192)])
def test_single_launch_plan_equals_two_kernel_plan(m, n, d):
    """The deterministic CountSketch's plan (hash, stable per-block bucket
    order, bucket-major row list) runs as one cooperative launch in
    snsolve_sketch and as two plain kernels in the allocation-free entry point;
    both feed the same gather, so SA and Sb must agree bit for bit."""
    import ctypes as C
    import paper_2409_14309_gb300 as sns
    from paper_2409_14309_gb300 import abi
    c = ctx()
    g = torch.Generator(device="cuda")
    g.manual_seed(m + d)
    A = torch.randn(m, n, generator=g, device="cuda")
    b = torch.randn(m, generator=g, device="cuda")
    SA, Sb = c.sketch(A, b, d, seed=4, variant="sorted")
    SA2 = torch.full_like(SA, float("nan"))
    Sb2 = torch.full_like(Sb, float("nan"))
    prob = sns.dense_problem(A, b)
    code = abi.lib().snsolve_sketch_countsketch_static(
        C.byref(prob), d, 4, C.c_void_p(SA2.data_ptr()), n, C.c_void_p(Sb2.data_ptr()),
        C.c_void_p(torch.cuda.current_stream().cuda_stream))
    if code == abi.SNS_ENOMEM:
        pytest.skip("problem larger than the fixed scratch of the allocation-free entry point")
    assert code == 0
    torch.cuda.synchronize()
    assert torch.equal(SA, SA2) and torch.equal(Sb, Sb2)


def test_countsketch_many_plan_blocks():
    """2^22 + 5 rows: 1025 plan blocks, all co-resident in the cooperative plan."""
    c = ctx()
    m, n, d = (1 << 22) + 5, 8, 1024
    rng = np.random.default_rng(12)
    A = rng.standard_normal((m, n)).astype(np.float32)
    b = rng.standard_normal(m).astype(np.float32)
    SA, Sb = c.sketch(dev(A), dev(b), d, seed=6, variant="sorted")
    scale = np.sqrt(np.linalg.norm(A.astype(np.float64)) ** 2 + np.linalg.norm(b.astype(np.float64)) ** 2)
    assert rel_fro(SA.cpu().numpy(), OS.countsketch_apply(A, d, 6), scale) <= TOL32
    assert rel_fro(Sb.cpu().numpy(), OS.countsketch_apply(b, d, 6), scale) <= TOL32


def test_sorted_variant_bitwise_reproducible():
    c = ctx()
    rng = np.random.default_rng(5)
    A = dev(rng.standard_normal((60000, 96)).astype(np.float32))
    b = dev(rng.standard_normal(60000).astype(np.float32))
    r1 = c.sketch(A, b, 384, seed=9, variant="sorted")
    r2 = c.sketch(A, b, 384, seed=9, variant="sorted")
    assert torch.equal(r1[0], r2[0]) and torch.equal(r1[1], r2[1])


@pytest.mark.parametrize("variant", ["auto", "sorted", "stream"])
@pytest.mark.parametrize("m,n,d,dens", [(1, 1, 1, 1.0), (5000, 40, 160, 0.05), (70001, 512, 2048, 0.01)])
def test_countsketch_csr(m, n, d, dens, variant):
    c = ctx()
    A, b, _ = csr_problem(m, n, seed=m, density=dens, n_dense=min(8, m))
    SA, Sb = c.sketch_csr(dev(A.rowptr), dev(A.col), dev(A.val), dev(b), n, d, seed=4, variant=variant)
    ref = OS.countsketch_apply_csr(A.rowptr, A.col, A.val, n, d, 4)
    scale = np.sqrt(np.sum(A.val.astype(np.float64) ** 2) + np.sum(b.astype(np.float64) ** 2))
    assert rel_fro(SA.cpu().numpy(), ref, scale) <= TOL32
    assert rel_fro(Sb.cpu().numpy(), OS.countsketch_apply(b, d, 4), scale) <= TOL32


def test_csr_sorted_bitwise_reproducible():
    """The sorted CSR sketch adds every bucket's rows in a fixed order:
    repeated and concurrent sketches are equal bit for bit."""
    c = ctx()
    A, b, _ = csr_problem(150000, 256, seed=8, density=0.03, n_dense=16)
    args = (dev(A.rowptr), dev(A.col), dev(A.val), dev(b), 256, 1024)
    SA1, Sb1 = c.sketch_csr(*args, seed=6, variant="sorted")
    outs = []
    for s in (torch.cuda.Stream(), torch.cuda.Stream()):
        with torch.cuda.stream(s):
            outs.append(c.sketch_csr(*args, seed=6, variant="sorted", stream=s))
    torch.cuda.synchronize()
    for SA, Sb in outs:
        assert torch.equal(SA, SA1) and torch.equal(Sb, Sb1)


@pytest.mark.slow
@pytest.mark.parametrize("variant", ["sorted", "stream"])
def test_full_size_ill_conditioned_sampled_rows(variant):
    """2^20 x 256 FP32, d = 1024, the benchmark's launch configuration: sampled
    output rows against the oracle's per-row definition."""
    c = ctx()
    A, b, _ = ill_conditioned_problem(1 << 20, 256, seed=1002, kappa=1e6, noise=1e-4)
    SA, Sb = c.sketch(dev(A), dev(b), 1024, seed=1, variant=variant)
    rows = [0, 1, 17, 511, 512, 1000, 1023]
    ref = OS.countsketch_rows(A, 1024, 1, rows)
    refb = OS.countsketch_rows(b, 1024, 1, rows)
    SAh = SA.cpu().numpy()
    Sbh = Sb.cpu().numpy()
    scale = np.linalg.norm(ref)
    assert rel_fro(SAh[rows], ref, scale) <= TOL32
    assert rel_fro(Sbh[rows], refb, np.linalg.norm(refb)) <= TOL32
    # property that holds at any size: ||SA||_F^2 + ||Sb||^2 close to ||[A|b]||_F^2 (E[S^T S] = I)
    tot = np.linalg.norm(SAh.astype(np.float64)) ** 2 + np.linalg.norm(Sbh.astype(np.float64)) ** 2
    ref_tot = np.linalg.norm(A.astype(np.float64)) ** 2 + np.linalg.norm(b.astype(np.float64)) ** 2
    assert abs(tot / ref_tot - 1) < 0.2


def test_bulk_copy_pipeline_variant_in_subprocess():
    """The alternative phase-2 kernel (bulk-copy ring, selected by the
    SNSOLVE_CS_GATHER=tma environment variable read once per process) against
    the oracle on shapes with one and two column tiles and split buckets."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    code = r'''
import sys, numpy as np, torch
sys.path.insert(0, ".")
import paper_2409_14309_gb300 as sns
from oracle import sketch as OS
c = sns.Context(0)
worst = 0.0
for (m, n, d) in [(70001, 64, 256), (20000, 300, 1200), (300000, 128, 256)]:
    rng = np.random.default_rng(m)
    A = rng.standard_normal((m, n)).astype(np.float32); b = rng.standard_normal(m).astype(np.float32)
    SA, Sb = c.sketch(torch.from_numpy(A).cuda(), torch.from_numpy(b).cuda(), d, seed=5, variant="sorted")
    scale = np.sqrt(np.linalg.norm(A.astype(np.float64))**2 + np.linalg.norm(b.astype(np.float64))**2)
    e = max(np.linalg.norm(SA.cpu().numpy() - OS.countsketch_apply(A, d, 5)),
            np.linalg.norm(Sb.cpu().numpy() - OS.countsketch_apply(b, d, 5))) / scale
    worst = max(worst, e)
print("WORST", worst)
'''
    env = dict(os.environ, SNSOLVE_CS_GATHER="tma")
    r = subprocess.run([sys.executable, "-c", code], cwd=root, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    worst = float(r.stdout.split("WORST")[1])
    assert worst <= TOL32


@pytest.mark.parametrize("variant", ["sorted", "stream"])
@pytest.mark.parametrize("m,n,d", [(100, 64, 1000), (22271, 128, 4096), (5000, 300, 8192)])
def test_empty_buckets_are_written_as_zero(variant, m, n, d):
    """d comparable to or above m leaves buckets no row hashes to: their SA rows
    and Sb entries must come out as zeros, whatever the output buffers held."""
    import ctypes as C
    import paper_2409_14309_gb300 as sns
    c = ctx()
    rng = np.random.default_rng(m + d)
    A = rng.standard_normal((m, n)).astype(np.float32)
    b = rng.standard_normal(m).astype(np.float32)
    Ad, bd = dev(A), dev(b)
    prob = sns.dense_problem(Ad, bd)
    sk = sns.sketch_desc(d, "countsketch", 9, variant)
    SA = torch.full((d, n), float("nan"), device="cuda")
    Sb = torch.full((d,), float("nan"), device="cuda")
    ws = torch.empty(max(c.sketch_workspace(prob, sk), 256), dtype=torch.uint8, device="cuda")
    code = c._L.snsolve_sketch(c.h, C.byref(prob), C.byref(sk), C.c_void_p(SA.data_ptr()), n,
                               C.c_void_p(Sb.data_ptr()), C.c_void_p(ws.data_ptr()), ws.numel(), None)
    assert code == 0
    torch.cuda.synchronize()
    h, _ = OH.countsketch_hash(9, m, d)
    assert len(set(range(d)) - set(h.tolist())) > 0            # there are empty buckets
    scale = np.sqrt(np.linalg.norm(A.astype(np.float64)) ** 2 + np.linalg.norm(b.astype(np.float64)) ** 2)
    assert np.isfinite(SA.cpu().numpy()).all() and np.isfinite(Sb.cpu().numpy()).all()
    assert rel_fro(SA.cpu().numpy(), OS.countsketch_apply(A, d, 9), scale) <= TOL32
    assert rel_fro(Sb.cpu().numpy(), OS.countsketch_apply(b, d, 9), scale) <= TOL32


@pytest.mark.parametrize("terms", [1, 2, 3])
@pytest.mark.parametrize("m,n,d", [(777, 1, 5), (3000, 20, 80), (20000, 100, 333), (50000, 256, 1024),
                                   (10000, 300, 1200), (4133, 257, 300)])
def test_gaussian_sketch_tensor_core(m, n, d, terms):
    """Gaussian sketch on the tensor cores (BF16 G and [A | b] as `terms` BF16
    terms, FP32 accumulation) against the oracle's FP64 product of the same
    operands (terms = 3: the FP32 values themselves).  The values span
    exponents so that the lower terms matter."""
    c = ctx()
    rng = np.random.default_rng(m + n)
    A = (rng.standard_normal((m, n)) * np.exp(rng.uniform(-3, 3, (m, n)))).astype(np.float32)
    b = rng.standard_normal(m).astype(np.float32)
    SA, Sb = c.sketch(dev(A), dev(b), d, kind="gaussian", seed=13, variant=str(terms))
    ref = OS.gaussian_apply(A, d, 13, terms=terms)
    refb = OS.gaussian_apply(b, d, 13, terms=terms)
    scale = np.sqrt(np.linalg.norm(ref) ** 2 + np.linalg.norm(refb) ** 2)
    assert rel_fro(SA.cpu().numpy(), ref, scale) <= 1e-6
    assert rel_fro(Sb.cpu().numpy(), refb, scale) <= 1e-6
    if terms == 3:   # and it is a different product from the one-term sketch
        one = OS.gaussian_apply(A, d, 13, terms=1)
        assert rel_fro(one, ref, scale) > 1e-4


def test_gaussian_three_terms_reproducible_and_auto_is_one_term():
    c = ctx()
    rng = np.random.default_rng(92)
    A = dev(rng.standard_normal((70000, 96)).astype(np.float32))
    b = dev(rng.standard_normal(70000).astype(np.float32))
    SA1, Sb1 = c.sketch(A, b, 384, kind="gaussian", seed=5, variant="3")
    outs = []
    for s in (torch.cuda.Stream(), torch.cuda.Stream()):
        with torch.cuda.stream(s):
            outs.append(c.sketch(A, b, 384, kind="gaussian", seed=5, variant="3", stream=s))
    torch.cuda.synchronize()
    for SA, Sb in outs:
        assert torch.equal(SA, SA1) and torch.equal(Sb, Sb1)
    SAa, Sba = c.sketch(A, b, 384, kind="gaussian", seed=5)
    SAo, Sbo = c.sketch(A, b, 384, kind="gaussian", seed=5, variant="1")
    assert torch.equal(SAa, SAo) and torch.equal(Sba, Sbo)
    with pytest.raises(RuntimeError):
        c.sketch(A, b, 384, kind="gaussian", seed=5, variant="4")


def test_gaussian_sketch_bitwise_reproducible():
    """The tensor-core Gaussian sketch adds its K splits' partial tiles in a
    fixed order: repeated sketches, including ones that overlap on two streams
    (so the CTAs finish in a different order), are equal bit for bit."""
    c = ctx()
    rng = np.random.default_rng(91)
    A = dev(rng.standard_normal((120000, 160)).astype(np.float32))
    b = dev(rng.standard_normal(120000).astype(np.float32))
    SA1, Sb1 = c.sketch(A, b, 640, kind="gaussian", seed=5)
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    outs = []
    for s in (s1, s2):
        with torch.cuda.stream(s):
            outs.append(c.sketch(A, b, 640, kind="gaussian", seed=5, stream=s))
    torch.cuda.synchronize()
    for SA, Sb in outs:
        assert torch.equal(SA, SA1) and torch.equal(Sb, Sb1)


def test_gaussian_simt_variant_in_subprocess():
    """The CUDA-core Gaussian kernel (SNSOLVE_GAUSS=simt) follows the same
    definition of G as the tensor-core kernel."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    code = r'''
import sys, numpy as np, torch
sys.path.insert(0, ".")
import paper_2409_14309_gb300 as sns
from oracle import sketch as OS
c = sns.Context(0)
worst = 0.0
for (m, n, d) in [(3000, 20, 80), (20000, 100, 333)]:
    rng = np.random.default_rng(m + n)
    A = rng.standard_normal((m, n)).astype(np.float32); b = rng.standard_normal(m).astype(np.float32)
    SA, Sb = c.sketch(torch.from_numpy(A).cuda(), torch.from_numpy(b).cuda(), d, kind="gaussian", seed=13)
    ref = OS.gaussian_apply(A, d, 13); refb = OS.gaussian_apply(b, d, 13)
    scale = np.sqrt(np.linalg.norm(ref)**2 + np.linalg.norm(refb)**2)
    worst = max(worst, np.linalg.norm(SA.cpu().numpy() - ref) / scale, np.linalg.norm(Sb.cpu().numpy() - refb) / scale)
print("WORST", worst)
'''
    env = dict(os.environ, SNSOLVE_GAUSS="simt")
    r = subprocess.run([sys.executable, "-c", code], cwd=root, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    assert float(r.stdout.split("WORST")[1]) <= 1e-5
