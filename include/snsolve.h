/*
 * snsolve.h -- C ABI of a GB300 (sm_103a) library for randomized least squares
 * by sketch-and-solve and sketch-and-precondition.
 *
 * Problem (Eq. 1 of "Sketch 'n Solve", arXiv 2409.14309, Sec. 1.3):
 *     min_x || A x - b ||_2^2,   A in R^{m x n}, b in R^m, m >> n.
 * Sketch-and-solve (Sec. 1.2 steps 1-3 and the reduced problem of Sec. 1.3):
 * draw S in R^{d x m} (d >= n), form SA and Sb, and solve
 *     min_x^ || SA x^ - Sb ||_2^2
 * by an FP64 Householder QR of [SA | Sb] and back substitution.
 * Sketch-and-precondition (SAP-SAS, Sec. 2.1): when a tolerance below what
 * sketch-and-solve reaches is asked for, R from that QR right-preconditions an
 * iterative solve on the original A, started from x^.
 *
 * Conventions shared by every entry point:
 *  - Matrix and vector arguments are DEVICE pointers owned by the caller
 *    (unless stated otherwise).  Dense matrices are row-major with a leading
 *    dimension in elements.
 *  - Work is enqueued on the caller's `stream` (a cudaStream_t passed as
 *    void*; NULL means the legacy default stream).  Argument errors are
 *    returned synchronously before anything is launched.
 *  - The library allocates no device memory on any compute path: scratch is a
 *    caller-provided workspace whose size comes from the matching *_size query.
 *    A workspace must be 256-byte aligned.
 *  - There is no CPU fallback: every arithmetic step runs in this library's
 *    CUDA kernels.  A missing or non-sm_103a device yields SNS_ECUDA.
 *  - Functions are thread-safe for distinct contexts; one context may be used
 *    from several threads if each call uses its own stream and workspace.
 */
#ifndef SNSOLVE_H
#define SNSOLVE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes returned by every call and stored in sns_info.status. */
typedef enum {
  SNS_OK = 0,
  SNS_EINVAL = 1,    /* invalid argument (shape, pointer, alignment, option) */
  SNS_ENOMEM = 2,    /* workspace too small / server pool exhausted */
  SNS_ERANK = 3,     /* |R_jj| <= n * 2^-53 * max_i |R_ii| in the QR of SA */
  SNS_ENOTCONV = 4,  /* iteration cap reached before the tolerance */
  SNS_EAGAIN = 5,    /* request not finished yet (poll) */
  SNS_ETIMEOUT = 6,  /* bounded wait expired (poll, or a device-side wait) */
  SNS_ECUDA = 7,     /* CUDA runtime error; see snsolve_last_cuda_error */
  SNS_EBUDGET = 8    /* one request alone exceeds the server's HBM budget */
} sns_status;

/* Sketch families (Sec. 1.2.1 dense: Gaussian, Hadamard; Sec. 1.2.2 sparse:
 * Clarkson-Woodruff, the paper's default). */
typedef enum {
  SNS_COUNTSKETCH = 0,  /* S[h(i), i] = s(i): one signed nonzero per column */
  SNS_GAUSSIAN = 1,     /* S = G / sqrt(d), G from a BF16 normal-quantile table */
  SNS_SRHT = 2,         /* S = P H D / sqrt(d) on m' = 2^ceil(log2 m) rows */
  SNS_SPARSE_SIGN = 3   /* zeta nonzeros +-1/sqrt(zeta) per column at distinct rows (Sec. 1.2.2,
                           after Martinsson & Tropp 2020); zeta = variant, 1..min(8, d); dense FP32
                           only; one streaming pass with float reductions (order varies) */
} sns_sketch_kind;

/* Storage of A (one entry point serves dense and sparse A, Sec. 2.1). */
typedef enum {
  SNS_DENSE_F32 = 0,    /* A float, row-major, lda >= n; b float */
  SNS_DENSE_F64 = 1,    /* A double, row-major, lda >= n; b double */
  SNS_CSR_F32 = 2       /* CSR: rowptr int64[m+1], col int32[nnz], val float[nnz]; b float */
} sns_format;

/* CountSketch variants. */
typedef enum {
  SNS_CS_AUTO = 0,          /* library picks: FP32 dense -> SORTED while d <= 8192, else STREAM;
                               FP64 dense -> SORTED; CSR -> STREAM */
  SNS_CS_SORTED = 1,        /* bucket-sorted segmented sum: bitwise reproducible (dense; CSR with
                               d <= 8192 and n <= 6399, SNS_EINVAL beyond).  On CSR it also makes
                               snsolve_lstsq's iterative passes reproducible (n <= 1422; about
                               2.5x slower per pass than the default) */
  SNS_CS_STREAM = 2         /* one streaming pass with float reductions into SA (FP32 dense, CSR;
                               order of additions varies run to run) */
} sns_cs_variant;

/* Implicit sketch descriptor.  S is never stored: its entries are functions of
 * (seed, row index) through the SplitMix64 counter-based stream (Steele, Lea &
 * Flood 2014): output i of stream t is mix64((seed ^ (t << 56)) + (i+1)*gamma).
 * CountSketch (t = 0): h(i) = ((k mod 2^32) * d) >> 32, s(i) = bit 63 ? -1 : +1.
 * SRHT: signs from t = 1, d distinct rows of [0, m') by Floyd's algorithm on t = 2.
 * Gaussian: G[k, i] = T[byte (i mod 8) of output (i div 8)*d + k of t = 3],
 * T[j] = BF16(Phi^-1((j + 1/2)/256)).
 * Sparse sign: draw z of column i uses output i of t = 0 (z = 0; zeta = 1 is the
 * CountSketch) or output i*(zeta-1) + z-1 of t = 4; rows by Floyd's algorithm on
 * [0, d): u = ((k mod 2^32)*(J+1)) >> 32 with J = d - zeta + z, or J if an earlier
 * draw of the column took u; the sign of draw z is bit 63 of its key. */
typedef struct {
  int32_t kind;        /* sns_sketch_kind */
  int32_t variant;     /* sns_cs_variant for CountSketch; zeta for SNS_SPARSE_SIGN; for SNS_GAUSSIAN
                          the BF16 terms [A | b] is split into for the tensor cores: 1 = rounded to
                          BF16 (fastest), 2 = 16 significant bits, 3 = the FP32 values exactly;
                          0 = auto: 1 in snsolve_sketch*, 3 in snsolve_lstsq and the server (a
                          one-term R preconditions ill-conditioned A poorly); ignored otherwise */
  int64_t d;           /* sketch rows, n <= d; SRHT also d <= m' */
  uint64_t seed;
} sns_sketch_desc;

/* One least-squares problem. */
typedef struct {
  int64_t m, n;
  int32_t fmt;             /* sns_format */
  int32_t reserved;
  const void* A;           /* dense: m x n row-major, leading dimension lda */
  int64_t lda;
  const int64_t* rowptr;   /* CSR only */
  const int32_t* col;      /* CSR only, each in [0, n) */
  const float* val;        /* CSR only */
  int64_t nnz;             /* CSR only: rowptr[m] */
  const void* b;           /* m entries, float (F32, CSR) or double (F64) */
} sns_problem;

/* Solve options. tol <= 0: sketch-and-solve only.  tol > 0: after
 * sketch-and-solve, eta(x) = ||A^T r|| / (||A||_F ||r||), r = b - A x, is
 * computed with FP64-class accumulation; while eta > tol the solver runs
 * R-preconditioned refinement steps (SAP-SAS) up to max_iter FP32 passes. */
typedef struct {
  sns_sketch_desc sk;
  double tol;
  int32_t max_iter;        /* cap on inner passes over A (0 = library default 400) */
  int32_t inner;           /* most inner CG steps per refinement step (0 = default 8); a step
                              ends earlier, on the device, once the preconditioned CG residual
                              has dropped by max(tol / (2 eta), 4e-3), eta the current backward
                              error (Sec. 1.2 sketch-and-precondition; the per-step floor reflects
                              the FP32 passes) */
  int32_t precondition;    /* 1 = R from QR(SA) (default when nonzero); 0 = R = I
                              (unpreconditioned reference iteration) */
  int32_t method;          /* sns_method: how R enters the iteration when tol > 0 */
} sns_opts;

/* Iterative phase (Sec. 2.1 names both, after Meier, Nakatsukasa, Townsend &
 * Webb 2023).  Both start from the sketch-and-solve answer and stop at
 * eta(x) <= tol; the residual passes r = b - A x always read the original A.
 *  SNS_SAP (sketch-and-precondition): the inner iteration applies R^-1
 *    implicitly: each pass reads A (w = A^T A z with z = R^-1 p).
 *  SNS_SAA (sketch-and-apply): Y = A R^-1 is formed once, explicitly, in A's
 *    precision (m x n extra workspace), and the inner iteration (CG on
 *    Y^T Y dz = R^-T A^T r, i.e. CGLS/LSQR on Y) reads Y; x += R^-1 dz.
 *    Dense input only, precondition must be nonzero. */
typedef enum { SNS_SAP = 0, SNS_SAA = 1 } sns_method;

/* Per-solve report. */
typedef struct {
  int32_t status;          /* sns_status of the solve */
  int32_t iters;           /* inner passes over A (FP32 normal-equation passes) */
  int32_t outer;           /* FP64-class residual passes */
  int32_t reserved;
  double eta;              /* final eta(x) (tol > 0), else 0 */
  double resid_norm;       /* ||b - A x|| (tol > 0), else 0 */
  double sketch_resid;     /* ||SA x^ - Sb|| from the QR: |R_aug[n, n]| */
  float ms_sketch;         /* snsolve_lstsq: device time of the sketch (CUDA events on the */
  float ms_qr;             /*   call's stream), of the QR + back-solve, and of everything */
  float ms_iter;           /*   after it (refinement); 0 where a phase did not run or in   */
  int32_t reserved2;       /*   snsolve_lstsq_batched */
} sns_info;

typedef struct sns_ctx sns_ctx;

/* Create a context on CUDA device `device`.  Checks that the device is
 * sm_103 and that the library's kernels load.  *ctx is NULL on failure. */
sns_status snsolve_create(sns_ctx** ctx, int device);
void snsolve_destroy(sns_ctx* ctx);

/* Human-readable name of a status code (static storage). */
const char* snsolve_status_string(int status);
/* Last CUDA error string seen by this thread (static thread-local storage). */
const char* snsolve_last_cuda_error(void);
/* Library version as MAJOR*10000 + MINOR*100 + PATCH. */
int snsolve_version(void);

/* ---- Step 2 of the paradigm (Sec. 1.2): SA and Sb -------------------------
 * Workspace bytes needed by snsolve_sketch for this problem and sketch. */
sns_status snsolve_sketch_workspace_size(const sns_problem* prob, const sns_sketch_desc* sk,
                                         size_t* bytes);

/* SA = S A (d x n, row-major, leading dimension ldsa >= n) and Sb = S b
 * (d entries).  SA and Sb are float for F32/CSR input and double for F64 input.
 * Gaussian sketches multiply [A | b] as 1-3 BF16 terms (sk->variant) in the
 * tensor cores with FP32 accumulation (F32 input only).  Asynchronous on `stream`.
 * Two sketch kernels wait on the device (the tensor-core Gaussian sketch and
 * the bulk-copy CountSketch gather, selected by SNSOLVE_CS_GATHER=t); their
 * waits are bounded, and one that gives up leaves SA/Sb incomplete and an
 * error word in the workspace: snsolve_sketch_status reads it. */
sns_status snsolve_sketch(sns_ctx* ctx, const sns_problem* prob, const sns_sketch_desc* sk,
                          void* SA, int64_t ldsa, void* Sb,
                          void* ws, size_t ws_bytes, void* stream);

/* Outcome of the device-side waits of the last snsolve_sketch call made with
 * this (prob, sk, ws): synchronizes `stream`, then returns SNS_ETIMEOUT if a
 * bounded wait of that call gave up (its SA/Sb are then invalid) and SNS_OK
 * otherwise (also for sketch kinds that never wait on the device).  The word
 * lives in the workspace, so call this before the workspace is reused.
 * SNS_EINVAL for invalid arguments, SNS_ECUDA if the synchronization fails. */
sns_status snsolve_sketch_status(const sns_problem* prob, const sns_sketch_desc* sk, const void* ws,
                                 size_t ws_bytes, void* stream);

/* ---- Rows of a larger matrix (row-sharded sketching) ------------------------
 * Sketch of rows row0 .. row0 + m - 1 of a larger matrix [A_full | b_full]
 * whose rows are split over several calls (or several GPUs): every row keeps
 * its global index i, so S's column i is the same as in a sketch of the whole
 * matrix, and S [A_full | b_full] is the sum of the parts' outputs (one sum,
 * e.g. an all-reduce of the d x (n+1) partials).  prob describes the local
 * rows (prob->m of them); the rest is as in snsolve_sketch.  CountSketch (all
 * variants), Gaussian (row0 a multiple of 8: one hash serves 8 consecutive
 * rows) and sparse sign sketches; SRHT mixes all rows through its Hadamard
 * transform and is rejected (SNS_EINVAL), as is row0 < 0. */
sns_status snsolve_sketch_rows(sns_ctx* ctx, const sns_problem* prob, const sns_sketch_desc* sk, int64_t row0,
                               void* SA, int64_t ldsa, void* Sb, void* ws, size_t ws_bytes, void* stream);

/* Step 3 of Sec. 1.2 on a sketch the caller already holds (for example the
 * sum of row-sharded partial sketches): FP64 Householder QR of the augmented
 * [SA | Sb] (d x (n+1), row-major with leading dimension ld >= n + 1, FP32 if
 * f64 == 0, else FP64; device) and x^ = R^-1 z into x (n doubles, device).
 * info (host, may be NULL) gets the status and ||SA x^ - Sb||.  Synchronizes
 * `stream`.  Returns SNS_ERANK on rank deficiency, SNS_ETIMEOUT if a bounded
 * wait of the multi-CTA QR gave up. */
sns_status snsolve_solve_sketched_workspace_size(int64_t d, int64_t n, size_t* bytes);
sns_status snsolve_solve_sketched(sns_ctx* ctx, const void* SAaug, int64_t ld, int32_t f64, int64_t d, int64_t n,
                                  double* x, sns_info* info, void* ws, size_t ws_bytes, void* stream);

/* ---- Step 3 (Sec. 1.2) and SAP-SAS (Sec. 2.1) ------------------------------
 * Workspace bytes for snsolve_lstsq. */
sns_status snsolve_lstsq_workspace_size(const sns_problem* prob, const sns_opts* opts,
                                        size_t* bytes);

/* Least-squares solve.  x: n doubles (device).  info: HOST pointer, filled
 * before return.  With tol <= 0 the call is asynchronous except that it waits
 * for the QR's rank check; with tol > 0 it synchronizes `stream` between
 * refinement steps (convergence scalars are computed on the device and read
 * from pinned memory).  Returns the same status as info->status: SNS_ERANK
 * from the QR's rank check, SNS_ETIMEOUT when a bounded device-side wait of
 * the sketch (tcgen05 Gaussian, bulk-copy CountSketch) or of the cooperative
 * QR expired (nothing of the solve is then valid), SNS_ENOTCONV at the
 * iteration cap. */
sns_status snsolve_lstsq(sns_ctx* ctx, const sns_problem* prob, const sns_opts* opts,
                         double* x, sns_info* info, void* ws, size_t ws_bytes, void* stream);

/* ---- Batched sketch-and-solve ----------------------------------------------
 * nprob independent dense F32 problems (each d = opts[i].sk.d, CountSketch),
 * solved by one fused persistent launch per stage (sketch, QR, back-solve)
 * that is captured once into a CUDA graph and replayed.  probs, opts, x and
 * infos are HOST arrays of length nprob; x[i] is a device pointer to n_i
 * doubles; infos may be NULL.  Synchronizes `stream` before returning. */
sns_status snsolve_lstsq_batched_workspace_size(const sns_problem* probs, const sns_opts* opts,
                                                int nprob, size_t* bytes);
sns_status snsolve_lstsq_batched(sns_ctx* ctx, const sns_problem* probs, const sns_opts* opts,
                                 int nprob, double* const* x, sns_info* infos,
                                 void* ws, size_t ws_bytes, void* stream);

/* ---- Serving: continuous batching of requests on one GPU --------------------
 * A server owns a device workspace arena (a quarter of hbm_budget_bytes, at
 * most 32 GiB, allocated here once; nothing is allocated while serving) and
 * max_slots worker threads, each with its own stream.  A request's footprint
 * is the bytes of its inputs (A and b, resident on the device and owned by the
 * caller) plus its solver workspace.  A free slot takes the oldest pending
 * request that fits (the admitted footprints sum to at most the budget and
 * the arena has room), so a request waiting for memory does not block smaller
 * ones behind it; the oldest request is passed over at most 2 x max_slots
 * times, then nothing overtakes it until it is admitted.  Admitted requests
 * run concurrently (their kernels overlap on the device) and each starts as
 * soon as a slot and memory free up.
 * Each request is solved exactly as snsolve_lstsq would solve it.  Problem
 * pointers given to submit must stay valid until the request is polled done. */
typedef struct sns_server sns_server;
sns_status snsolve_server_create(sns_server** srv, sns_ctx* ctx, size_t hbm_budget_bytes,
                                 int max_slots);
/* Waits for running requests, then frees the arena; pending ones are dropped. */
void snsolve_server_destroy(sns_server* srv);
/* Queue a request; x is a device pointer to n doubles.  Returns at once.
 * SNS_EBUDGET when the request's footprint alone exceeds the budget (or its
 * workspace exceeds the arena); SNS_EINVAL for invalid arguments. */
sns_status snsolve_submit(sns_server* srv, const sns_problem* prob, const sns_opts* opts,
                          double* x, uint64_t* req_id);
/* SNS_OK with *info filled (info->status is the solve's status) once the
 * request is done; the id is then forgotten.  If it is not done: SNS_EAGAIN
 * when timeout_us == 0, otherwise SNS_ETIMEOUT after waiting timeout_us
 * microseconds.  SNS_EINVAL for an unknown or already collected id. */
sns_status snsolve_poll(sns_server* srv, uint64_t req_id, int64_t timeout_us, sns_info* info);
/* Requests running now, requests waiting for admission, and the footprint
 * bytes admitted (any pointer may be NULL). */
sns_status snsolve_server_stats(sns_server* srv, int* running, int* pending, size_t* used_bytes);

/* ---- CountSketch without any allocation ------------------------------------
 * The paper has no counterpart to this entry point; it exists for callers that
 * cannot allocate device memory at the time they need a sketch (for example
 * code inside a host callback or another library's critical section, or a
 * process whose device memory is fully reserved up front), and so cannot
 * provide the workspace snsolve_sketch asks for.
 *
 * Computes SA = S A (d x n FP32, row-major, leading dimension ldsa >= n) and
 * Sb = S b (d floats) for a dense FP32 problem with the deterministic
 * bucket-sorted CountSketch (the same kernels and results as snsolve_sketch
 * with kind SNS_COUNTSKETCH and variant SNS_CS_SORTED; always the warp gather,
 * which has no device-side waits, so there is no timeout status to read
 * afterwards).  Its scratch is a fixed
 * 16 MiB array inside the library's device image, held by every GPU that loads
 * the library until the process exits; no memory is allocated or freed.
 * Problems whose scratch need exceeds 16 MiB (roughly 8 bytes per row of A plus
 * 4*d bytes per 4096 rows, plus partial rows when buckets are split: about
 * 1.2 million rows at n = 256, d = 1024) are rejected with SNS_ENOMEM before
 * anything is launched.  SNS_EINVAL for other
 * invalid arguments (non-FP32 input, d < n, d > 8192, null pointers).
 *
 * The first call on a device looks up the scratch's device address with that
 * device current; make that first call before any stream capture.  All calls
 * in the process share the one array: calls whose work overlaps on the GPU
 * (different streams, or different host threads) race and corrupt each
 * other's results, so serialize them.  The array keeps the last call's
 * contents; the kernels rewrite everything they read, so no clearing is
 * needed between calls.  Asynchronous on `stream`. */
sns_status snsolve_sketch_countsketch_static(const sns_problem* prob, int64_t d, uint64_t seed, float* SA,
                                             int64_t ldsa, float* Sb, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* SNSOLVE_H */
