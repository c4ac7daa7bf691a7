// Internal interfaces between the snsolve dispatch layer and its kernels.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "snsolve.h"

namespace sns {

// row0: global index of row 0 (the rows are rows row0.. of a larger matrix
// whose sketch is the sum of the parts' sketches); 0 for a whole matrix.
struct DenseArgs {
  const void* A;
  int64_t lda;
  const void* b;
  int64_t m, n;
  bool f64;
  int64_t row0 = 0;
};
struct CsrArgs {
  const int64_t* rowptr;
  const int32_t* col;
  const float* val;
  const float* b;
  int64_t m, n, nnz;
  int64_t row0 = 0;
  bool det = false;        // iterative passes: bitwise reproducible scatters (slower)
};

// CountSketch workspace layout.
struct CsLayout {
  int64_t nblk, spi, parts, ct, ntile, tma_parts, nticket;
  size_t off_sorted, off_seg, off_ticket, off_part, off_list, off_btot, off_bbase, off_err, off_cbase, off_ctab,
      off_wpart, bytes;
};
// Bulk-copy pipeline of the deterministic dense FP32 CountSketch (phase 1b + 2).
bool cs_tma_eligible(const DenseArgs& a);
int64_t cs_tma_parts(int64_t m, int64_t d);
int64_t cs_warp_max_chunks(int64_t m, int64_t d);
// allow_bulk: kernels with bounded device-side waits may run (the cooperative
// plan with its grid barriers; the bulk-copy gather when SNSOLVE_CS_GATHER=t);
// otherwise the two-kernel plan and the warp gather, which never wait, run.
sns_status cs_tma_phase2(const DenseArgs& a, int64_t d, const CsLayout& L, uint8_t* ws, float* SA, int64_t ldsa,
                         float* Sb, int64_t sbs, cudaStream_t st, bool allow_bulk = true);
// Single-launch plan (cooperative) + warp gather for dense FP32; *used = false
// when the plan's blocks cannot all be co-resident (nothing launched then).
sns_status cs_coop_apply(const DenseArgs& a, int64_t d, uint64_t seed, const CsLayout& L, uint8_t* ws, float* SA,
                         int64_t ldsa, float* Sb, int64_t sbs, cudaStream_t st, bool* used);
bool cs_bulk_gather_selected();
CsLayout cs_layout(int64_t m, int64_t n, int64_t d, bool f64, bool csr);
int64_t cs_sorted_max_d();
// Largest n for which the sorted CSR gather's per-warp accumulator rows fit.
int64_t cs_csr_sorted_max_n();
// Largest n whose CSR iterative passes can run bitwise reproducibly (per-warp
// accumulator rows for every pass variant).
int64_t csr_det_max_n();
int num_sms();

sns_status cs_apply_dense_sorted(const DenseArgs& a, int64_t d, uint64_t seed, void* SA, int64_t ldsa, void* Sb,
                                 int64_t sbs, void* ws, size_t ws_bytes, cudaStream_t st, bool allow_bulk = true);
// Sparse sign embedding, dense FP32 (1 <= zeta <= min(8, d)); zeroes SA and Sb.
sns_status cs_apply_sparse_sign(const DenseArgs& a, int64_t d, int zeta, uint64_t seed, float* SA, int64_t ldsa,
                                float* Sb, int64_t sbs, cudaStream_t st);
sns_status cs_apply_dense_stream(const DenseArgs& a, int64_t d, uint64_t seed, void* SA, int64_t ldsa, void* Sb,
                                 int64_t sbs, cudaStream_t st);
// Streaming CountSketch on CSR (one pass, float reductions into SA; SA and Sb
// are zeroed here).  The order of additions varies run to run.
sns_status cs_apply_csr_stream(const CsrArgs& a, int64_t d, uint64_t seed, float* SA, int64_t ldsa, float* Sb,
                               int64_t sbs, cudaStream_t st);
sns_status cs_apply_csr(const CsrArgs& a, int64_t d, uint64_t seed, float* SA, int64_t ldsa, float* Sb, int64_t sbs,
                        void* ws, size_t ws_bytes, cudaStream_t st);
sns_status debug_countsketch_hash(int64_t m, int64_t d, uint64_t seed, uint32_t* h, int8_t* s, cudaStream_t st);
sns_status debug_stream_keys(uint64_t seed, int stream, int64_t start, int64_t count, uint64_t* out, cudaStream_t st);

// SRHT.
size_t srht_ws_bytes(int64_t m, int64_t n, int64_t d, bool f64);
sns_status srht_apply_dense(const DenseArgs& a, int64_t d, uint64_t seed, void* SA, int64_t ldsa, void* Sb,
                            int64_t sbs, void* ws, size_t ws_bytes, cudaStream_t st);
sns_status debug_srht_sample(int64_t mp, int64_t d, uint64_t seed, int64_t* out, void* ws, size_t ws_bytes,
                             cudaStream_t st);

// Gaussian.  `terms` (1..3): BF16 terms of [A | b] in the tensor-core product.
size_t gauss_ws_bytes(int64_t m, int64_t n, int64_t d, int terms);
// Byte offset in the Gaussian workspace of the error word its bounded waits
// set (0 after a sketch that completed).
size_t gauss_err_offset();
sns_status gauss_apply_dense(const DenseArgs& a, int64_t d, uint64_t seed, int terms, float* SA, int64_t ldsa,
                             float* Sb, int64_t sbs, void* ws, size_t ws_bytes, cudaStream_t st);
// Levels of the BF16 normal-quantile table T of the Gaussian sketch.
constexpr int kGaussLevels = 256;
void gauss_table_host(uint16_t* out);

// QR / triangular solves (FP64).  W is column-major d x q with leading dim d.
struct QrOut {
  double* W;        // in: column-major [SA | Sb] in FP64; out: R_aug in the upper triangle
  int64_t d, q;     // q = n + 1
  double* x;        // n entries: x^ = R^{-1} z (may be null)
  int32_t* status;  // device int: SNS_OK / SNS_ERANK
  double* sres;     // device double: |R_aug[n, n]|
};
sns_status qr_load_colmajor(const void* SAaug, int64_t ld, bool f64, int64_t d, int64_t q, double* W, cudaStream_t st);
sns_status qr_solve_one(const QrOut& o, cudaStream_t st);
// Multi-CTA factorisation of one large problem; ws holds qr_coop_ws_bytes(d, q)
// bytes (published reflectors and scalars, error word).  The error word is set if a wait gave up.
size_t qr_coop_ws_bytes(int64_t d, int64_t q);
// Byte offset, within that workspace, of the int error word (nonzero: a wait timed out).
size_t qr_coop_err_offset(int64_t d, int64_t q);
sns_status qr_solve_coop(const QrOut& o, void* ws, cudaStream_t st);
// Polls a cooperative factorisation's waits make before giving up (<= 0: default).
void set_qr_wait_limit(long long polls);
sns_status qr_solve_tasks(const QrOut* tasks_dev, int ntasks, int64_t max_d, cudaStream_t st);
sns_status rinv_build(const double* W, int64_t ldw, int64_t n, double* Rinv, double* RinvT, bool identity,
                      cudaStream_t st);

// Iterative refinement (SAP-SAS).
struct IterWs {
  double *Rinv, *RinvT;       // n x n row-major
  double* P;                  // n x n: R^-1 R^-T, the inner solver's preconditioner
  double *g, *w, *z, *rx, *s, *dx, *scal;  // n-vectors and scalars
  float *xhi, *xlo, *z32;     // n
  float* part;                // partial n-vectors from passes [grid][n]
  double* partd;              // FP64 partials [grid][n + 4]
  uint32_t* ticket;           // reduction tickets (group counters + top)
  double* lvl2;               // level-2 partial rows
  int grid;
};
size_t iter_ws_bytes(int64_t n, int grid);
IterWs iter_ws_carve(void* base, int64_t n, int grid);
int iter_grid();
// exact_g: exact FP32 products in g = A^T r (needed for eta targets below
// about 1e-6; otherwise g's per-term FP32 rounding is negligible).
sns_status resid_pass(const DenseArgs* da, const CsrArgs* ca, const double* x, const IterWs& W, bool want_anorm,
                      bool exact_g, cudaStream_t st);
sns_status normal_pass(const DenseArgs* da, const CsrArgs* ca, const IterWs& W, cudaStream_t st);
// P = R^-1 R^-T (symmetric) from the row-major R^-1.
sns_status pgram_build(const double* Rinv, int64_t n, double* P, cudaStream_t st);
// Zeroes the inner-loop control words (stop level, done flag, pass count).
sns_status iter_reset(const IterWs& W, cudaStream_t st);
// Refinement cycle of the inner solver (preconditioned CG on A^T A dx = g with
// M^-1 = P; g from the last residual pass): pcg_start sets dx = 0, r = g,
// z = P g and the stop level, after which each normal_pass + pcg_step is one
// iteration; the cycle ends on the device once the CG residual has dropped by
// max(tol / (2 eta), 4e-3) (later launches return at once) or the host's
// launch budget runs out.  pcg_apply adds dx to x.
// factored: apply M^-1 as R^-1 (R^-T r) (two n x n products) instead of the
// formed P = R^-1 R^-T, whose FP64 rounding (relative to kappa(R)^2) makes it
// indefinite for badly conditioned R.
sns_status pcg_start(const IterWs& W, int64_t n, double tol, cudaStream_t st, bool factored = false);
sns_status pcg_step(const IterWs& W, int64_t n, cudaStream_t st, bool factored = false);
// out[0] = max |R_ii|, out[1] = min |R_ii| (device), i < n, W column-major.
sns_status diag_range(const double* W, int64_t ldw, int64_t n, double* out, cudaStream_t st);
sns_status pcg_apply(const IterWs& W, int64_t n, double* x, cudaStream_t st);
sns_status eta_eval(const IterWs& W, int64_t n, double* host_out, cudaStream_t st);

// Sketch-and-apply (SAA-SAS).  Y = A R^-1 (m x n, A's precision, leading
// dimension saa_ldy) from the FP64 row-major R^-1; out = M v (or += M v) for an
// n x n FP64 row-major M; P = I.
int64_t saa_ldy(int64_t n, bool f64);
size_t saa_y_bytes(int64_t m, int64_t n, bool f64);
sns_status saa_form_y(const DenseArgs& a, const double* Rinv, void* Y, cudaStream_t st, int64_t ldy = 0);
sns_status saa_matvec(const double* M, int64_t n, const double* v, double* out, bool accumulate, cudaStream_t st);
sns_status ident_build(double* P, int64_t n, cudaStream_t st);
// pcg_start with the right-hand side v instead of the residual pass's g.
sns_status pcg_start_rhs(const IterWs& W, int64_t n, double tol, const double* v, cudaStream_t st);

// Batched.
size_t batch_ws_bytes(const sns_problem* probs, const sns_opts* opts, int nprob);
sns_status lstsq_batched(const sns_problem* probs, const sns_opts* opts, int nprob, double* const* x,
                         sns_info* infos, void* ws, size_t ws_bytes, cudaStream_t st);
}  // namespace sns
