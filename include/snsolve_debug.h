/*
 * snsolve_debug.h -- verification entry points of the snsolve library.
 *
 * They expose, bit for bit, the random structure of the implicit sketch S as
 * the library's kernels compute it ("generate a sketch matrix S", step 1 of the
 * sketch-and-solve paradigm, Sec. 1.2 of arXiv 2409.14309), so tests can compare
 * it with an independent implementation.  Not needed to solve problems.
 * Device pointers unless stated; asynchronous on `stream` like snsolve.h.
 */
#ifndef SNSOLVE_DEBUG_H
#define SNSOLVE_DEBUG_H

#include <stddef.h>
#include <stdint.h>

#include "snsolve.h"

#ifdef __cplusplus
extern "C" {
#endif

/* CountSketch bucket h(i) in [0, d) and sign s(i) in {-1, +1} of rows 0..m-1
 * (Clarkson-Woodruff sketch, Sec. 1.2.2): h and s are device arrays of m
 * entries.  SNS_EINVAL if m < 0, d < 1 or a pointer is NULL. */
sns_status snsolve_debug_countsketch_hash(int64_t m, int64_t d, uint64_t seed, uint32_t* h, int8_t* s,
                                          void* stream);

/* Raw 64-bit outputs start..start+count-1 of SplitMix64 stream `stream_id`
 * (0 = CountSketch, 1 = SRHT signs, 2 = SRHT sampling, 3 = Gaussian) for
 * `seed`; keys is a device array of count entries. */
sns_status snsolve_debug_stream_keys(uint64_t seed, int stream_id, int64_t start, int64_t count, uint64_t* keys,
                                     void* stream);

/* The d sorted, distinct SRHT row indices of [0, mp) (mp a power of two,
 * 1 <= d <= min(mp, 16384), Sec. 1.2.1 Hadamard sketch), written to idx
 * (device, d int64).  ws: device workspace of snsolve_debug_srht_sample_ws
 * bytes. */
sns_status snsolve_debug_srht_sample_ws(int64_t mp, int64_t d, size_t* bytes);
sns_status snsolve_debug_srht_sample(int64_t mp, int64_t d, uint64_t seed, int64_t* idx, void* ws, size_t ws_bytes,
                                     void* stream);

/* The 256-entry BF16 normal-quantile table T of the Gaussian sketch
 * (Sec. 1.2.1), as raw BF16 bit patterns, written to a HOST array of 256. */
sns_status snsolve_debug_gaussian_table(uint16_t* bf16_bits_host);

/* Y = A R^-1, the explicit preconditioned matrix of sketch-and-apply (SNS_SAA,
 * Sec. 2.1), exactly as snsolve_lstsq forms it: prob dense (F32 or F64), Rinv a
 * device FP64 n x n row-major upper-triangular matrix, Y a device array in A's
 * precision with leading dimension ldy >= n.  SNS_EINVAL for CSR input or bad
 * arguments. */
sns_status snsolve_debug_form_y(const sns_problem* prob, const double* Rinv, void* Y, int64_t ldy, void* stream);

/* ---- Bounded device-side waits ----------------------------------------------
 * The multi-CTA QR of snsolve_lstsq (q = n + 1 >= 32) hands each Householder
 * reflector from the CTA that builds it to the others through device memory;
 * every wait for one is bounded.  This sets how many polls such a wait makes
 * before it gives up (polls <= 0 restores the default, 2^22).  A wait that
 * gives up sets the factorisation's error word and carries on with zeros, later
 * waits stop polling, the kernel ends, and snsolve_lstsq returns SNS_ETIMEOUT
 * (the solve's outputs are then invalid).  Process-wide, read at each launch;
 * meant for tests of the timeout path. */
void snsolve_debug_set_qr_wait_limit(int64_t polls);

/* ---- Host-side fault injection ----------------------------------------------
 * Arms one failure that a host-side check reports; no GPU faults, traps or
 * hangs.  spec = "<kind>[:<n>]": the n-th occurrence (n >= 1, default 1) of
 * <kind> fails, once, and the fault disarms.  Kinds:
 *   "alloc"   one of the library's own allocations (snsolve_create's pinned
 *             buffer, a thread's pinned status buffer, the server arena, the
 *             batched staging buffer) returns SNS_ENOMEM without allocating;
 *   "launch"  the check after a kernel launch returns SNS_ECUDA (the kernel
 *             was launched and completes; the call stops there);
 *   "timeout" the host's read of a device error word (sketch waits, QR polls)
 *             reports an expired wait: SNS_ETIMEOUT.
 * NULL, "" or "none" disarms.  SNS_EINVAL for any other spec.  Process-wide;
 * the environment variable SNSOLVE_FAULT holds the same spec, read at the
 * first check unless this call came first.  snsolve_last_cuda_error() names
 * an injected failure. */
sns_status snsolve_debug_set_fault(const char* spec);

/* Armed kind (0 none, 1 alloc, 2 launch, 3 timeout) and, in *left (may be
 * NULL), the occurrences still to pass before it fires (counting this one). */
int snsolve_debug_fault_armed(int64_t* left);

/* ---- Measurement ----------------------------------------------------------
 * Number of kernel launches this library has issued in this process. */
uint64_t snsolve_launch_count(void);
/* Per-kernel timing: with snsolve_profile(1), every launch is bracketed by a
 * CUDA event pair recorded on its own stream.  snsolve_profile_read
 * synchronizes those events, writes total milliseconds and launch counts per
 * kernel class (nid >= snsolve_profile_num_kernels() entries, HOST arrays) and
 * clears the records.  Kernel classes are named by snsolve_profile_kernel_name. */
sns_status snsolve_profile(int enable);
int snsolve_profile_num_kernels(void);
const char* snsolve_profile_kernel_name(int id);
sns_status snsolve_profile_read(double* ms, uint64_t* count, int nid);
/* Forgets the launch shapes the batched solver's tuner has measured in this
 * process (its cache file, $SNSOLVE_TUNE_CACHE or ~/.cache/snsolve_tune.txt,
 * is left alone), so the next batched call measures again. */
void snsolve_tune_reset(void);

#ifdef __cplusplus
}
#endif
#endif /* SNSOLVE_DEBUG_H */
