/* apo diagnostics: measurement entry points of libapo.so used by the benchmark.  They are
 * not part of the method (the paper has no counterpart); they make the roofline figures
 * reproducible.  Conventions as in apo.h. */
#ifndef APO_DIAG_H
#define APO_DIAG_H

#include <stddef.h>
#include <stdint.h>

#include "apo.h"

#ifdef __cplusplus
extern "C" {
#endif

/* apo_vote on the full level-0 grid that also counts the work the coarse kernel does
 * (votes_out NULL: the form apo_solve_batch runs, each coarse block keeping only its topk
 * best cells in the workspace, instead of writing every vote; counts_out NULL: no counting,
 * the kernel exactly as the search runs it):
 * counts_out (device, 8 x uint64, zeroed by the call) receives FP64 parent-cell
 * evaluations, FP64 per-(cell, hit) prefix evaluations, FP64 tan(lambda) tail evaluations,
 * the number of coarse-kernel launches, then the same three FP32 counts.  For APO_F64_MID
 * slots 1 and 2 count the midpoint form's per-(cell, hit) prefixes and tan(lambda) tails. */
int apo_diag_vote_coarse_counts(const apo_geometry *geom, const apo_hits *hits, int32_t precision,
                                int32_t *votes_out, unsigned long long *counts_out,
                                void *workspace, size_t workspace_bytes, void *stream);

/* Number of coarse-kernel launches apo_vote / apo_solve_batch make for n_events events. */
int32_t apo_diag_coarse_launches(const apo_geometry *geom, int32_t n_events);

/* Throughput microbenchmark of one directed-rounding operation on the current device:
 * precision APO_F64 / APO_F32, op 0 = add (__dadd_rd), 1 = mul (__dmul_rd), 2 = an
 * alternating add/mul chain; FP64 only: 3 = alternating rd square root (the library's own
 * integer-pipe form) and mul by 3, 4 = the same with the CUDA library's __dsqrt_rd.  Many
 * independent chains per thread, every SM busy.  *ops_per_s = operations per second.
 * Synchronous, about 0.1 s. */
int apo_diag_pipe_peak(int32_t precision, int32_t op, double *ops_per_s);

/* Elementwise FP64 operations on device arrays x -> out (n elements, on `stream`), for
 * testing the library's integer-pipe operations against the CUDA library: op 0-2 =
 * reciprocal rounded down / up / to nearest (integer pipe), 3-5 = square root rd / ru /
 * rn (integer pipe), 6-11 = the same six with the CUDA library's __drcp_* / __dsqrt_*;
 * 12-14 = quotient x[i] / x[i ^ 1] rd / ru / rn (integer pipe; n must be even), 15-17 =
 * the same with __ddiv_*.  Every op accepts any double. */
int apo_diag_dops(int32_t op, const double *x, double *out, int64_t n, void *stream);
/* The vote program's evaluated intervals for n explicit (cell, hit) pairs, on `stream`,
 * for comparing end points with the oracle (Eq. ApoVote; G = rho F per drift sign).
 * Device arrays: cells[12 n] = (d0, sin phi0, cos phi0, omega, z0, tan(lambda)) as lo, hi
 * pairs; hits[9 n] = (x0, y0, sin phi_s, cos phi_s, tan tau, sin phi_s tan tau,
 * cos phi_s tan tau, tan^2 tau, drift); out[10 n] = the vote (0 / 1), G+ lo, G+ hi, G- lo,
 * G- hi, a guard flag (1 when a divisor reached 0 and the pair votes unevaluated), and the
 * phase corrections delta+ lo, hi, delta- lo, hi; zeros past a guard; the flag is 2 when
 * the direction condition refused the vote.  precision APO_F64 or APO_F32 (cells and hits
 * rounded outward to FP32 first; results widened to double), optionally | APO_OUTGOING. */
int apo_diag_vote_pair_ends(const apo_geometry *geom, int32_t precision, const double *cells,
                            const double *hits, double *out, int64_t n, void *stream);
/* Exercises the device-side wait limit: one kernel waits on a barrier that nothing
 * completes, for at most `limit_polls` polls, then records a timeout in a status word and
 * ends normally.  Returns APO_ETIMEOUT when the status word shows it (the expected
 * outcome), APO_OK if it did not, APO_ECUDA on a CUDA failure.  Synchronous; the device
 * stays usable afterwards. */
int apo_diag_wait_timeout(int32_t limit_polls);

/* The same wait on the status word of apo_vote_coarse_noalloc's fixed array (queued on
 * `stream`): afterwards apo_vote_coarse_noalloc_status reports APO_ETIMEOUT, until the next
 * apo_vote_coarse_noalloc call clears the word. */
int apo_diag_noalloc_wait_timeout(int32_t limit_polls, void *stream);

/* Reads the status word of a workspace after the work queued on it (synchronises
 * `stream`): APO_ETIMEOUT if a device wait ran out, APO_OK otherwise. */
int apo_workspace_status(const apo_geometry *geom, int32_t n_events, const void *workspace,
                         void *stream);

#ifdef __cplusplus
}
#endif

#endif /* APO_DIAG_H */
