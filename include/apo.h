/* apo: interval-arithmetic Apollonius voting for a full-stereo drift chamber on one GPU.
 *
 * C ABI of libapo.so.  Method: arXiv:2401.04576 (da Silva, Lebrun, Angelique, Del Buono).
 * Every hit (a stereo wire and its drift distance) votes, with both drift signs, for every
 * cell of a 5-D helix parameter grid whose outward-rounded interval extension of the
 * Apollonius tangency condition contains zero (Section 3.1, Eq. ApoVote, with d^Ax of
 * Eq. defdiAX_b and Phi of Eqs. ApproxPhi_a-d, Appendix A).  The best cells are kept and
 * bisected, coarse to fine; the final cells with the most votes give the helix and its
 * errors (Section 3.3).
 *
 * Conventions of every entry point:
 *  - returns an apo_status; never aborts the process;
 *  - the caller owns every buffer it passes; the library owns only its handles;
 *  - "device" pointers are CUDA global memory on the current device; "host" pointers are
 *    ordinary host memory; all device work is queued on the caller's stream (a
 *    cudaStream_t passed as void*; NULL = legacy default stream) and is asynchronous
 *    unless stated otherwise;
 *  - there is no CPU fallback: without a usable CUDA device calls return APO_ECUDA.
 *
 * Parameter cell axes (index a): 0 d0 [m] (signed POCA distance to the origin along
 * (-sin phi0, cos phi0)), 1 phi0 [rad] (tangent azimuth at the POCA), 2 omega [1/m]
 * (signed curvature; helix centre (-(R+d0) sin phi0, (R+d0) cos phi0), R = 1/omega),
 * 3 z0 [m] (z at the POCA), 4 tanl = tan(dip angle).  A level-L cell index idx_a is in
 * [0, bins[a] << L); its key is sum_a idx_a << s_a, where axis a is b_a = max(10,
 * ceil(log2(bins[a] << levels))) bits wide and s_a = b_0 + ... + b_(a-1) (so 10 a when every
 * axis has at most 1024 finest cells); its 32 children are 2 idx_a + bit_a.
 */
#ifndef APO_H
#define APO_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
typedef enum {
    APO_OK = 0,
    APO_EINVAL = -1,   /* bad argument or malformed input                          */
    APO_ENOMEM = -2,   /* workspace too small / device allocation failed           */
    APO_ECUDA = -3,    /* a CUDA call failed (message: apo_last_error())           */
    APO_ETIMEOUT = -4, /* a device wait hit its iteration limit                    */
    APO_EBUSY = -5     /* serving queue full: retry later                          */
} apo_status;

/* interval precision of one level.  APO_F64: FP64 intervals.  APO_F32: FP32 intervals.
 * APO_F64_FILTERED: FP64 intervals evaluated only where the FP32 program votes first (FP32
 * intervals contain the FP64 ones, so the votes are exactly APO_F64's; it pays only where
 * most FP32 votes are "no").
 * APO_F64_MID: the midpoint form of Section 3.1 (last paragraph): the quantities that build
 * d^Ax (Eq. defdiAX_b) are evaluated at the voxel centre in round-to-nearest FP64, and only
 * (x^Ax - x_c)^2 + (y^Ax - y_c)^2 - (R + d^Ax)^2 keeps the voxel's FP64 intervals.  Faster
 * and not sound (a voxel holding the solution can lose a vote).  Needs the grid's
 * sincos_mid table.
 * APO_F64_EXACT: FP64 intervals with the exact phase of Eq. CSAXtoPHI_a (an interval
 * fixed-point enclosure per drift sign, started from the expansion of Eqs. ApproxPhi_a-d)
 * instead of the expansion; sound for the unexpanded equations, several times costlier. */
enum { APO_F64 = 0, APO_F32 = 1, APO_F64_FILTERED = 2, APO_F64_MID = 3, APO_F64_EXACT = 4 };

/* Flag OR-ed into any precision above except APO_F64_MID: the direction condition.  The
 * track is taken to leave its point of closest approach (POCA) to the origin and each hit
 * to lie on that outgoing arc, at a turning angle psi >= 0 from the POCA along the helix
 * (the paper's toy tracks start at the target, Section 3.2).  A hit then votes for a cell
 * only where psi can be >= 0; sin psi has the sign of the wire point's coordinate along the
 * helix tangent at the POCA, and a cell where that coordinate is negative throughout gets
 * no vote from the hit.  Without the flag, a helix and the same helix run backwards,
 * (-d0, phi0 + pi, -omega, z0, -tanl), get identical votes. */
#define APO_OUTGOING 16

/* Coarse-to-fine schedules of apo_solve_batch.  APO_SCHED_TOPK: at each level the grid's
 * topk cells by (votes desc, key asc) survive.  APO_SCHED_MAXSET: whole vote groups
 * survive (Section 3.3 takes the result from the set of maximum-vote voxels): with vmax the
 * level's best count, the kept cells are {votes >= T} for the smallest T >= max(vmax -
 * slack, min(vmax, 1)) with at most max_keep of them; if the vmax group alone exceeds
 * max_keep, the event's search ends at that level.  The estimate is over the last level's
 * vmax group: per axis the mean of the cells' centres, summed by cell index in ascending
 * order (n_i centre_i for the n_i cells at index i, round-to-nearest), and the half-extent
 * of their union. */
enum { APO_SCHED_TOPK = 0, APO_SCHED_MAXSET = 1 };

#define APO_HIT_CAP 256      /* hits per event */
#define APO_MAX_LEVELS 8     /* bisection levels after the coarse level */
#define APO_MAX_TRACKS 8     /* tracks per event in multi-track extraction */

typedef struct apo_geometry apo_geometry;

/* Wire table (paper Appendix A, Eqs. wirePar_a,b): wire i passes through (x0, y0, 0) with
 * direction (sin phi_s tan tau, -cos phi_s tan tau, 1).  Host arrays of n_wires doubles,
 * copied by apo_geometry_create; sphi_t, cphi_t, t2 are the products sin(phi_s) tan(tau),
 * cos(phi_s) tan(tau), tan(tau)^2 rounded once by the caller and used as given. */
typedef struct {
    int32_t n_wires;
    const double *x0, *y0, *sin_phis, *cos_phis, *tan_tau, *sphi_t, *cphi_t, *t2;
} apo_wires;

/* Parameter grid (the voxel discretisation of Section 3.1, extended to five axes).
 * lo_edge[a] / hi_edge[a]: host arrays of bins[a] << levels finest-level cell edges; a
 * level-L cell idx spans [lo_edge[idx << (levels-L)], hi_edge[((idx+1) << (levels-L)) - 1]].
 * No omega cell may contain 0.  sincos: host array of rows (sin lo, sin hi, cos lo,
 * cos hi), outward enclosures of sin/cos over each phi0 cell, level by level (level L
 * starts at row sum_{l<L} bins[1] << l).  sincos_mid (may be NULL): rows (sin c, cos c) at
 * each phi0 cell's centre c = (lo + hi) / 2, same row order; needed by APO_F64_MID only.
 * All copied.  Limits: bins[a] << levels <= 65536 with the key widths above summing to at
 * most 64 bits, bins[0] * bins[3] <= 256, bins[4] <= 32, levels <= APO_MAX_LEVELS,
 * 1 <= topk, topk * 32 <= 4096, topk <= number of level-0 cells.  APO_SCHED_TOPK needs the
 * key widths to sum to at most 50 bits. */
typedef struct {
    int32_t bins[5];
    int32_t levels;
    int32_t topk;
    const double *lo_edge[5];
    const double *hi_edge[5];
    const double *sincos;
    const double *sincos_mid;
} apo_grid;

/* A batch of events in CSR form; DEVICE arrays owned by the caller.  Event e owns hits
 * offsets[e] .. offsets[e+1]-1 (at most APO_HIT_CAP); wire_id in [0, n_wires); drift >= 0
 * and finite.  A malformed event does not stop the batch: its track gets votes =
 * APO_EINVAL. */
typedef struct {
    int32_t n_events;
    const int32_t *offsets;
    const int32_t *wire_id;
    const double *drift;
} apo_hits;

/* One reconstructed helix (Section 3.3): p = mean centre of the final maximum-vote cells,
 * w = half-extent of their union, votes = their vote count (< 0: status of a malformed
 * event), n_hits = hits of the event. */
typedef struct {
    double p[5];
    double w[5];
    int32_t votes;
    int32_t n_hits;
} apo_track;

/* Execution knobs of apo_solve_batch.  None of them changes any result (every setting
 * evaluates the same interval program cell by cell); apo_autotune picks them by timing.
 * Zero means the default. */
typedef struct {
    int32_t coarse_filter;   /* 1: on the level-0 grid, evaluate FP64 levels only where the
                                FP32 program votes (as APO_F64_FILTERED) */
    int32_t cells_filter;    /* 1: the same for the bisected cells of levels >= 1 */
    int32_t cells_block;     /* threads per block of the cell-voting kernel: 128 or 256 */
    int32_t chunk_events;    /* events per level-0 launch (at most the workspace's chunk) */
    int32_t coarse_full;     /* 1 (APO_SCHED_TOPK): level 0 writes every cell's vote and selects
                                from them, instead of each block keeping its topk best cells
                                (more workspace, fewer instructions per block); the same
                                kept set either way */
    int32_t persistent;      /* 1 (APO_SCHED_TOPK only): one persistent launch for the whole
                                batch; each block pulls the next event from a device counter
                                and runs its whole search (every round, tile and level),
                                instead of one launch per step and level.  Levels must share
                                their APO_OUTGOING flag and use APO_F64, APO_F32 or
                                APO_F64_FILTERED; no trace. */
} apo_tune;

/* Options of apo_solve_batch.  precision[L] selects FP64 or FP32 intervals at level L
 * (L = 0 is the coarse grid); FP32 end points are rounded outward, so an FP32 vote set
 * contains the FP64 one cell by cell.  trace_keys / trace_votes (device, may be NULL):
 * n_events x (levels + 1) x topk, the cells kept after each level (the last row holds the
 * best topk final cells). */
typedef struct {
    int32_t precision[APO_MAX_LEVELS + 1];
    int32_t max_tracks;      /* tracks per event, 1 .. APO_MAX_TRACKS */
    int32_t min_votes;       /* stop when the best final vote count is below this */
    double mask_sigma;       /* drift resolution: found hits are masked with d +- 3 sigma */
    uint64_t *trace_keys;
    int32_t *trace_votes;
    apo_tune tune;
    int32_t use_graph;       /* 1: record the whole search as a CUDA graph on the first call
                                with these arguments, and replay it on later calls */
    int32_t *hit_track;      /* device, may be NULL: for every hit of the batch (CSR order of
                                apo_hits) the track whose final maximum-vote cells took it in
                                the hit finding of Section 3.3 (0-based), or -1 if none did.
                                With APO_SCHED_MAXSET it needs max_tracks > 1 (each round's
                                track cells, see apo_solve_batch).  apo_solve_batch_host and
                                the server require NULL. */
    int32_t schedule;        /* APO_SCHED_TOPK (default) or APO_SCHED_MAXSET */
    int32_t max_keep;        /* APO_SCHED_MAXSET: cells kept per event and level, >= 1 */
    int32_t slack;           /* APO_SCHED_MAXSET: vote groups down to vmax - slack are kept */
    int32_t *final_level;    /* device, may be NULL (APO_SCHED_MAXSET): per event and track
                                (n_events x max_tracks), the level whose vmax group gave the
                                estimate */
    int32_t *n_final;        /* device, may be NULL (APO_SCHED_MAXSET): per event and track, the
                                number of cells the estimate was taken over */
    int32_t *trace_count;    /* device, may be NULL (APO_SCHED_MAXSET, max_tracks 1): n_events x
                                (levels + 1) kept counts; trace_keys / trace_votes are then
                                n_events x (levels + 1) x max_keep, the kept cells of each
                                level before the final one (in the order of the level's cells) */
} apo_solve_opts;

/* Fills *opts with: all levels FP64, one track, min_votes 0, mask_sigma 150e-6, no trace,
 * tune = {coarse_filter 0, cells_filter 1, cells_block 256, chunk 0}, no graph, no
 * hit_track, schedule APO_SCHED_TOPK, max_keep 32768, slack 0. */
void apo_solve_opts_default(apo_solve_opts *opts);

/* Text of the last error on this thread ("" if none). */
const char *apo_last_error(void);

/* Copies the wire table and grid to the current device and prepares the series constants
 * used by the transcendental enclosures.  The geometry is immutable afterwards and may be
 * used from any stream.  Synchronous.  APO_EINVAL on limits above, APO_ECUDA on failure. */
int apo_geometry_create(const apo_wires *wires, const apo_grid *grid, apo_geometry **out);
void apo_geometry_destroy(apo_geometry *geom);

/* Number of level-0 cells (product of bins). */
int64_t apo_coarse_cells(const apo_geometry *geom);

/* Device workspace needed by apo_vote / apo_refine / apo_solve_batch for n_events events
 * (opts may be NULL for the first two).  The caller allocates it (any device allocator,
 * 256-byte aligned) and passes it back; it may be reused across calls on one stream. */
int apo_workspace_bytes(const apo_geometry *geom, int32_t n_events, const apo_solve_opts *opts,
                        size_t *bytes);

/* Eq. (ApoVote) summed over each event's hits for a set of cells at `level` (Section 3.1:
 * one vote per hit when either drift sign passes).  cell_keys: device, n_events x
 * n_cells_per_event keys; NULL = the full level-0 grid in linear order (d0 fastest,
 * tanl slowest; then level must be 0 and n_cells_per_event = apo_coarse_cells).
 * votes_out: device int32, n_events x n_cells_per_event.  The call only queues work: a
 * device wait that ran out of its poll limit (the votes of that launch are then untrusted)
 * shows in the workspace's status word; read it with apo_workspace_status (apo_diag.h)
 * after the work, as apo_solve_batch_host and the server do. */
int apo_vote(const apo_geometry *geom, const apo_hits *hits, const uint64_t *cell_keys,
             int64_t n_cells_per_event, int32_t level, int32_t precision, int32_t *votes_out,
             void *workspace, size_t workspace_bytes, void *stream);

/* One coarse-to-fine step: per event, keeps the topk cells of (keys_in, votes_in) by
 * (votes descending, key ascending) and writes them to kept_keys / kept_votes (device,
 * n_events x topk, may be NULL) and their 32 children each (level + 1) to children_out
 * (device, n_events x topk x 32).  keys_in NULL = the full level-0 grid in linear order.
 * Needs keys of at most 50 bits.  As for apo_vote, check apo_workspace_status after the
 * work. */
int apo_refine(const apo_geometry *geom, const apo_hits *hits, const uint64_t *keys_in,
               const int32_t *votes_in, int64_t n_in_per_event, int32_t level,
               uint64_t *kept_keys, int32_t *kept_votes, uint64_t *children_out,
               void *workspace, size_t workspace_bytes, void *stream);

/* Whole search for every event: level-0 voting, top-K, `levels` rounds of bisection,
 * voting and top-K, and the estimate of Section 3.3, repeated per track: after each track,
 * every remaining hit that votes (FP64) for one of its final maximum-vote cells with the
 * drift widened to [d - 3 mask_sigma, d + 3 mask_sigma] is removed (the hit finding of
 * Section 3.3 with a widened box) and the event is searched again.  An event stops at
 * max_tracks tracks, when no hit is left, or when the best final vote count is below
 * min_votes (that search gives no track).
 * With APO_SCHED_MAXSET and max_tracks > 1 the final vmax group of a search can hold the
 * cells of several tracks (tracks with equal hit counts tie), so each round takes one of
 * them: the seed is the group's lowest key, S the searched hits that vote for it at the
 * final level's precision, and the track's cells are the group's cells that every hit of
 * S votes for.  The estimate is taken over those cells; the track takes S and the hits
 * that vote for one of them with the widened drift.  With max_tracks 1 the estimate is
 * over the whole group.  APO_F64_MID levels are refused there.  tracks_out: device, n_events x
 * opts->max_tracks records (unused records zeroed); n_tracks_out: device int32 per event
 * (may be NULL).  No host synchronisation: the call only queues work on the stream. */
int apo_solve_batch(const apo_geometry *geom, const apo_hits *hits, const apo_solve_opts *opts,
                    apo_track *tracks_out, int32_t *n_tracks_out, void *workspace,
                    size_t workspace_bytes, void *stream);

/* Times apo_solve_batch on `hits` (typically a sample of the batch to come) for every
 * combination of the apo_tune knobs and writes the fastest to *best (its time to *best_ms,
 * may be NULL): the launch schedule (per-level launches, or the persistent launch when
 * the options allow it), the FP32-first filters, the threads per block of the bisected
 * cells' kernel and the events per level-0 launch.  opts: as for apo_solve_batch (its tune and use_graph are ignored).
 * Workspace as for apo_solve_batch.  Synchronous. */
int apo_autotune(const apo_geometry *geom, const apo_hits *hits, const apo_solve_opts *opts,
                 void *workspace, size_t workspace_bytes, void *stream, apo_tune *best,
                 float *best_ms);

/* As apo_solve_batch with HOST inputs and outputs: copies offsets / wire_id / drift to
 * the workspace, runs, copies the tracks back and synchronises the stream.  The hits
 * arrays must hold offsets[n_events] entries; workspace from apo_workspace_bytes with
 * apo_host_extra_bytes(n_hits) added. */
size_t apo_host_extra_bytes(int32_t n_events, int64_t n_hits);
int apo_solve_batch_host(const apo_geometry *geom, int32_t n_events, const int32_t *offsets,
                         const int32_t *wire_id, const double *drift, const apo_solve_opts *opts,
                         apo_track *tracks_out, int32_t *n_tracks_out, void *workspace,
                         size_t workspace_bytes, void *stream);

/* ---- Serving: continuous batching of events as they arrive ----
 * A server owns a fixed set of batch slots on the geometry's device, each with its own
 * stream, device workspace and pinned host staging, all allocated at creation and kept
 * resident.  A background host thread moves submitted events into a free slot as soon as
 * one frees up (up to batch_events per slot), queues the whole search for that batch, and
 * collects finished batches; batches in different slots run concurrently on the device,
 * and requests arriving meanwhile wait only for the next free slot.  Every event's search
 * is independent of the others in its batch, so its result is the same alone and in any
 * mix.  The paper has no counterpart (it processes one track at a time, Section 3.3). */
typedef struct apo_server apo_server;

typedef struct {
    apo_solve_opts solve;        /* search options for every event (trace / graph ignored) */
    int32_t batch_events;        /* events per batch slot (>= 1) */
    int32_t max_slots;           /* upper bound on slots; the memory budget may allow fewer */
    size_t device_bytes;         /* device memory budget for all slots (0: one slot) */
    int32_t max_pending;         /* submitted events waiting for a slot before APO_EBUSY */
    int32_t inject_error_after;  /* > 0: fail the n-th batch as a CUDA error would (tests) */
} apo_serve_opts;

/* Defaults: default search, 64 events per slot, 4 slots, budget 0, 4096 pending, no
 * injection. */
void apo_serve_opts_default(apo_serve_opts *opts);

/* Device bytes of one batch slot for these options (workspace + staged inputs / outputs):
 * the unit of the memory budget device_bytes.  0 on bad arguments. */
size_t apo_serve_slot_bytes(const apo_geometry *geom, const apo_serve_opts *opts);

/* Creates the slots (as many as max_slots and device_bytes allow, at least one) and starts
 * the scheduling thread.  APO_ENOMEM if even one slot does not fit. */
int apo_serve_create(const apo_geometry *geom, const apo_serve_opts *opts, apo_server **out);

/* Number of batch slots the server created. */
int32_t apo_serve_slots(const apo_server *srv);

/* Submits one event (host arrays of n_hits wire ids and drifts, copied).  APO_EBUSY when
 * max_pending events are already waiting (back-pressure: retry later), APO_EINVAL for
 * n_hits outside [0, APO_HIT_CAP], APO_ECUDA once the server has failed. */
int apo_serve_submit(apo_server *srv, const int32_t *wire_id, const double *drift, int32_t n_hits,
                     uint64_t request_id);

/* Moves up to max finished events into host arrays: tracks (max x solve.max_tracks
 * records), n_tracks and request_id (max each); *n_done = how many.  Non-blocking.
 * Returns APO_ECUDA (with the message in apo_last_error) if a batch failed. */
int apo_serve_poll(apo_server *srv, apo_track *tracks, int32_t *n_tracks, uint64_t *request_id,
                   int32_t max, int32_t *n_done);

/* Waits until every submitted event has finished (or timeout_ms passes: APO_ETIMEOUT). */
int apo_serve_drain(apo_server *srv, int32_t timeout_ms);

/* Batches launched so far and the largest number of slots that were in flight at once. */
int apo_serve_stats(const apo_server *srv, int32_t *batches, int32_t *max_busy_slots);

/* Latency measured inside the library for every event finished so far: from
 * apo_serve_submit accepting the event to the scheduling thread seeing its batch complete
 * (steady clock; the thread polls every 50 us).  Writes the median and the 99th percentile
 * in ms (nearest rank: the ceil(p n)-th smallest of n) and n; zeros before any event. */
int apo_serve_latency(const apo_server *srv, double *p50_ms, double *p99_ms, int64_t *n_events);

/* Stops the scheduling thread after the batches in flight and frees the slots. */
void apo_serve_destroy(apo_server *srv);

/* Full level-0 voting (as apo_vote with cell_keys = NULL) that allocates nothing and takes
 * no workspace.  The paper has no counterpart: this is a library service.  It is for
 * callers that may not allocate device memory while they vote, e.g. a process whose
 * framework allocator owns the whole device budget, or a latency-bound loop in which
 * cudaMalloc / cudaFree, which can synchronise the device, are not allowed after start-up.
 * They still pass their inputs (hits, device) and the output votes_out (device int32,
 * n_events x apo_coarse_cells).  The scratch (staged hits, hit counts, status, vote
 * histograms: about 2.7 MB) is one fixed array compiled into libapo.so, held on every
 * device that loads the library until the process exits; hence at most
 * APO_NOALLOC_MAX_EVENTS events per call (more: APO_EINVAL, see apo_last_error()).
 * The first call on a device looks up that array's device address (cudaGetSymbolAddress)
 * and caches it; make that first call before any stream capture.  Every call reuses the
 * same array and clears what must start at zero; calls whose work overlaps on the GPU
 * (other streams, other threads) race on it and must be serialised by the caller. */
#define APO_NOALLOC_MAX_EVENTS 64
int apo_vote_coarse_noalloc(const apo_geometry *geom, const apo_hits *hits, int32_t precision,
                            int32_t *votes_out, void *stream);

/* Status of the last apo_vote_coarse_noalloc call on the current device (its status word
 * lives in the same fixed array, so apo_workspace_status cannot see it).  Synchronises
 * `stream` (the stream of that call), then writes the raw status bits to *flags_out (host,
 * may be NULL): APO_STATUS_TIMEOUT (a device wait ran out of its poll limit; the votes are
 * untrusted), APO_STATUS_BADHIT (a wire id out of range or a negative / non-finite drift),
 * APO_STATUS_TOOMANY (an event above APO_HIT_CAP hits), APO_STATUS_BADOFFS (decreasing
 * offsets).  A malformed event gets zero votes and does not stop the batch.  Returns
 * APO_ETIMEOUT if the timeout bit is set, else APO_EINVAL if any malformed-event bit is set,
 * else APO_OK.  Each apo_vote_coarse_noalloc call clears the word first. */
#define APO_STATUS_TIMEOUT 1u
#define APO_STATUS_BADHIT 2u
#define APO_STATUS_TOOMANY 4u
#define APO_STATUS_BADOFFS 8u
int apo_vote_coarse_noalloc_status(uint32_t *flags_out, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* APO_H */
