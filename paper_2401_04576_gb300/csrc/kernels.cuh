// Device-side data layout shared by the kernels and the C-ABI host code.
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/apo.h"
#include "vote_program.cuh"

namespace apo {

constexpr int kHitCap = 256;        // hits per event
constexpr int kMaxLevels = 8;
constexpr int kHistBins = kHitCap + 1;

// Read-only device tables of one geometry, passed to kernels by value.
struct DevGeom {
    int bins[5];
    int levels;
    int topk;
    int n_wires;
    const double *lo_edge[5];       // finest-level cell edges per axis
    const double *hi_edge[5];
    const double *sincos;           // (sin lo, sin hi, cos lo, cos hi) per phi0 cell per level
    long long sincos_off[kMaxLevels + 1];
    const double *sincos_mid;       // (sin, cos) at each phi0 cell's centre, same rows; may be null
    const double *wire[8];          // x0, y0, sin phis, cos phis, tan tau, sphi*t, cphi*t, t^2
    SeriesConsts k;                 // k.outgoing: set per call from the precision's flag bit
    int key_shift[5];               // cell key layout: idx_a << key_shift[a], key_bits[a] wide
    int key_bits[5];
};

// One hit as staged for the vote kernels: 80 bytes, a multiple of 16 so an event's hits
// form one contiguous, 16-byte aligned block for a bulk (TMA) copy into shared memory.
struct alignas(16) HitRecD { double v[9]; double pad; };          // x0 y0 sph cph t spt cpt t2 d
struct alignas(16) HitRecF { float lo[9]; float hi[9]; float pad[2]; };
static_assert(sizeof(HitRecD) == 80 && sizeof(HitRecF) == 80, "hit record size");

// Cell edges on axis a for index i at `level`.
__device__ __forceinline__ IV<double> edge(const DevGeom &g, int a, int level, int i) {
    int sh = g.levels - level;
    return {g.lo_edge[a][(long long)i << sh], g.hi_edge[a][(((long long)i + 1) << sh) - 1]};
}
__device__ __forceinline__ IV<double> sin_phi0(const DevGeom &g, int level, int i) {
    const double *r = g.sincos + 4 * (g.sincos_off[level] + i);
    return {r[0], r[1]};
}
__device__ __forceinline__ IV<double> cos_phi0(const DevGeom &g, int level, int i) {
    const double *r = g.sincos + 4 * (g.sincos_off[level] + i);
    return {r[2], r[3]};
}

// sin / cos of the phi0 centre of cell i at `level` (midpoint form)
__device__ __forceinline__ void sincos_phi0_centre(const DevGeom &g, int level, int i, double &s, double &c) {
    const double *r = g.sincos_mid + 2 * (g.sincos_off[level] + i);
    s = r[0];
    c = r[1];
}

// Conversion of an FP64 interval to the working precision (outward for FP32).
template <typename T> __device__ __forceinline__ IV<T> to_prec(IV<double> a);
template <> __device__ __forceinline__ IV<double> to_prec<double>(IV<double> a) { return a; }
template <> __device__ __forceinline__ IV<float> to_prec<float>(IV<double> a) {
    return {__double2float_rd(a.lo), __double2float_ru(a.hi)};
}

template <typename T> __device__ __forceinline__ Hit<T> load_hit(const void *rec);
template <> __device__ __forceinline__ Hit<double> load_hit<double>(const void *rec) {
    const HitRecD &r = *reinterpret_cast<const HitRecD *>(rec);
    Hit<double> h;
    IV<double> *f = &h.x0;
#pragma unroll
    for (int i = 0; i < 9; i++) f[i] = {r.v[i], r.v[i]};
    return h;
}
template <> __device__ __forceinline__ Hit<float> load_hit<float>(const void *rec) {
    const HitRecF &r = *reinterpret_cast<const HitRecF *>(rec);
    Hit<float> h;
    IV<float> *f = &h.x0;
#pragma unroll
    for (int i = 0; i < 9; i++) f[i] = {r.lo[i], r.hi[i]};
    return h;
}

// Cell key: idx_a << key_shift[a]; axis a is key_bits[a] = max(10, ceil(log2(bins_a <<
// levels))) wide, d0 lowest, so the level-0 linear order (d0 fastest) is the key order.
__device__ __forceinline__ uint64_t pack_key(const DevGeom &g, const int idx[5]) {
    uint64_t k = 0;
#pragma unroll
    for (int a = 0; a < 5; a++) k |= (uint64_t)idx[a] << g.key_shift[a];
    return k;
}
__device__ __forceinline__ void unpack_key(const DevGeom &g, uint64_t k, int idx[5]) {
#pragma unroll
    for (int a = 0; a < 5; a++) idx[a] = (int)((k >> g.key_shift[a]) & ((1u << g.key_bits[a]) - 1u));
}

// Status words written by kernels (bit flags, OR-ed into a device word).
enum : unsigned { ST_TIMEOUT = 1u, ST_BADHIT = 2u, ST_TOOMANY = 4u, ST_BADOFFS = 8u };

// ---- launch wrappers (kernels.cu) ----
// hit_track (may be null): set to -1 for every hit of the batch
void launch_stage(const DevGeom &g, int n_events, const int32_t *offsets, const int32_t *wire_id,
                  const double *drift, HitRecD *hd, HitRecF *hf, int32_t *n_hits,
                  uint32_t *active, int32_t *done, unsigned *status, cudaStream_t s,
                  int32_t *hit_track = nullptr);
// active: per event 8 words of hit-activity bits (nullptr: every hit active)
// cand_k / cand_v (may be null): instead of every cell's vote, each block writes its K best
// cells by (votes desc, key asc) (unused slots: votes -1), coarse_lists(g, prec) blocks per
// event in order; votes is then unused.  The midpoint form takes no candidates.
void launch_vote_coarse(const DevGeom &g, int prec, int ev0, int n_ev, const HitRecD *hd,
                        const HitRecF *hf, const int32_t *n_hits, int32_t *votes, uint32_t *hist,
                        unsigned *status, cudaStream_t s, unsigned long long *ctr = nullptr,
                        const uint32_t *active = nullptr, uint64_t *cand_k = nullptr,
                        int32_t *cand_v = nullptr, int K = 0);
int coarse_lists(const DevGeom &g, int prec);   // level-0 blocks per event of a precision
// The K best level-0 cells of each event from its blocks' candidates (n_lists x K per
// event) and its histogram of all cells' votes, to out_keys / out_votes (K per event, in
// no particular order; the set is that of launch_select_coarse).
void launch_select_candidates(const DevGeom &g, int ev0, int n_ev, const uint64_t *cand_k,
                              const int32_t *cand_v, int n_lists, const uint32_t *hist, int K,
                              uint64_t *out_keys, int32_t *out_votes, cudaStream_t s);
void launch_vote_keys(const DevGeom &g, int prec, int n_ev, const HitRecD *hd, const HitRecF *hf,
                      const int32_t *n_hits, int level, const uint64_t *keys, long long n_per_ev,
                      int32_t *votes, cudaStream_t s, const uint32_t *active = nullptr);
void launch_vote_children(const DevGeom &g, int prec, int n_ev, const HitRecD *hd,
                          const HitRecF *hf, const int32_t *n_hits, int child_level,
                          const uint64_t *parents, int n_par, uint64_t *child_keys,
                          int32_t *child_votes, cudaStream_t s, const uint32_t *active = nullptr,
                          int block = 256, const int32_t *n_valid = nullptr);
void init_kernel_attributes();
void launch_wait_never(long limit, unsigned *status, cudaStream_t s);
void launch_select_coarse(const DevGeom &g, int ev0, int n_ev, const int32_t *votes,
                          const uint32_t *hist, int K, uint64_t *out_keys, int32_t *out_votes,
                          cudaStream_t s);
void launch_topk(int n_ev, const uint64_t *keys, const int32_t *votes, int n_in, int K,
                 uint64_t *out_keys, int32_t *out_votes, cudaStream_t s);
// offsets / hit_track (hit_track may be null): the batch's CSR offsets of these events and
// the per-hit track index, written for the hits this round's track takes
void launch_estimate_mask(const DevGeom &g, int n_ev, const uint64_t *keys, const int32_t *votes,
                          int n_in, int level, const int32_t *n_hits, uint32_t *active, int32_t *done,
                          const HitRecD *hd, int round, int max_tracks, int min_votes, double width,
                          apo_track *out, int32_t *n_tracks, cudaStream_t s,
                          const int32_t *offsets = nullptr, int32_t *hit_track = nullptr);
void launch_series_consts(SeriesConsts *dev_out, cudaStream_t s);

// maxset.cu: one level of the max-set schedule for n_ev events (pointers already offset to
// the first of them).  votes / keys: the level's cells, stride cells per event (keys null:
// the level-0 grid in linear order, n_coarse per event); count_in (levels >= 1): parents of
// each event, so 32 x count_in[e] children.  Writes the kept cells to front (max_keep per
// event) and their number to count_out, or, at the end of an event's search, its track,
// n_tracks (1 when vmax >= min_votes), final_level and n_final, and sets stop.
// One event's pending track step: flag (1: its search ended at this level and it has a
// track), the final vmax, the level's cell count, the track's cell count, S (the seed
// cell's voting hits) and the hits taken so far.
struct TrackStep {
    int32_t flag, vmax, n, mc;
    uint32_t S[8], take[8];
};
struct MaxsetArgs {
    int level, levels, max_keep, slack, min_votes;
    long long n_coarse, stride;
    int32_t *votes;                // the level's votes (the multi-track step marks cells in it)
    const uint64_t *keys;
    const int32_t *count_in;
    uint64_t *front;
    int32_t *count_out, *stop;
    const int32_t *n_hits;
    apo_track *tracks;             // events x max_tracks
    int32_t *n_tracks, *final_level, *n_final;   // the last two: events x max_tracks
    uint64_t *trace_keys;          // may be null: events x (levels + 1) x max_keep
    int32_t *trace_votes, *trace_count;
    // multi-track extraction (max_tracks > 1): round, the level's precision code (no flag),
    // 3 sigma, the events' active-hit words, done flags, staged hits, batch offsets of the
    // events' first hits and the hit_track output (may be null)
    int max_tracks, round, prec;
    double width;
    uint32_t *active;
    int32_t *done;
    const HitRecD *hd;
    const HitRecF *hf;
    const int32_t *offsets;
    int32_t *hit_track;
    // the round's track step (max_tracks > 1): per event of the chunk, set by the selection
    // when its search ends, finished by k_track_cells / k_track_finish; per-axis index
    // counters (cnt_stride each, zero between uses)
    TrackStep *ts;
    uint32_t *tcnt;
    int cnt_stride;
};
// Persistent batch search (kernels.cu): the top-K schedule with multi-track rounds, every
// event's whole search in one block, blocks pulling events from next_event (zeroed by the
// host).  mode[L]: the vote kernel mode of level L (FP32, FP64 or FP32-filtered FP64).
// votes / hist: per-block scratch (blocks x level-0 cells, blocks x kHistBins).
enum : int { kPersistF32 = 0, kPersistF64 = 1, kPersistF64Filtered = 2 };   // the vote kernel modes
struct PersistArgs {
    int n_events, max_tracks, min_votes;
    double width;
    int mode[kMaxLevels + 1];
    const HitRecD *hd;
    const HitRecF *hf;
    const int32_t *n_hits, *offsets;
    uint32_t *active;
    int32_t *done, *next_event;
    unsigned *status;
    int32_t *votes;
    uint32_t *hist;
    uint64_t *fk, *ck;
    int32_t *fv, *cv;
    apo_track *tracks;
    int32_t *n_tracks, *hit_track;
};
size_t persist_smem_bytes(const DevGeom &g);
int persist_blocks(const DevGeom &g);   // blocks resident at once on the current device
void launch_solve_persistent(const DevGeom &g, int blocks, const PersistArgs &A, cudaStream_t s);
size_t maxset_smem_bytes(const DevGeom &g);
void launch_maxset_select(const DevGeom &g, int n_ev, const MaxsetArgs &A, cudaStream_t s);
// The multi-track round's track step after each level's selection: the track's cells (every
// vmax cell that all hits of S vote for) with the hit finding over them, then the estimate
// and the active-hit update.  Events without a pending step return at once.
void launch_track_step(const DevGeom &g, int n_ev, const MaxsetArgs &A, cudaStream_t s);
void init_maxset_attributes();
double pipe_peak(int precision, int op);   // diag.cu: directed operations per second
int launch_dops(int op, const double *x, double *out, long long n, cudaStream_t s);   // diag.cu
int launch_pair_ends(const SeriesConsts &k, int precision, const double *cells, const double *hits,
                     double *out, long long n, cudaStream_t s);                        // diag.cu

// apo_abi.cu: the device tables and device ordinal of a geometry handle, and the message
// returned by apo_last_error() on this thread.
const DevGeom *geometry_device_tables(const apo_geometry *g, int *device);
void set_last_error(const char *msg);
void launch_hist(int n_ev, const int32_t *votes, long long n, uint32_t *hist, cudaStream_t s);
void launch_children(const DevGeom &g, const uint64_t *keys, long long n, uint64_t *out, cudaStream_t s);

}  // namespace apo
