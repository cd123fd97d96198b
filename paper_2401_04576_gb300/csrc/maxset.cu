// Max-set schedule (Section 3.3: the result is the set of maximum-vote voxels): per event
// and level, keep whole vote groups {votes >= T} of the level's cells, at most max_keep of
// them, T >= vmax - slack; when even the vmax group does not fit, or at the last level, the
// search ends and the estimate is taken over that level's vmax group.
//
// One block per event.  Pass 1 builds the histogram of vote counts (257 bins) in shared
// memory; thread 0 picks T.  Pass 2 is an order-preserving compaction of the kept cells
// into the frontier (4096-cell tiles, block scan), or, at the end, per-axis counters of the
// vmax group's cell indices, from which one warp per axis sums count x centre in ascending
// index order: the mean of the group's cell centres with a summation order fixed by the
// indices, so the result does not depend on the order the cells arrive in.
//
// Multi-track extraction (max_tracks > 1, one search per round on the hits still active):
// the final vmax group can hold several tracks' cells (tracks with equal hit counts tie),
// so a round keeps one of them.  The seed is the group's lowest key, S the active hits
// that vote for it at the level's precision, and the track's cells are the group's cells
// that every hit of S votes for (each has vmax votes, so its voting hits are exactly S).
// The selection finds the seed and S; k_track_cells (many blocks per event) finds the
// track's cells, counts their indices per axis and runs the hit finding over them;
// k_track_finish takes the estimate as above.  The track takes S and every active hit
// that votes (FP64) for one of its cells with the drift widened by 3 sigma (Section 3.3's
// hit finding); those hits leave the active set.
#include <cuda_runtime.h>

#include <climits>

#include "kernels.cuh"

namespace apo {

namespace {

constexpr int kMsThreads = 1024;
constexpr int kMsTile = 4 * kMsThreads;

// index of the j-th cell of the event at this level: level 0 in linear order, else a key
__device__ __forceinline__ void cell_index(const DevGeom &g, const uint64_t *keys, long long j, int idx[5]) {
    if (!keys) {
        long long r = j;
#pragma unroll
        for (int a = 0; a < 5; a++) { idx[a] = (int)(r % g.bins[a]); r /= g.bins[a]; }
    } else {
        unpack_key(g, keys[j], idx);
    }
}

__device__ __forceinline__ int clamp_votes(int v) { return v < 0 ? 0 : (v > kHitCap ? kHitCap : v); }

__device__ __forceinline__ Cell<double> cell_at(const DevGeom &g, int level, const int idx[5]) {
    return Cell<double>{edge(g, 0, level, idx[0]), sin_phi0(g, level, idx[1]), cos_phi0(g, level, idx[1]),
                        edge(g, 2, level, idx[2]), edge(g, 3, level, idx[3]), edge(g, 4, level, idx[4])};
}

__device__ __forceinline__ Cell<float> cell32(const Cell<double> &c) {
    return Cell<float>{to_prec<float>(c.D), to_prec<float>(c.S0), to_prec<float>(c.C0), to_prec<float>(c.W),
                       to_prec<float>(c.Z), to_prec<float>(c.L)};
}

// The vote of staged hit i for a cell at the level's precision code, as the voting
// kernels count it (FP32 cells are the FP64 edges rounded outward; the FP32-filtered mode
// votes as FP64).  FP64 (expansion) votes are decided by the FP32 program first: its
// intervals contain the FP64 ones, so an FP32 refusal is an FP64 refusal.
__device__ __forceinline__ bool vote_at(const DevGeom &g, int prec, const Cell<double> &c, const HitRecD *hd,
                                        const HitRecF *hf, int i) {
    if (prec == APO_F32) return vote_pair<float>(cell32(c), load_hit<float>(hf + i), g.k);
    if (prec == APO_F64_EXACT) return vote_pair_exact(c, load_hit<double>(hd + i), g.k);
    if (!vote_pair<float>(cell32(c), load_hit<float>(hf + i), g.k)) return false;
    return vote_pair<double>(c, load_hit<double>(hd + i), g.k);
}

// The FP64 vote of staged hit i for a cell with its drift widened to [max(rd(d - width),
// 0), ru(d + width)] (the hit finding), decided by the FP32 program on the outward-rounded
// FP32 copy of that interval first.
__device__ __forceinline__ bool vote_widened(const DevGeom &g, const Cell<double> &c, const Cell<float> &c32,
                                             const HitRecD *hd, const HitRecF *hf, int i, double width) {
    Hit<double> h = load_hit<double>(hd + i);
    const double d = h.d.lo;
    const double dlo = __dsub_rd(d, width);
    h.d = {gt0(dlo) ? dlo : 0.0, __dadd_ru(d, width)};
    Hit<float> h32 = load_hit<float>(hf + i);
    h32.d = {__double2float_rd(h.d.lo), __double2float_ru(h.d.hi)};
    if (!vote_pair<float>(c32, h32, g.k)) return false;
    return vote_pair<double>(c, h, g.k);
}

// Estimate from per-axis index counters (off[a] .. off[a + 1] - 1 hold axis a's bins at
// `level`): warp a < 5 walks axis a's nonzero bins in ascending index order and sums
// count x centre in round-to-nearest; value = sum / m, error = half the extent of the bins
// present.  Written when vmax >= min_votes.
__device__ __forceinline__ void ordered_estimate(const DevGeom &g, int level, int sh, const int off[6],
                                                 const uint32_t *cnt, int vmax, int m, int min_votes,
                                                 apo_track &t, int wid, int lane) {
    (void)level;
    if (wid >= 5) return;
    const int a = wid, nb = off[a + 1] - off[a];
    const uint32_t *ca = cnt + off[a];
    double sum = 0.0, lo_min = 0.0, hi_max = 0.0;
    bool first = true;
    for (int i0 = 0; i0 < nb; i0 += 32) {
        const int i = i0 + lane;
        const uint32_t c = i < nb ? ca[i] : 0u;
        unsigned msk = __ballot_sync(0xffffffffu, c != 0u);
        while (msk) {   // every lane walks the chunk's nonzero bins in index order
            const int b = __ffs(msk) - 1;
            msk &= msk - 1;
            const int ib = i0 + b;
            const uint32_t cb = __shfl_sync(0xffffffffu, c, b);
            const double lo = g.lo_edge[a][(long long)ib << sh];
            const double hi = g.hi_edge[a][(((long long)ib + 1) << sh) - 1];
            sum = __dadd_rn(sum, __dmul_rn((double)cb, __dmul_rn(__dadd_rn(lo, hi), 0.5)));
            if (first) { lo_min = lo; first = false; }
            hi_max = hi;
        }
    }
    if (lane == 0 && vmax >= min_votes) {
        t.p[a] = __ddiv_rn(sum, (double)m);
        t.w[a] = __dmul_rn(__dsub_rn(hi_max, lo_min), 0.5);
    }
}

__global__ void __launch_bounds__(kMsThreads)
k_maxset_select(DevGeom g, MaxsetArgs A) {
    extern __shared__ __align__(16) unsigned char smem[];
    uint32_t *cnt = reinterpret_cast<uint32_t *>(smem);    // per-axis index counters
    __shared__ uint32_t hist[kHistBins];
    __shared__ int s_warp[32];
    __shared__ int s_T, s_final, s_vmax, s_kept;
    const int e = blockIdx.x, tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    if (A.stop[e]) return;
    const int mt = A.max_tracks;
    if (A.done && A.done[e]) {   // a later round of an event whose extraction has ended
        if (tid == 0) {
            A.stop[e] = 1;
            A.count_out[e] = 0;
        }
        return;
    }
    const int nh = A.n_hits[e];
    apo_track *te = A.tracks + (long long)e * mt;
    apo_track &t = te[A.round];
    if (A.level == 0 && A.round == 0) {
        for (int q = tid; q < 5 * mt; q += kMsThreads) {
            te[q / 5].p[q % 5] = 0.0;
            te[q / 5].w[q % 5] = 0.0;
        }
        if (tid < mt) {
            te[tid].votes = (tid == 0 && nh < 0) ? nh : 0;
            te[tid].n_hits = nh < 0 ? 0 : nh;
        }
        if (tid == 0) A.n_tracks[e] = 0;
        if (nh < 0) {   // malformed event: no search
            if (tid == 0) {
                A.stop[e] = 1;
                A.count_out[e] = 0;
                if (A.final_level) A.final_level[(long long)e * mt] = 0;
                if (A.done) A.done[e] = 1;
            }
            return;
        }
    }
    const long long n = A.keys ? 32LL * A.count_in[e] : A.n_coarse;
    const int32_t *vo = A.votes + (long long)e * A.stride;
    const uint64_t *ke = A.keys ? A.keys + (long long)e * A.stride : nullptr;
    for (int i = tid; i < kHistBins; i += kMsThreads) hist[i] = 0;
    __syncthreads();
    for (long long j = tid; j < n; j += kMsThreads) atomicAdd(&hist[clamp_votes(vo[j])], 1u);
    __syncthreads();
    if (tid == 0) {
        int vmax = 0;
        for (int v = kHistBins - 1; v > 0; v--)
            if (hist[v]) { vmax = v; break; }
        const bool fin = A.level == A.levels || (long long)hist[vmax] > A.max_keep;
        int T = vmax;
        long long kept = hist[vmax];
        if (!fin) {
            int lb = vmax - A.slack;
            const int floor1 = vmax < 1 ? vmax : 1;
            if (lb < floor1) lb = floor1;
            while (T - 1 >= lb && kept + hist[T - 1] <= A.max_keep) { T--; kept += hist[T]; }
        }
        s_T = T;
        s_final = fin;
        s_vmax = vmax;
        s_kept = (int)kept;
    }
    __syncthreads();
    const int T = s_T, vmax = s_vmax, kept = s_kept;
    if (s_final) {
        if (mt > 1) {
            // ---- multi-track: the seed and S here; the track step kernels do the rest ----
            __shared__ unsigned long long s_seed;
            __shared__ uint32_t s_act[8], s_S[8];
            if (vmax < A.min_votes) {   // no track this round: the extraction ends
                if (tid < 8) A.active[(long long)e * 8 + tid] = 0u;   // later rounds vote no hit
                if (tid == 0) {
                    A.stop[e] = 1;
                    A.count_out[e] = 0;
                    A.done[e] = 1;
                }
                return;
            }
            const HitRecD *hde = A.hd + (long long)e * kHitCap;
            const HitRecF *hfe = A.hf + (long long)e * kHitCap;
            if (tid == 0) s_seed = ~0ull;
            if (tid < 8) { s_act[tid] = A.active[(long long)e * 8 + tid]; s_S[tid] = 0u; }
            __syncthreads();
            // the seed: the group's lowest key
            unsigned long long kmin = ~0ull;
            for (long long j = tid; j < n; j += kMsThreads) {
                if (clamp_votes(vo[j]) != vmax) continue;
                int idx[5];
                cell_index(g, ke, j, idx);
                const unsigned long long key = pack_key(g, idx);
                kmin = key < kmin ? key : kmin;
            }
            atomicMin(&s_seed, kmin);
            __syncthreads();
            // S: the active hits that vote for it, one hit per thread
            {
                int idx[5];
                unpack_key(g, s_seed, idx);
                const Cell<double> cs = cell_at(g, A.level, idx);
                for (int i = tid; i < nh; i += kMsThreads)
                    if (((s_act[i >> 5] >> (i & 31)) & 1u) && vote_at(g, A.prec, cs, hde, hfe, i))
                        atomicOr(&s_S[i >> 5], 1u << (i & 31));
            }
            __syncthreads();
            TrackStep &ts = A.ts[e];
            if (tid < 8) { ts.S[tid] = s_S[tid]; ts.take[tid] = s_S[tid]; }
            if (tid == 0) {
                ts.flag = 1;
                ts.vmax = vmax;
                ts.n = (int)n;
                ts.mc = 0;
                A.stop[e] = 1;
                A.count_out[e] = 0;
            }
            return;
        }
        // ---- estimate over the vmax group ----
        const int sh = g.levels - A.level;
        int off[6];
        off[0] = 0;
#pragma unroll
        for (int a = 0; a < 5; a++) off[a + 1] = off[a] + (g.bins[a] << A.level);
        for (int i = tid; i < off[5]; i += kMsThreads) cnt[i] = 0;
        __syncthreads();
        for (long long j = tid; j < n; j += kMsThreads) {
            if (clamp_votes(vo[j]) != vmax) continue;
            int idx[5];
            cell_index(g, ke, j, idx);
#pragma unroll
            for (int a = 0; a < 5; a++) atomicAdd(&cnt[off[a] + idx[a]], 1u);
        }
        __syncthreads();
        ordered_estimate(g, A.level, sh, off, cnt, vmax, kept, A.min_votes, t, wid, lane);
        if (tid == 0) {
            if (vmax >= A.min_votes) {
                t.votes = vmax;
                A.n_tracks[e] = A.round + 1;
            }
            A.stop[e] = 1;
            A.count_out[e] = 0;
            if (A.final_level) A.final_level[(long long)e * mt + A.round] = A.level;
            if (A.n_final) A.n_final[(long long)e * mt + A.round] = kept;
        }
        return;
    }
    // ---- order-preserving compaction of {votes >= T} ----
    uint64_t *fe = A.front + (long long)e * A.max_keep;
    uint64_t *tk = A.trace_keys ? A.trace_keys + ((long long)e * (A.levels + 1) + A.level) * A.max_keep : nullptr;
    int32_t *tv = A.trace_votes ? A.trace_votes + ((long long)e * (A.levels + 1) + A.level) * A.max_keep : nullptr;
    int run = 0;
    for (long long t0 = 0; t0 < n && run < kept; t0 += kMsTile) {
        const long long j0 = t0 + 4LL * tid;
        int v[4], x = 0;
#pragma unroll
        for (int r = 0; r < 4; r++) {
            v[r] = j0 + r < n ? clamp_votes(vo[j0 + r]) : -1;
            x += v[r] >= T;
        }
        if (!__syncthreads_or(x > 0)) continue;
        int inc = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += y;
        }
        if (lane == 31) s_warp[wid] = inc;
        __syncthreads();
        const int w = s_warp[lane];
        int winc = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, winc, o);
            if (lane >= o) winc += y;
        }
        const int wpre = __shfl_sync(0xffffffffu, winc - w, wid);
        const int total = __shfl_sync(0xffffffffu, winc, 31);
        int pos = run + wpre + inc - x;
#pragma unroll
        for (int r = 0; r < 4; r++) {
            if (v[r] < T) continue;
            int idx[5];
            cell_index(g, ke, j0 + r, idx);
            const uint64_t key = pack_key(g, idx);
            fe[pos] = key;
            if (tk) tk[pos] = key;
            if (tv) tv[pos] = v[r];
            pos++;
        }
        run += total;
        __syncthreads();   // s_warp is rewritten by the next scanned tile
    }
    if (tid == 0) {
        A.count_out[e] = kept;
        if (A.trace_count) A.trace_count[(long long)e * (A.levels + 1) + A.level] = kept;
    }
}

constexpr int kTsThreads = 128;
constexpr int kTsBlocks = 96;    // blocks per event of the track-cell kernel
constexpr int kTsChunk = 2048;   // cells a block scans per pass
constexpr int kTfThreads = 192;  // the step's end: one warp per axis for the estimate

// The track's cells of every event with a pending step: each vmax cell of the level is
// tested against the hits of S (at the level's precision, stopping at the first that does
// not vote); a track cell adds its indices to the event's per-axis counters and takes
// every active hit not yet taken that votes (FP64) for it with the drift widened by 3 sigma.
// Each block scans its cells in chunks of kTsChunk: the chunk's vmax cells are queued in
// shared memory, the queue is tested one cell per thread, and the hit finding runs over
// the (track cell, hit) pairs one pair per thread, so that whole warps do the votes.
__global__ void __launch_bounds__(kTsThreads, 3)
k_track_cells(DevGeom g, MaxsetArgs A) {
    const int e = blockIdx.y, tid = threadIdx.x;
    TrackStep &ts = A.ts[e];
    if (!ts.flag) return;
    __shared__ uint32_t s_S[8];
    __shared__ int s_q[kTsChunk], s_t[kTsChunk];
    __shared__ unsigned char s_hit[kHitCap];
    __shared__ int s_mc, s_nq, s_nt, s_na;
    const int nh = A.n_hits[e];
    if (tid < 8) s_S[tid] = ts.S[tid];
    if (tid == 0) {   // the active hits outside S (S is taken already), in index order
        s_mc = 0;
        int na = 0;
        for (int i = 0; i < nh; i++) {
            const uint32_t bit = 1u << (i & 31);
            if ((A.active[(long long)e * 8 + (i >> 5)] & bit) && !(ts.S[i >> 5] & bit)) s_hit[na++] = (unsigned char)i;
        }
        s_na = na;
    }
    __syncthreads();
    const int vmax = ts.vmax, na = s_na;
    const long long n = ts.n;
    const int32_t *vo = A.votes + (long long)e * A.stride;
    const uint64_t *ke = A.keys ? A.keys + (long long)e * A.stride : nullptr;
    const HitRecD *hde = A.hd + (long long)e * kHitCap;
    const HitRecF *hfe = A.hf + (long long)e * kHitCap;
    uint32_t *cnt = A.tcnt + (long long)e * A.cnt_stride;
    volatile uint32_t *take = ts.take;
    int off[6];
    off[0] = 0;
#pragma unroll
    for (int a = 0; a < 5; a++) off[a + 1] = off[a] + (g.bins[a] << A.level);
    int mc = 0;
    for (long long base = (long long)blockIdx.x * kTsChunk; base < n; base += (long long)gridDim.x * kTsChunk) {
        if (tid == 0) { s_nq = 0; s_nt = 0; }
        __syncthreads();
        // the chunk's vmax cells
        for (int k = tid; k < kTsChunk; k += kTsThreads) {
            const long long j = base + k;
            if (j < n && clamp_votes(vo[j]) == vmax) s_q[atomicAdd(&s_nq, 1)] = k;
        }
        __syncthreads();
        // the cluster test, one queued cell per thread
        const int nq = s_nq;
        for (int q = tid; q < nq; q += kTsThreads) {
            int idx[5];
            cell_index(g, ke, base + s_q[q], idx);
            const Cell<double> c = cell_at(g, A.level, idx);
            bool ok = true;
            for (int w8 = 0; w8 < 8 && ok; w8++) {
                uint32_t m = s_S[w8];
                while (m && ok) {
                    const int i = w8 * 32 + __ffs(m) - 1;
                    m &= m - 1;
                    ok = vote_at(g, A.prec, c, hde, hfe, i);
                }
            }
            if (!ok) continue;
            s_t[atomicAdd(&s_nt, 1)] = s_q[q];
            mc++;
#pragma unroll
            for (int a = 0; a < 5; a++) atomicAdd(&cnt[off[a] + idx[a]], 1u);
        }
        __syncthreads();
        // the hit finding over (track cell, listed hit) pairs, one pair per thread
        const long long np = (long long)s_nt * na;
        for (long long pr = tid; pr < np; pr += kTsThreads) {
            const int q = (int)(pr / na), i = s_hit[pr % na];
            const uint32_t bit = 1u << (i & 31);
            if (take[i >> 5] & bit) continue;
            int idx[5];
            cell_index(g, ke, base + s_t[q], idx);
            const Cell<double> c = cell_at(g, A.level, idx);
            if (vote_widened(g, c, cell32(c), hde, hfe, i, A.width)) atomicOr(&ts.take[i >> 5], bit);
        }
        __syncthreads();   // the queues are refilled by the next chunk
    }
    if (mc) atomicAdd(&s_mc, mc);
    __syncthreads();
    if (tid == 0 && s_mc) atomicAdd(&ts.mc, s_mc);
}

// The step's end: the estimate over the track's cells (per-axis counters, ordered sums),
// the record, the active-hit update, hit_track and the done flag; the counters and the
// flag are cleared for the next use.
__global__ void __launch_bounds__(kTfThreads)
k_track_finish(DevGeom g, MaxsetArgs A) {
    const int e = blockIdx.x, tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    TrackStep &ts = A.ts[e];
    if (!ts.flag) return;
    const int mt = A.max_tracks;
    apo_track &t = A.tracks[(long long)e * mt + A.round];
    uint32_t *cnt = A.tcnt + (long long)e * A.cnt_stride;
    const int sh = g.levels - A.level;
    int off[6];
    off[0] = 0;
#pragma unroll
    for (int a = 0; a < 5; a++) off[a + 1] = off[a] + (g.bins[a] << A.level);
    const int vmax = ts.vmax, mc = ts.mc;
    ordered_estimate(g, A.level, sh, off, cnt, vmax, mc, A.min_votes, t, wid, lane);
    __shared__ int s_left;
    if (tid == 0) s_left = 0;
    __syncthreads();
    for (int i = tid; i < off[5]; i += kTfThreads) cnt[i] = 0u;
    if (tid < 8) {
        const uint32_t act = A.active[(long long)e * 8 + tid];
        const uint32_t took = act & ts.take[tid], left = act & ~ts.take[tid];
        A.active[(long long)e * 8 + tid] = left;
        if (left) atomicOr(&s_left, 1);
        if (A.hit_track) {
            const int a0 = A.offsets[e];
            uint32_t m = took;
            while (m) {
                const int i = tid * 32 + __ffs(m) - 1;
                m &= m - 1;
                A.hit_track[a0 + i] = A.round;
            }
        }
    }
    __syncthreads();
    if (tid == 0) {
        t.votes = vmax;
        A.n_tracks[e] = A.round + 1;
        if (A.final_level) A.final_level[(long long)e * mt + A.round] = A.level;
        if (A.n_final) A.n_final[(long long)e * mt + A.round] = mc;
        if (!s_left || A.round + 1 >= mt) A.done[e] = 1;
        ts.flag = 0;
    }
}

}  // namespace

size_t maxset_smem_bytes(const DevGeom &g) {
    size_t n = 0;
    for (int a = 0; a < 5; a++) n += (size_t)g.bins[a] << g.levels;
    return n * sizeof(uint32_t);
}

void init_maxset_attributes() {
    cudaFuncSetAttribute(k_maxset_select, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024);
}

void launch_maxset_select(const DevGeom &g, int n_ev, const MaxsetArgs &A, cudaStream_t s) {
    if (n_ev <= 0) return;
    k_maxset_select<<<n_ev, kMsThreads, maxset_smem_bytes(g), s>>>(g, A);
}

void launch_track_step(const DevGeom &g, int n_ev, const MaxsetArgs &A, cudaStream_t s) {
    if (n_ev <= 0) return;
    k_track_cells<<<dim3(kTsBlocks, n_ev), kTsThreads, 0, s>>>(g, A);
    k_track_finish<<<n_ev, kTfThreads, 0, s>>>(g, A);
}

}  // namespace apo
