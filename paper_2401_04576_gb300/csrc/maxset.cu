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

__global__ void __launch_bounds__(kMsThreads)
k_maxset_select(DevGeom g, MaxsetArgs A) {
    extern __shared__ __align__(16) unsigned char smem[];
    uint32_t *cnt = reinterpret_cast<uint32_t *>(smem);    // per-axis index counters
    __shared__ uint32_t hist[kHistBins];
    __shared__ int s_warp[32];
    __shared__ int s_T, s_final, s_vmax, s_kept;
    const int e = blockIdx.x, tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    if (A.stop[e]) return;
    const int nh = A.n_hits[e];
    apo_track &t = A.tracks[e];
    if (A.level == 0) {
        if (tid < 5) { t.p[tid] = 0.0; t.w[tid] = 0.0; }
        if (tid == 0) {
            t.votes = nh < 0 ? nh : 0;
            t.n_hits = nh < 0 ? 0 : nh;
            A.n_tracks[e] = 0;
        }
        if (nh < 0) {   // malformed event: no search
            if (tid == 0) {
                A.stop[e] = 1;
                A.count_out[e] = 0;
                if (A.final_level) A.final_level[e] = 0;
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
        if (wid < 5) {
            const int a = wid, nb = off[a + 1] - off[a];
            const uint32_t *ca = cnt + off[a];
            double sum = 0.0, lo_min = 0.0, hi_max = 0.0;
            bool first = true;
            for (int i0 = 0; i0 < nb; i0 += 32) {
                const int i = i0 + lane;
                const uint32_t c = i < nb ? ca[i] : 0u;
                unsigned m = __ballot_sync(0xffffffffu, c != 0u);
                while (m) {   // every lane walks the chunk's nonzero bins in index order
                    const int b = __ffs(m) - 1;
                    m &= m - 1;
                    const int ib = i0 + b;
                    const uint32_t cb = __shfl_sync(0xffffffffu, c, b);
                    const double lo = g.lo_edge[a][(long long)ib << sh];
                    const double hi = g.hi_edge[a][(((long long)ib + 1) << sh) - 1];
                    sum = __dadd_rn(sum, __dmul_rn((double)cb, __dmul_rn(__dadd_rn(lo, hi), 0.5)));
                    if (first) { lo_min = lo; first = false; }
                    hi_max = hi;
                }
            }
            if (lane == 0 && vmax >= A.min_votes) {
                t.p[a] = __ddiv_rn(sum, (double)kept);
                t.w[a] = __dmul_rn(__dsub_rn(hi_max, lo_min), 0.5);
            }
        }
        if (tid == 0) {
            if (vmax >= A.min_votes) {
                t.votes = vmax;
                A.n_tracks[e] = 1;
            }
            A.stop[e] = 1;
            A.count_out[e] = 0;
            if (A.final_level) A.final_level[e] = A.level;
            if (A.n_final) A.n_final[e] = kept;
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

}  // namespace apo
