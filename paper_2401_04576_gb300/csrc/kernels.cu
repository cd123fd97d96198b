// sm_103a kernels of the interval-voting hot path (arXiv:2401.04576, Section 3.1):
// hit staging, coarse-grid voting, voting of explicit / bisected cells, top-K selection and
// the final max-vote estimate.
#include <cuda_runtime.h>

#include "../../include/apo.h"
#include "kernels.cuh"

namespace apo {

// ---------------------------------------------------------------------------------------
// Bulk (TMA) copy global -> shared with an mbarrier, every wait bounded.
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ unsigned smem_u32(const void *p) {
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
constexpr long kWaitLimit = 1L << 22;

// Copies `bytes` (multiple of 16, 16-byte aligned ends) of an event's hit records into
// shared memory.  Returns false (and flags ST_TIMEOUT) if the copy did not complete within
// the wait limit; the caller then skips the block's work.
__device__ bool stage_to_smem(void *dst, const void *src, unsigned bytes, uint64_t *bar,
                              unsigned *status) {
    if (threadIdx.x == 0) {
        mbar_init(bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();
    if (bytes == 0) return true;
    if (threadIdx.x == 0) {
        mbar_expect_tx(bar, bytes);
        bulk_g2s(dst, src, bytes, bar);
    }
    long it = 0;
    while (!mbar_try_wait(bar, 0)) {
        if (++it > kWaitLimit) {
            atomicOr(status, ST_TIMEOUT);
            // give the copy in flight a second bounded chance before leaving the smem
            for (long j = 0; j < kWaitLimit && !mbar_try_wait(bar, 0); j++) {
            }
            return false;
        }
    }
    return true;
}

// ---------------------------------------------------------------------------------------
// Series constants [rd(1/k), ru(1/k)] computed once on the device.
// ---------------------------------------------------------------------------------------
__global__ void k_series_consts(SeriesConsts *out) {
    int i = threadIdx.x;
    if (i < 16) {
        int k = series_divisor(i);
        out->d_lo[i] = __drcp_rd((double)k);
        out->d_hi[i] = __drcp_ru((double)k);
        out->f_lo[i] = __frcp_rd((float)k);
        out->f_hi[i] = __frcp_ru((float)k);
    }
}

void launch_series_consts(SeriesConsts *dev_out, cudaStream_t s) {
    k_series_consts<<<1, 32, 0, s>>>(dev_out);
}

// ---------------------------------------------------------------------------------------
// Stage: gather each event's hits into contiguous FP64 and outward-rounded FP32 records,
// validating wire ids, drifts and hit counts.  n_hits[e] < 0 marks an invalid event.
// ---------------------------------------------------------------------------------------
__global__ void k_stage(DevGeom g, int n_events, const int32_t *offsets, const int32_t *wire_id,
                        const double *drift, HitRecD *hd, HitRecF *hf, int32_t *n_hits,
                        unsigned *status) {
    int e = blockIdx.x;
    if (e >= n_events) return;
    __shared__ int bad;
    if (threadIdx.x == 0) bad = 0;
    __syncthreads();
    int a = offsets[e], b = offsets[e + 1];
    int n = b - a;
    if (n < 0 || a < 0) {
        if (threadIdx.x == 0) { n_hits[e] = APO_EINVAL; atomicOr(status, ST_BADOFFS); }
        return;
    }
    if (n > kHitCap) {
        if (threadIdx.x == 0) { n_hits[e] = APO_EINVAL; atomicOr(status, ST_TOOMANY); }
        return;
    }
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        int w = wire_id[a + i];
        double d = drift[a + i];
        bool ok = (w >= 0 && w < g.n_wires && d >= 0.0 && d <= 1e300);
        if (!ok) { bad = 1; continue; }
        HitRecD rd;
        HitRecF rf;
        for (int j = 0; j < 8; j++) rd.v[j] = g.wire[j][w];
        rd.v[8] = d;
        rd.pad = 0.0;
        for (int j = 0; j < 9; j++) {
            rf.lo[j] = __double2float_rd(rd.v[j]);
            rf.hi[j] = __double2float_ru(rd.v[j]);
        }
        rf.pad[0] = rf.pad[1] = 0.f;
        hd[(long long)e * kHitCap + i] = rd;
        hf[(long long)e * kHitCap + i] = rf;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if (bad) { n_hits[e] = APO_EINVAL; atomicOr(status, ST_BADHIT); }
        else n_hits[e] = n;
    }
}

void launch_stage(const DevGeom &g, int n_events, const int32_t *offsets, const int32_t *wire_id,
                  const double *drift, HitRecD *hd, HitRecF *hf, int32_t *n_hits, unsigned *status,
                  cudaStream_t s) {
    if (n_events <= 0) return;
    k_stage<<<n_events, 128, 0, s>>>(g, n_events, offsets, wire_id, drift, hd, hf, n_hits, status);
}

template <typename T> __device__ __forceinline__ const void *hit_base(const HitRecD *hd, const HitRecF *hf, int ev);
template <> __device__ __forceinline__ const void *hit_base<double>(const HitRecD *hd, const HitRecF *, int ev) {
    return hd + (long long)ev * kHitCap;
}
template <> __device__ __forceinline__ const void *hit_base<float>(const HitRecD *, const HitRecF *hf, int ev) {
    return hf + (long long)ev * kHitCap;
}

// ---------------------------------------------------------------------------------------
// Coarse-grid voting.  Block = (event, phi0 bin p, omega bin w); thread = (d0 bin, z0 bin);
// each thread loops over the tan(lambda) bins, reusing the tan(lambda)-free prefix of the
// program.  Before that, every hit is tested once on the block's parent cell (all d0, z0,
// tan(lambda) bins joined): interval operations are inclusion-isotonic and the guards only
// fire on a parent when they fire on a child, so a hit that fails there fails on every
// child cell; skipping it leaves every vote unchanged.
// Writes votes[e][lin], lin = d + Bd (p + Bp (w + Bw (z + Bz l))), and the per-event
// histogram of vote counts.
// ---------------------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256)
k_vote_coarse(DevGeom g, int ev0, const HitRecD *hd, const HitRecF *hf, const int32_t *n_hits,
              int32_t *votes, uint32_t *hist, unsigned *status, unsigned long long *ctr) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int Bd = g.bins[0], Bp = g.bins[1], Bw = g.bins[2], Bz = g.bins[3], Bl = g.bins[4];
    const int nthr = Bd * Bz;
    const int e = blockIdx.y, ev = ev0 + e;
    const int p = blockIdx.x % Bp, w = blockIdx.x / Bp;
    const int tid = threadIdx.x;
    unsigned char *hits_s = smem;                                        // kHitCap * 80
    uint32_t *hist_s = reinterpret_cast<uint32_t *>(smem + kHitCap * 80);    // kHistBins
    uint32_t *mask_s = hist_s + kHistBins + 3;                            // 8 words
    uint64_t *bar = reinterpret_cast<uint64_t *>(mask_s + 8);
    IV<T> *Ls = reinterpret_cast<IV<T> *>(bar + 1);                       // Bl
    int32_t *cnt = reinterpret_cast<int32_t *>(Ls + Bl);                  // Bl * nthr

    int nh = n_hits[ev];
    if (nh < 0) nh = 0;
    for (int i = tid; i < kHistBins; i += nthr) hist_s[i] = 0;
    if (tid < 8) mask_s[tid] = 0;
    for (int l = tid; l < Bl; l += nthr) Ls[l] = to_prec<T>(edge(g, 4, 0, l));
    for (int i = tid; i < Bl * nthr; i += nthr) cnt[i] = 0;
    bool ok = stage_to_smem(hits_s, hit_base<T>(hd, hf, ev), (unsigned)nh * 80u, bar, status);
    __syncthreads();
    if (!ok) nh = 0;

    const SeriesConsts &k = g.k;
    const IV<T> S0 = to_prec<T>(sin_phi0(g, 0, p)), C0 = to_prec<T>(cos_phi0(g, 0, p));
    const IV<T> W = to_prec<T>(edge(g, 2, 0, w));
    // parent cell test, one hit per thread
    {
        IV<double> D0 = edge(g, 0, 0, 0), D1 = edge(g, 0, 0, Bd - 1);
        IV<double> Z0 = edge(g, 3, 0, 0), Z1 = edge(g, 3, 0, Bz - 1);
        IV<double> L0 = edge(g, 4, 0, 0), L1 = edge(g, 4, 0, Bl - 1);
        Cell<T> par;
        par.D = to_prec<T>(IV<double>{D0.lo, D1.hi});
        par.S0 = S0;
        par.C0 = C0;
        par.W = W;
        par.Z = to_prec<T>(IV<double>{Z0.lo, Z1.hi});
        par.L = to_prec<T>(IV<double>{L0.lo, L1.hi});
        for (int h = tid; h < nh; h += nthr) {
            Hit<T> hh = load_hit<T>(hits_s + h * 80);
            if (vote_pair<T>(par, hh, k)) atomicOr(&mask_s[h >> 5], 1u << (h & 31));
        }
    }
    __syncthreads();

    const int d = tid % Bd, z = tid / Bd;
    Cell<T> c;
    c.D = to_prec<T>(edge(g, 0, 0, d));
    c.S0 = S0;
    c.C0 = C0;
    c.W = W;
    c.Z = to_prec<T>(edge(g, 3, 0, z));
    c.L = Ls[0];
    const bool mir = mirror_cell(c);
    const bool wguard = !(c.W.lo > T(0));
    const IV<T> R = recip(c.W);
    unsigned n_pre = 0, n_tail = 0;     // work counters (diagnostics only)
    for (int wd = 0; wd < 8; wd++) {
        uint32_t m = mask_s[wd];
        while (m) {
            int h = wd * 32 + __ffs(m) - 1;
            m &= m - 1;
            Hit<T> hh = load_hit<T>(hits_s + h * 80);
            if (mir) mirror_hit(hh);
            Pre<T> pre;
            if (!wguard) pre = prefix<T>(c, hh, k);
            n_pre++;
            if (wguard || pre.guard) {
                for (int l = 0; l < Bl; l++) cnt[l * nthr + tid]++;
                continue;
            }
            n_tail += Bl;
#pragma unroll 1
            for (int l = 0; l < Bl; l++)
                if (tail<T>(pre, Ls[l], hh, R, c.W, k)) cnt[l * nthr + tid]++;
        }
    }
    const long long ncell = (long long)Bd * Bp * Bw * Bz * Bl;
    int32_t *vo = votes + (long long)e * ncell;
    for (int l = 0; l < Bl; l++) {
        int v = cnt[l * nthr + tid];
        long long lin = d + (long long)Bd * (p + (long long)Bp * (w + (long long)Bw * (z + (long long)Bz * l)));
        vo[lin] = v;
        atomicAdd(&hist_s[v], 1u);
    }
    __syncthreads();
    for (int i = tid; i < kHistBins; i += nthr)
        if (hist_s[i]) atomicAdd(&hist[(long long)e * kHistBins + i], hist_s[i]);
    if (ctr) {
        if (tid == 0) atomicAdd(&ctr[0], (unsigned long long)nh);     // parent evaluations
        atomicAdd(&ctr[1], (unsigned long long)n_pre);                // prefix evaluations
        atomicAdd(&ctr[2], (unsigned long long)n_tail);               // tail evaluations
    }
}

template <typename T> static size_t coarse_smem(const DevGeom &g) {
    int nthr = g.bins[0] * g.bins[3];
    return kHitCap * 80 + (kHistBins + 3 + 8) * 4 + 8 + sizeof(IV<T>) * g.bins[4] +
           sizeof(int32_t) * g.bins[4] * nthr + 16;
}

void launch_vote_coarse(const DevGeom &g, int prec, int ev0, int n_ev, const HitRecD *hd,
                        const HitRecF *hf, const int32_t *n_hits, int32_t *votes, uint32_t *hist,
                        unsigned *status, cudaStream_t s, unsigned long long *ctr) {
    if (n_ev <= 0) return;
    dim3 grid(g.bins[1] * g.bins[2], n_ev);
    int nthr = g.bins[0] * g.bins[3];
    if (prec == APO_F64) {
        size_t sm = coarse_smem<double>(g);
        cudaFuncSetAttribute(k_vote_coarse<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        k_vote_coarse<double><<<grid, nthr, sm, s>>>(g, ev0, hd, hf, n_hits, votes, hist, status, ctr);
    } else {
        size_t sm = coarse_smem<float>(g);
        cudaFuncSetAttribute(k_vote_coarse<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        k_vote_coarse<float><<<grid, nthr, sm, s>>>(g, ev0, hd, hf, n_hits, votes, hist, status, ctr);
    }
}

// ---------------------------------------------------------------------------------------
// Voting of explicit cells: either given keys (keys != nullptr, n_per_ev per event) or the
// 32 children of each parent key (parents != nullptr).  Thread = one cell, looping over
// all hits of its event; child keys are written out when parents are given.
// ---------------------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256)
k_vote_cells(DevGeom g, const HitRecD *hd, const HitRecF *hf, const int32_t *n_hits, int level,
             const uint64_t *keys, const uint64_t *parents, long long n_per_ev, uint64_t *out_keys,
             int32_t *out_votes, unsigned *status) {
    extern __shared__ __align__(16) unsigned char smem[];
    unsigned char *hits_s = smem;
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + kHitCap * 80);
    const int ev = blockIdx.y;
    int nh = n_hits[ev];
    if (nh < 0) nh = 0;
    bool ok = stage_to_smem(hits_s, hit_base<T>(hd, hf, ev), (unsigned)nh * 80u, bar, status);
    __syncthreads();
    if (!ok) nh = 0;
    long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n_per_ev) return;
    uint64_t key;
    if (parents) {
        uint64_t pk = parents[(long long)ev * (n_per_ev / 32) + j / 32];
        int idx[5], b = (int)(j % 32);
        unpack_key(pk, idx);
#pragma unroll
        for (int a = 0; a < 5; a++) idx[a] = 2 * idx[a] + ((b >> a) & 1);
        key = pack_key(idx);
    } else {
        key = keys[(long long)ev * n_per_ev + j];
    }
    int idx[5];
    unpack_key(key, idx);
    long long o = (long long)ev * n_per_ev + j;
    bool valid = true;
#pragma unroll
    for (int a = 0; a < 5; a++) valid = valid && idx[a] < (g.bins[a] << level);
    if (!valid) {   // a key outside the grid of this level: no lookup, vote count -1
        out_votes[o] = -1;
        if (out_keys) out_keys[o] = key;
        return;
    }
    Cell<T> c;
    c.D = to_prec<T>(edge(g, 0, level, idx[0]));
    c.S0 = to_prec<T>(sin_phi0(g, level, idx[1]));
    c.C0 = to_prec<T>(cos_phi0(g, level, idx[1]));
    c.W = to_prec<T>(edge(g, 2, level, idx[2]));
    c.Z = to_prec<T>(edge(g, 3, level, idx[3]));
    c.L = to_prec<T>(edge(g, 4, level, idx[4]));
    const SeriesConsts &k = g.k;
    int v = 0;
    for (int h = 0; h < nh; h++) {
        Hit<T> hh = load_hit<T>(hits_s + h * 80);
        v += vote_pair<T>(c, hh, k) ? 1 : 0;
    }
    out_votes[o] = v;
    if (out_keys) out_keys[o] = key;
}

template <typename T>
static void launch_cells(const DevGeom &g, int n_ev, const HitRecD *hd, const HitRecF *hf,
                         const int32_t *n_hits, int level, const uint64_t *keys,
                         const uint64_t *parents, long long n_per_ev, uint64_t *out_keys,
                         int32_t *out_votes, unsigned *status, cudaStream_t s) {
    size_t sm = kHitCap * 80 + 16;
    dim3 grid((unsigned)((n_per_ev + 255) / 256), n_ev);
    k_vote_cells<T><<<grid, 256, sm, s>>>(g, hd, hf, n_hits, level, keys, parents, n_per_ev,
                                           out_keys, out_votes, status);
}

void launch_vote_keys(const DevGeom &g, int prec, int n_ev, const HitRecD *hd, const HitRecF *hf,
                      const int32_t *n_hits, int level, const uint64_t *keys, long long n_per_ev,
                      int32_t *votes, cudaStream_t s) {
    if (n_ev <= 0 || n_per_ev <= 0) return;
    if (prec == APO_F64)
        launch_cells<double>(g, n_ev, hd, hf, n_hits, level, keys, nullptr, n_per_ev, nullptr, votes,
                             nullptr, s);
    else
        launch_cells<float>(g, n_ev, hd, hf, n_hits, level, keys, nullptr, n_per_ev, nullptr, votes,
                            nullptr, s);
}

void launch_vote_children(const DevGeom &g, int prec, int n_ev, const HitRecD *hd,
                          const HitRecF *hf, const int32_t *n_hits, int child_level,
                          const uint64_t *parents, int n_par, uint64_t *child_keys,
                          int32_t *child_votes, cudaStream_t s) {
    if (n_ev <= 0 || n_par <= 0) return;
    long long n = (long long)n_par * 32;
    if (prec == APO_F64)
        launch_cells<double>(g, n_ev, hd, hf, n_hits, child_level, nullptr, parents, n, child_keys,
                             child_votes, nullptr, s);
    else
        launch_cells<float>(g, n_ev, hd, hf, n_hits, child_level, nullptr, parents, n, child_keys,
                            child_votes, nullptr, s);
}

// ---------------------------------------------------------------------------------------
// Coarse top-K: threshold from the vote histogram, then an order-preserving compaction.
// Keeps every cell with votes above the threshold and the lowest-key cells at it, so the
// kept set is the K best by (votes desc, key asc).
// ---------------------------------------------------------------------------------------
__global__ void __launch_bounds__(1024)
k_select_coarse(DevGeom g, int ev0, const int32_t *votes, const uint32_t *hist, int K,
                uint64_t *out_keys, int32_t *out_votes) {
    __shared__ int s_vstar, s_need;
    __shared__ int sa[1024], sb[1024];
    const int e = blockIdx.x, ev = ev0 + e, tid = threadIdx.x;
    const int Bd = g.bins[0], Bp = g.bins[1], Bw = g.bins[2], Bz = g.bins[3];
    const long long n = (long long)Bd * Bp * Bw * Bz * g.bins[4];
    if (tid == 0) {
        long long cum = 0;
        int vstar = -1, need = 0;
        for (int v = kHistBins - 1; v >= 0; v--) {
            long long h = hist[(long long)e * kHistBins + v];
            if (cum + h >= K) { vstar = v; need = (int)(K - cum); break; }
            cum += h;
        }
        s_vstar = vstar;
        s_need = need;
    }
    __syncthreads();
    const int vstar = s_vstar, need = s_need;
    const int32_t *vo = votes + (long long)e * n;
    long long chunk = (n + 1023) / 1024;
    long long beg = tid * chunk, end = beg + chunk < n ? beg + chunk : n;
    int a = 0, b = 0;
    for (long long j = beg; j < end; j++) {
        int v = vo[j];
        a += v > vstar;
        b += v == vstar;
    }
    sa[tid] = a;
    sb[tid] = b;
    __syncthreads();
    // inclusive Hillis-Steele scans
    for (int off = 1; off < 1024; off <<= 1) {
        int xa = tid >= off ? sa[tid - off] : 0, xb = tid >= off ? sb[tid - off] : 0;
        __syncthreads();
        sa[tid] += xa;
        sb[tid] += xb;
        __syncthreads();
    }
    const int totalA = sa[1023];
    int pa = sa[tid] - a, pb = sb[tid] - b;
    uint64_t *ok_ = out_keys + (long long)ev * K;
    int32_t *ov = out_votes + (long long)ev * K;
    for (long long j = beg; j < end; j++) {
        int v = vo[j];
        if (v > vstar || (v == vstar && pb < need)) {
            long long r = j;
            int idx[5];
            for (int q = 0; q < 5; q++) { idx[q] = (int)(r % g.bins[q]); r /= g.bins[q]; }
            int pos = v > vstar ? pa++ : totalA + pb++;
            ok_[pos] = pack_key(idx);
            ov[pos] = v;
        } else if (v == vstar) {
            pb++;
        }
    }
}

void launch_select_coarse(const DevGeom &g, int ev0, int n_ev, const int32_t *votes,
                          const uint32_t *hist, int K, uint64_t *out_keys, int32_t *out_votes,
                          cudaStream_t s) {
    if (n_ev <= 0) return;
    k_select_coarse<<<n_ev, 1024, 0, s>>>(g, ev0, votes, hist, K, out_keys, out_votes);
}

// ---------------------------------------------------------------------------------------
// Per-event bitonic sort of (votes desc, key asc) packed as ((1023 - v) << 50) | key.
// ---------------------------------------------------------------------------------------
constexpr int kSortMax = 4096;
__device__ void block_sort(uint64_t *s, int n_pow2) {
    for (int size = 2; size <= n_pow2; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int i = threadIdx.x; i < n_pow2 / 2; i += blockDim.x) {
                int lo = 2 * i - (i & (stride - 1));
                int hi = lo + stride;
                bool up = ((lo & size) == 0);
                uint64_t x = s[lo], y = s[hi];
                if ((x > y) == up) { s[lo] = y; s[hi] = x; }
            }
            __syncthreads();
        }
    }
}
__device__ __forceinline__ int pow2_ge(int n) {
    int p = 1;
    while (p < n) p <<= 1;
    return p;
}
constexpr uint64_t kKeyMask = (1ULL << 50) - 1;

__device__ void load_sorted(uint64_t *s, const uint64_t *keys, const int32_t *votes, int n, int np2) {
    for (int i = threadIdx.x; i < np2; i += blockDim.x)
        s[i] = i < n ? (((uint64_t)(1023 - votes[i]) << 50) | (keys[i] & kKeyMask)) : ~0ULL;
    __syncthreads();
    block_sort(s, np2);
}

__global__ void __launch_bounds__(1024)
k_topk(const uint64_t *keys, const int32_t *votes, int n_in, int K, uint64_t *out_keys,
       int32_t *out_votes) {
    __shared__ uint64_t s[kSortMax];
    const int e = blockIdx.x;
    int np2 = pow2_ge(n_in);
    load_sorted(s, keys + (long long)e * n_in, votes + (long long)e * n_in, n_in, np2);
    for (int i = threadIdx.x; i < K; i += blockDim.x) {
        uint64_t x = i < n_in ? s[i] : ~0ULL;
        out_keys[(long long)e * K + i] = x & kKeyMask;
        out_votes[(long long)e * K + i] = i < n_in ? 1023 - (int)(x >> 50) : 0;
    }
}

void launch_topk(int n_ev, const uint64_t *keys, const int32_t *votes, int n_in, int K,
                 uint64_t *out_keys, int32_t *out_votes, cudaStream_t s) {
    if (n_ev <= 0) return;
    k_topk<<<n_ev, 1024, 0, s>>>(keys, votes, n_in, K, out_keys, out_votes);
}

// ---------------------------------------------------------------------------------------
// Final estimate (Section 3.3): over the maximum-vote cells in ascending key order, the
// mean of the cell centres and the half-extent of their union per axis, in
// round-to-nearest; written into apo_track records (stride tracks per event).
// ---------------------------------------------------------------------------------------
__global__ void __launch_bounds__(1024)
k_estimate(DevGeom g, const uint64_t *keys, const int32_t *votes, int n_in, int level,
           const int32_t *n_hits, apo_track *out, int stride, int32_t *n_tracks) {
    __shared__ uint64_t s[kSortMax];
    const int e = blockIdx.x;
    int np2 = pow2_ge(n_in);
    load_sorted(s, keys + (long long)e * n_in, votes + (long long)e * n_in, n_in, np2);
    if (threadIdx.x != 0) return;
    apo_track &t = out[(long long)e * stride];
    int nh = n_hits[e];
    if (nh < 0) {
        for (int a = 0; a < 5; a++) { t.p[a] = 0.0; t.w[a] = 0.0; }
        t.votes = nh;
        t.n_hits = 0;
        if (n_tracks) n_tracks[e] = 0;
        return;
    }
    int vmax = 1023 - (int)(s[0] >> 50);
    int m = 0;
    while (m < n_in && 1023 - (int)(s[m] >> 50) == vmax) m++;
    for (int a = 0; a < 5; a++) {
        double sum = 0.0, lo_min = 1e300, hi_max = -1e300;
        for (int j = 0; j < m; j++) {
            int idx[5];
            unpack_key(s[j] & kKeyMask, idx);
            IV<double> ed = edge(g, a, level, idx[a]);
            sum = __dadd_rn(sum, __dmul_rn(__dadd_rn(ed.lo, ed.hi), 0.5));
            lo_min = ed.lo < lo_min ? ed.lo : lo_min;
            hi_max = ed.hi > hi_max ? ed.hi : hi_max;
        }
        t.p[a] = __ddiv_rn(sum, (double)m);
        t.w[a] = __dmul_rn(__dsub_rn(hi_max, lo_min), 0.5);
    }
    t.votes = vmax;
    t.n_hits = nh;
    if (n_tracks) n_tracks[e] = 1;
}

void launch_estimate_tracks(const DevGeom &g, int n_ev, const uint64_t *keys, const int32_t *votes,
                            int n_in, int level, const int32_t *n_hits, apo_track *out, int stride,
                            int32_t *n_tracks, cudaStream_t s) {
    if (n_ev <= 0) return;
    k_estimate<<<n_ev, 1024, 0, s>>>(g, keys, votes, n_in, level, n_hits, out, stride, n_tracks);
}

}  // namespace apo

namespace apo {

// ---------------------------------------------------------------------------------------
// Histogram of level-0 votes (for apo_refine on caller-provided coarse votes).
// ---------------------------------------------------------------------------------------
__global__ void k_hist(const int32_t *votes, long long n, uint32_t *hist) {
    __shared__ uint32_t hs[kHistBins];
    const int e = blockIdx.y;
    for (int i = threadIdx.x; i < kHistBins; i += blockDim.x) hs[i] = 0;
    __syncthreads();
    const int32_t *v = votes + (long long)e * n;
    for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < n;
         j += (long long)gridDim.x * blockDim.x) {
        int x = v[j];
        x = x < 0 ? 0 : (x > kHitCap ? kHitCap : x);
        atomicAdd(&hs[x], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kHistBins; i += blockDim.x)
        if (hs[i]) atomicAdd(&hist[(long long)e * kHistBins + i], hs[i]);
}

void launch_hist(int n_ev, const int32_t *votes, long long n, uint32_t *hist, cudaStream_t s) {
    if (n_ev <= 0) return;
    dim3 grid(64, n_ev);
    k_hist<<<grid, 256, 0, s>>>(votes, n, hist);
}

// 32 children of each key (level + 1)
__global__ void k_children(const uint64_t *keys, long long n, uint64_t *out) {
    long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n * 32) return;
    int idx[5], b = (int)(j % 32);
    unpack_key(keys[j / 32], idx);
#pragma unroll
    for (int a = 0; a < 5; a++) idx[a] = 2 * idx[a] + ((b >> a) & 1);
    out[j] = pack_key(idx);
}

void launch_children(const uint64_t *keys, long long n, uint64_t *out, cudaStream_t s) {
    if (n <= 0) return;
    k_children<<<(unsigned)((n * 32 + 255) / 256), 256, 0, s>>>(keys, n, out);
}

}  // namespace apo
