// sm_103a kernels of the interval-voting hot path (arXiv:2401.04576, Section 3.1):
// hit staging, coarse-grid voting, voting of explicit / bisected cells, top-K selection and
// the final max-vote estimate.
#include <cuda_runtime.h>

#include <climits>
#include <cstdint>

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
__device__ __forceinline__ void mbar_inval(uint64_t *bar) {
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(bar)) : "memory");
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

// Waits for phase `parity` of an mbarrier for at most `limit` polls.  On running out it sets
// ST_TIMEOUT in *status (if given) and returns false; the caller then leaves the barrier's
// work undone and the kernel ends normally, so the context stays usable.
__device__ bool bounded_wait(uint64_t *bar, unsigned parity, long limit, unsigned *status) {
    for (long it = 0; it < limit; it++)
        if (mbar_try_wait(bar, parity)) return true;
    if (status) atomicOr(status, ST_TIMEOUT);
    return false;
}

// Copies up to two blocks (bytes0 / bytes1: multiples of 16, 16-byte aligned ends) of an
// event's hit records into shared memory with one mbarrier.  Returns false (and flags
// ST_TIMEOUT) if the copies did not complete within the wait limit; the caller then skips
// the block's work.
__device__ bool stage_to_smem(void *dst0, const void *src0, unsigned bytes0, void *dst1,
                              const void *src1, unsigned bytes1, uint64_t *bar, unsigned *status) {
    if (threadIdx.x == 0) {
        mbar_init(bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();
    if (bytes0 + bytes1 == 0) return true;
    if (threadIdx.x == 0) {
        mbar_expect_tx(bar, bytes0 + bytes1);
        if (bytes0) bulk_g2s(dst0, src0, bytes0, bar);
        if (bytes1) bulk_g2s(dst1, src1, bytes1, bar);
    }
    if (bounded_wait(bar, 0, kWaitLimit, status)) return true;
    // give the copies in flight a second bounded chance before leaving the shared memory
    bounded_wait(bar, 0, kWaitLimit, nullptr);
    return false;
}

// Diagnostic: every thread waits on an mbarrier whose expected bytes never arrive (no copy
// is issued, so nothing is in flight), with a short limit.  The wait must run out and
// report ST_TIMEOUT; used to test the timeout path without any device fault.
__global__ void k_wait_never(long limit, unsigned *status) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        mbar_expect_tx(&bar, 16);
    }
    __syncthreads();
    bounded_wait(&bar, 0, limit, status);
}

void launch_wait_never(long limit, unsigned *status, cudaStream_t s) {
    k_wait_never<<<1, 32, 0, s>>>(limit, status);
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
                        uint32_t *active, int32_t *done, unsigned *status, int32_t *hit_track) {
    int e = blockIdx.x;
    if (e >= n_events) return;
    __shared__ int bad;
    if (threadIdx.x == 0) bad = 0;
    __syncthreads();
    int a = offsets[e], b = offsets[e + 1];
    int n = b - a;
    if (n < 0 || a < 0 || n > kHitCap) {
        if (threadIdx.x < 8) active[(long long)e * 8 + threadIdx.x] = 0u;
        if (threadIdx.x == 0) {
            n_hits[e] = APO_EINVAL;
            done[e] = 0;
            atomicOr(status, n > kHitCap ? ST_TOOMANY : ST_BADOFFS);
        }
        return;
    }
    if (hit_track)
        for (int i = threadIdx.x; i < n; i += blockDim.x) hit_track[a + i] = -1;
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
    if (threadIdx.x < 8) {   // every valid hit starts active
        int lo = 32 * threadIdx.x;
        uint32_t m = bad ? 0u : (n >= lo + 32 ? 0xffffffffu : (n > lo ? (1u << (n - lo)) - 1u : 0u));
        active[(long long)e * 8 + threadIdx.x] = m;
    }
    if (threadIdx.x == 0) {
        done[e] = 0;
        if (bad) { n_hits[e] = APO_EINVAL; atomicOr(status, ST_BADHIT); }
        else n_hits[e] = n;
    }
}

void launch_stage(const DevGeom &g, int n_events, const int32_t *offsets, const int32_t *wire_id,
                  const double *drift, HitRecD *hd, HitRecF *hf, int32_t *n_hits, uint32_t *active,
                  int32_t *done, unsigned *status, cudaStream_t s, int32_t *hit_track) {
    if (n_events <= 0) return;
    k_stage<<<n_events, 128, 0, s>>>(g, n_events, offsets, wire_id, drift, hd, hf, n_hits, active,
                                      done, status, hit_track);
}

// ---------------------------------------------------------------------------------------
// Coarse-grid voting.  Block = (event, phi0 bin p, omega bin w); thread = (d0 bin, z0 bin);
// each thread loops over the tan(lambda) bins, reusing the tan(lambda)-free prefix of the
// program.  Before that, every hit is tested once on the block's parent cell (all d0, z0,
// tan(lambda) bins joined): interval operations are inclusion-isotonic and the guards only
// fire on a parent when they fire on a child, so a hit that fails there fails on every
// child cell; skipping it leaves every vote unchanged.
// Modes: FP32 intervals; FP64 intervals; FP64 intervals evaluated only where the FP32
// program votes (FP32 intervals contain the FP64 ones, so an FP32 "no" is an FP64 "no":
// the votes are those of the plain FP64 program).
// Writes votes[e][lin], lin = d + Bd (p + Bp (w + Bw (z + Bz l))), and the per-event
// histogram of vote counts.
// ---------------------------------------------------------------------------------------
enum : int { kModeF32 = 0, kModeF64 = 1, kModeF64Filtered = 2, kModeF64Exact = 3 };
// precisions a mode evaluates: FP64 intervals (all but FP32), FP32 intervals (FP32 and the
// FP32-first filter); kModeF64Exact uses the exact-phase program for its FP64 steps
template <int MODE> struct ModeOf {
    static constexpr bool k64 = MODE != kModeF32;
    static constexpr bool k32 = MODE == kModeF32 || MODE == kModeF64Filtered;
    static constexpr bool exact = MODE == kModeF64Exact;
};

template <int MODE> struct CoarseSmem {
    static constexpr bool k64 = ModeOf<MODE>::k64, k32 = ModeOf<MODE>::k32;
    static constexpr size_t hits64 = 0;
    static constexpr size_t hits32 = k64 ? kHitCap * 80 : 0;
    static constexpr size_t hist = hits32 + (k32 ? kHitCap * 80 : 0);
    static constexpr size_t mask = hist + kHistBins * 4 + 12;
    static constexpr size_t bar = mask + 32;
    static constexpr size_t L64 = bar + 8;
    __host__ __device__ static size_t L32(int Bl) { return L64 + 16 * Bl; }
    __host__ __device__ static size_t total(int Bl, int) { return L32(Bl) + 8 * Bl + 16; }
};

// The FP32 coarse kernel splits each tile's (d0, z0) cells over APO_F32_COARSE_SPLIT
// blocks, and asks the compiler for APO_F32_COARSE_MIN_BLOCKS resident blocks per SM (it
// caps registers at 64K / (threads x this)); the FP64 kernels are bound by the FP64 pipe.
#ifndef APO_F32_COARSE_SPLIT
#define APO_F32_COARSE_SPLIT 1
#endif
#ifndef APO_F32_COARSE_MIN_BLOCKS
#define APO_F32_COARSE_MIN_BLOCKS (3 * APO_F32_COARSE_SPLIT)
#endif
// The FP64 modes split each (phi0, omega) tile's (d0, z0) cells over APO_F64_COARSE_SPLIT
// blocks (consecutive ranges of the d0-fastest index): smaller blocks with the same register
// budget let more warps share an SM, which hides more FP64 latency.
#ifndef APO_F64_COARSE_SPLIT
#define APO_F64_COARSE_SPLIT 2
#endif
#ifndef APO_F64_COARSE_MIN_BLOCKS
#define APO_F64_COARSE_MIN_BLOCKS (APO_F64_COARSE_SPLIT == 1 ? 1 : 3)
#endif
template <int MODE> struct CoarseShape {
    static constexpr int split = MODE == kModeF32 ? APO_F32_COARSE_SPLIT : APO_F64_COARSE_SPLIT;
    static constexpr int threads = 256 / split;
    static constexpr int min_blocks = MODE == kModeF32 ? APO_F32_COARSE_MIN_BLOCKS : APO_F64_COARSE_MIN_BLOCKS;
};

// One block's work: part `part` (of `split`) of the (phi0 bin p, omega bin w) tile of event
// ev; votes to vo (the event's level-0 votes), the histogram added to hist_e.  Shared by
// k_vote_coarse (one tile per block) and the persistent batch kernel (tiles in a loop);
// any block size of at least one warp works (threads past the part's cells idle).
template <int MODE>
__device__ __forceinline__ void coarse_block(const DevGeom &g, int ev, int split, int part, int p, int w,
                                             const HitRecD *hd, const HitRecF *hf, const int32_t *n_hits,
                                             const uint32_t *active, int32_t *vo, uint32_t *hist_e,
                                             unsigned *status, unsigned long long *ctr, unsigned char *smem,
                                             uint64_t *cand_k = nullptr, int32_t *cand_v = nullptr, int K = 0) {
    using S = CoarseSmem<MODE>;
    constexpr bool k64 = S::k64, k32 = S::k32;
    const int Bd = g.bins[0], Bz = g.bins[3], Bl = g.bins[4];
    const int ntile = Bd * Bz;                    // (d0, z0) cells of one (phi0, omega) tile
    const int per = (ntile + split - 1) / split;  // of them in this block
    const int nthr = blockDim.x;
    const int tid = threadIdx.x;
    const int c0 = part * per, c1 = c0 + per < ntile ? c0 + per : ntile;   // this block's cells
    const bool has_cell = c0 + tid < c1;
    unsigned char *h64s = smem + S::hits64;
    unsigned char *h32s = smem + S::hits32;
    uint32_t *hist_s = reinterpret_cast<uint32_t *>(smem + S::hist);
    uint32_t *mask_s = reinterpret_cast<uint32_t *>(smem + S::mask);
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + S::bar);
    IV<double> *L64 = reinterpret_cast<IV<double> *>(smem + S::L64);
    IV<float> *L32 = reinterpret_cast<IV<float> *>(smem + S::L32(Bl));

    int nh = n_hits[ev];
    if (nh < 0) nh = 0;
    for (int i = tid; i < kHistBins; i += nthr) hist_s[i] = 0;
    if (tid < 8) mask_s[tid] = 0;
    for (int l = tid; l < Bl; l += nthr) {
        IV<double> el = edge(g, 4, 0, l);
        L64[l] = el;
        L32[l] = to_prec<float>(el);
    }
    const unsigned bytes = (unsigned)nh * 80u;
    bool ok = stage_to_smem(h64s, hd + (long long)ev * kHitCap, k64 ? bytes : 0u, h32s,
                            hf + (long long)ev * kHitCap, k32 ? bytes : 0u, bar, status);
    __syncthreads();
    if (tid == 0) mbar_inval(bar);   // the barrier's memory may be set up again by a later call
    if (!ok) nh = 0;

    const SeriesConsts &k = g.k;
    const IV<double> S0 = sin_phi0(g, 0, p), C0 = cos_phi0(g, 0, p), W = edge(g, 2, 0, w);
    unsigned n_par32 = 0, n_pre32 = 0, n_tail32 = 0, n_par64 = 0, n_pre64 = 0, n_tail64 = 0;
    // parent cell test, one hit per thread
    {
        IV<double> D0 = edge(g, 0, 0, c1 - c0 >= Bd ? 0 : c0 % Bd);
        IV<double> D1 = edge(g, 0, 0, c1 - c0 >= Bd ? Bd - 1 : (c1 - 1) % Bd);
        if (c0 / Bd != (c1 - 1) / Bd) { D0 = edge(g, 0, 0, 0); D1 = edge(g, 0, 0, Bd - 1); }
        IV<double> Z0 = edge(g, 3, 0, c0 / Bd), Z1 = edge(g, 3, 0, (c1 - 1) / Bd);
        IV<double> L0 = edge(g, 4, 0, 0), L1 = edge(g, 4, 0, Bl - 1);
        Cell<double> par{{D0.lo, D1.hi}, S0, C0, W, {Z0.lo, Z1.hi}, {L0.lo, L1.hi}};
        Cell<float> par32{to_prec<float>(par.D), to_prec<float>(S0), to_prec<float>(C0),
                          to_prec<float>(W), to_prec<float>(par.Z), to_prec<float>(par.L)};
        const uint32_t *act = active ? active + (long long)ev * 8 : nullptr;
        auto parent_vote = [&](int h) -> bool {
            if (h >= nh || (act && !((act[h >> 5] >> (h & 31)) & 1u))) return false;
            bool v = true;
            if (k32) { v = vote_pair<float>(par32, load_hit<float>(h32s + h * 80), k); n_par32++; }
            if (k64 && v) {
                v = ModeOf<MODE>::exact ? vote_pair_exact(par, load_hit<double>(h64s + h * 80), k)
                                        : vote_pair<double>(par, load_hit<double>(h64s + h * 80), k);
                n_par64++;
            }
            return v;
        };
        const int lane = tid & 31, warp = tid >> 5, nfull = nthr >> 5;
        if (nfull > 0) {   // full warps take 32 hits each; the warp ballot is the mask word
            if (warp < nfull)
                for (int base = warp * 32; base < nh; base += nfull * 32) {
                    unsigned m = __ballot_sync(0xffffffffu, parent_vote(base + lane));
                    if (lane == 0) mask_s[base >> 5] = m;
                }
        } else {
            for (int h = tid; h < nh; h += nthr)
                if (parent_vote(h)) atomicOr(&mask_s[h >> 5], 1u << (h & 31));
        }
    }
    __syncthreads();

    const int cell = has_cell ? c0 + tid : c0;   // threads past the block's cells idle
    const int d = cell % Bd, z = cell / Bd;
    Cell<double> c{edge(g, 0, 0, d), S0, C0, W, edge(g, 3, 0, z), L64[0]};
    Cell<float> c32{to_prec<float>(c.D), to_prec<float>(S0), to_prec<float>(C0), to_prec<float>(W),
                    to_prec<float>(c.Z), L32[0]};
    const bool mir = mirror_cell(c);
    mirror_cell(c32);
    const bool wguard = !gt0(c.W.lo) || !gt0(c32.W.lo);
    const IV<double> R = recip(c.W);
    const IV<float> R32 = recip(c32.W);
    const unsigned all = Bl >= 32 ? 0xffffffffu : ((1u << Bl) - 1u);
    // The Bl vote counters of this thread, bit-sliced: bit l of plane k is bit k of counter
    // l (counts <= 256 need 9 planes).  Adding a mask of votes is a ripple-carry add.
    uint32_t pl[9];
#pragma unroll
    for (int q = 0; q < 9; q++) pl[q] = 0u;
    auto add_votes = [&](uint32_t m) {
#pragma unroll
        for (int q = 0; q < 9; q++) {
            const uint32_t c = pl[q] & m;
            pl[q] ^= m;
            m = c;
        }
    };
    for (int wd = 0; wd < 8 && has_cell; wd++) {
        uint32_t m = mask_s[wd];
        while (m) {
            int h = wd * 32 + __ffs(m) - 1;
            m &= m - 1;
            if (wguard) {
                add_votes(all);
                continue;
            }
            // tan(lambda) bins still in question after the FP32 program
            unsigned lm = all;
            if (k32) {
                Hit<float> h32 = load_hit<float>(h32s + h * 80);
                if (mir) mirror_hit(h32);
                Pre<float> p32 = prefix<float>(c32, h32, k);
                n_pre32++;
                if (p32.novote) {
                    lm = 0;
                } else if (!p32.guard) {
                    lm = 0;
                    n_tail32 += Bl;
                    // sign of the wire's stereo tangent (0: unknown)
                    const int tsg = h32.t.lo >= 0.f ? 1 : (h32.t.hi <= 0.f ? -1 : 0);
#pragma unroll 1
                    for (int l = 0; l < Bl; l++) {
                        const IV<float> Ll = L32[l];
                        bool tv;
                        if (MODE == kModeF32) {
                            // The block's threads share the bin and the hit: uniform branches
                            // on the signs of L and t.  A bin with L <= 0 is evaluated
                            // reflected, (L, t) -> (-L, -t), which gives the same vote, so the
                            // tail always sees L >= 0 and a known sign of t.  (In the filtered
                            // FP64 mode the extra FP32 tails cost more code than they save.)
                            const bool lpos = Ll.lo >= 0.f, lneg = Ll.hi <= 0.f;
                            const int ts = lpos ? tsg : (lneg ? -tsg : 0);
                            Hit<float> hr = h32;
                            if (!lpos) hr.t = neg(h32.t);
                            const IV<float> Lr = lpos ? Ll : neg(Ll);
                            tv = ts > 0 ? tail<float, 1, false, 1>(p32, Lr, hr, R32, c32.W, k)
                               : ts < 0 ? tail<float, 1, false, -1>(p32, Lr, hr, R32, c32.W, k)
                                        : tail<float, 0>(p32, Ll, h32, R32, c32.W, k);
                        } else {
                            tv = tail<float>(p32, Ll, h32, R32, c32.W, k);
                        }
                        if (tv) lm |= 1u << l;
                    }
                }
                if (!k64) {
                    add_votes(lm);
                    continue;
                }
            }
            if (!lm) continue;
            Hit<double> h64 = load_hit<double>(h64s + h * 80);
            if (mir) mirror_hit(h64);
            Pre<double> p64 = prefix<double>(c, h64, k);
            n_pre64++;
            if (p64.novote) continue;
            if (p64.guard) {
                add_votes(all);
                continue;
            }
            uint32_t v64 = 0;
            while (lm) {
                int l = __ffs(lm) - 1;
                lm &= lm - 1;
                n_tail64++;
                const bool tv = ModeOf<MODE>::exact ? tail_exact(p64, L64[l], h64, R, c.W, k)
                                                    : tail<double>(p64, L64[l], h64, R, c.W, k);
                if (tv) v64 |= 1u << l;
            }
            add_votes(v64);
        }
    }
    const int Bp = g.bins[1], Bw = g.bins[2];
    auto vote_of = [&](int l) {
        int v = 0;
#pragma unroll
        for (int q = 0; q < 9; q++) v |= (int)((pl[q] >> l) & 1u) << q;
        return v;
    };
    for (int l = 0; l < Bl && has_cell; l++) {
        const int v = vote_of(l);
        if (!cand_k) {
            long long lin = d + (long long)Bd * (p + (long long)Bp * (w + (long long)Bw * (z + (long long)Bz * l)));
            vo[lin] = v;
        }
        atomicAdd(&hist_s[v], 1u);
    }
    __syncthreads();
    for (int i = tid; i < kHistBins; i += nthr)
        if (hist_s[i]) atomicAdd(&hist_e[i], hist_s[i]);
    if (cand_k) {
        // The part's K best cells by (votes desc, key asc), from its own histogram: every
        // cell above v_t, then the lowest keys at v_t.  Within a part, cells in the order
        // (tan(lambda) bin, thread) are in key order.  Any cell among the event's K best is
        // among its part's K best, so these candidates are all the selection needs.
        __shared__ int s_vt, s_need, s_above;
        // warp 0 (its cw lanes: a block may have fewer than 32 threads): suffix sums of the
        // histogram from the top, cw bins a step
        const int cw = nthr < 32 ? nthr : 32;
        if (tid < cw) {
            const unsigned m0 = cw == 32 ? 0xffffffffu : ((1u << cw) - 1u);
            int cum = 0;
            bool found = false;
            for (int top = kHistBins - 1; top >= 0 && !found; top -= cw) {
                const int v = top - tid;
                const int h = v >= 0 ? (int)hist_s[v] : 0;
                int inc = h;   // cells with votes in [v, top]
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int y = __shfl_up_sync(m0, inc, o);
                    if (tid >= o) inc += y;
                }
                const unsigned hit = __ballot_sync(m0, v >= 0 && cum + inc >= K);
                if (hit) {   // the first bin from the top where the count reaches K
                    const int b = __ffs(hit) - 1;
                    const int incb = __shfl_sync(m0, inc, b), hb = __shfl_sync(m0, h, b);
                    if (tid == 0) {
                        s_vt = top - b;
                        s_above = cum + incb - hb;
                        s_need = K - (cum + incb - hb);
                    }
                    found = true;
                } else {
                    cum += __shfl_sync(m0, inc, cw - 1);
                }
            }
            if (!found && tid == 0) {   // fewer than K cells in the part
                s_vt = -1;
                s_above = cum;
                s_need = 0;
            }
        }
        __syncthreads();
        const int vt = s_vt, need = s_need, above = s_above;
        const int lane = tid & 31, wid = tid >> 5, nwarps = (nthr + 31) >> 5;
        // the block may end in a partial warp (e.g. 100 or 50 threads): ballots over the
        // lanes that exist (lanes 0 .. r - 1 of the last warp)
        const int rem = nthr - (wid << 5);
        const unsigned wmask = rem >= 32 ? 0xffffffffu : ((1u << rem) - 1u);
        const unsigned lt = (1u << lane) - 1u;
        // Ranks in key order ((tan(lambda) bin, thread) order): per bin and warp, counts of
        // cells above v_t / at v_t from ballots; exclusive prefixes over warps, then over
        // bins; a cell's rank is its bin's base + its warp's prefix + its lane's prefix.
        __shared__ int s_wa[8][32], s_wb[8][32], s_ba[33], s_bb[33];
        for (int l = 0; l < Bl; l++) {
            const int v = has_cell ? vote_of(l) : -1;
            const unsigned ma = __ballot_sync(wmask, v > vt), mb = __ballot_sync(wmask, v == vt);
            if (lane == 0) { s_wa[wid][l] = __popc(ma); s_wb[wid][l] = __popc(mb); }
        }
        __syncthreads();
        if (tid < Bl) {   // exclusive prefix over warps, bin by bin
            int ra = 0, rb = 0;
            for (int q = 0; q < nwarps; q++) {
                const int xa = s_wa[q][tid], xb = s_wb[q][tid];
                s_wa[q][tid] = ra;
                s_wb[q][tid] = rb;
                ra += xa;
                rb += xb;
            }
            s_ba[tid] = ra;   // the bin's totals, turned into bases below
            s_bb[tid] = rb;
        }
        __syncthreads();
        if (tid == 0) {   // exclusive prefix over bins
            int ra = 0, rb = 0;
            for (int l = 0; l < Bl; l++) {
                const int xa = s_ba[l], xb = s_bb[l];
                s_ba[l] = ra;
                s_bb[l] = rb;
                ra += xa;
                rb += xb;
            }
            s_ba[Bl] = ra;
            s_bb[Bl] = rb;
        }
        __syncthreads();
        for (int l = 0; l < Bl; l++) {
            const int v = has_cell ? vote_of(l) : -1;
            const bool a = v > vt, b = v == vt;
            const unsigned ma = __ballot_sync(wmask, a), mb = __ballot_sync(wmask, b);
            int pos = -1;
            if (a) {
                pos = s_ba[l] + s_wa[wid][l] + __popc(ma & lt);
            } else if (b) {
                const int rb = s_bb[l] + s_wb[wid][l] + __popc(mb & lt);
                if (rb < need) pos = above + rb;
            }
            if (pos >= 0 && pos < K) {   // always below K when the counts agree; never past it
                int idx[5] = {d, p, w, z, l};
                cand_k[pos] = pack_key(g, idx);
                cand_v[pos] = v;
            }
        }
        const int runB = s_bb[Bl];
        const int placed = above + (runB < need ? runB : need);
        for (int i = placed + tid; i < K; i += nthr) {   // a part with fewer than K cells
            cand_k[i] = 0;
            cand_v[i] = -1;
        }
    }
    if (ctr) {   // work counters (diagnostics): FP64 parent / prefix / tail, -, FP32 ones
        unsigned long long v[6] = {n_par64, n_pre64, n_tail64, n_par32, n_pre32, n_tail32};
        const int slot[6] = {0, 1, 2, 4, 5, 6};
#pragma unroll
        for (int i = 0; i < 6; i++) {
            unsigned long long x = v[i];
            if (nthr - (tid & ~31) >= 32) {   // a full warp: reduce, one add per warp
                for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
                if ((tid & 31) == 0 && x) atomicAdd(&ctr[slot[i]], x);
            } else if (x) {                   // the lanes of a partial last warp add their own
                atomicAdd(&ctr[slot[i]], x);
            }
        }
    }
    __syncthreads();   // shared memory is reused by the caller's next step
}

template <int MODE>
__global__ void __launch_bounds__(CoarseShape<MODE>::threads, CoarseShape<MODE>::min_blocks)
k_vote_coarse(DevGeom g, int ev0, const HitRecD *hd, const HitRecF *hf, const int32_t *n_hits,
              const uint32_t *active, int32_t *votes, uint32_t *hist, unsigned *status,
              unsigned long long *ctr, uint64_t *cand_k, int32_t *cand_v, int K) {
    extern __shared__ __align__(16) unsigned char smem[];
    constexpr int split = CoarseShape<MODE>::split;
    const int e = blockIdx.y;
    const int part = blockIdx.x % split, pw = blockIdx.x / split;
    const int p = pw % g.bins[1], w = pw / g.bins[1];
    const long long ncell = (long long)g.bins[0] * g.bins[1] * g.bins[2] * g.bins[3] * g.bins[4];
    // candidates: K slots per block, the blocks of an event in blockIdx.x order
    const long long co = ((long long)e * gridDim.x + blockIdx.x) * K;
    coarse_block<MODE>(g, ev0 + e, split, part, p, w, hd, hf, n_hits, active,
                       votes ? votes + (long long)e * ncell : nullptr, hist + (long long)e * kHistBins, status,
                       ctr, smem, cand_k ? cand_k + co : nullptr, cand_v ? cand_v + co : nullptr, K);
}

// ---------------------------------------------------------------------------------------
// Midpoint-form voting (APO_F64_MID, Section 3.1's variant with the quantities of d^Ax at
// the voxel centre).  Coarse grid: the same block / thread layout as k_vote_coarse, the
// tan(lambda)-free part shared by the tan(lambda) bins, bit-sliced counters; there is no
// parent-cell test, because the midpoint form is not inclusion-isotonic (a parent's
// centre says nothing about its children's centres).
// ---------------------------------------------------------------------------------------
struct MidSmem {
    static constexpr size_t hits = 0;
    static constexpr size_t hist = kHitCap * 80;
    static constexpr size_t bar = hist + ((kHistBins * 4 + 15) & ~size_t(15));
    static constexpr size_t Lc = bar + 16;
    __host__ __device__ static size_t total(int Bl) { return Lc + 8 * Bl; }
};

__global__ void __launch_bounds__(256)
k_vote_coarse_mid(DevGeom g, int ev0, const HitRecD *hd, const int32_t *n_hits,
                  const uint32_t *active, int32_t *votes, uint32_t *hist, unsigned *status,
                  unsigned long long *ctr) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int Bd = g.bins[0], Bp = g.bins[1], Bw = g.bins[2], Bz = g.bins[3], Bl = g.bins[4];
    const int nthr = Bd * Bz;
    const int e = blockIdx.y, ev = ev0 + e;
    const int p = blockIdx.x % Bp, w = blockIdx.x / Bp;
    const int tid = threadIdx.x;
    unsigned char *hs = smem + MidSmem::hits;
    uint32_t *hist_s = reinterpret_cast<uint32_t *>(smem + MidSmem::hist);
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + MidSmem::bar);
    double *Lc = reinterpret_cast<double *>(smem + MidSmem::Lc);

    int nh = n_hits[ev];
    if (nh < 0) nh = 0;
    for (int i = tid; i < kHistBins; i += nthr) hist_s[i] = 0;
    for (int l = tid; l < Bl; l += nthr) Lc[l] = pt::centre(edge(g, 4, 0, l));
    bool ok = stage_to_smem(hs, hd + (long long)ev * kHitCap, (unsigned)nh * 80u, nullptr, nullptr, 0u,
                            bar, status);
    __syncthreads();
    if (!ok) nh = 0;

    const int d = tid % Bd, z = tid / Bd;
    Cell<double> c{edge(g, 0, 0, d), sin_phi0(g, 0, p), cos_phi0(g, 0, p), edge(g, 2, 0, w),
                   edge(g, 3, 0, z), {0.0, 0.0}};
    MidCentre m;
    sincos_phi0_centre(g, 0, p, m.S0, m.C0);
    m.D = pt::centre(c.D);
    m.W = pt::centre(c.W);
    m.Z = pt::centre(c.Z);
    const bool mir = mirror_cell(c);
    if (mir) { m.D = -m.D; m.S0 = -m.S0; m.W = -m.W; }
    const bool wguard = le0(c.W.lo);
    const unsigned all = Bl >= 32 ? 0xffffffffu : ((1u << Bl) - 1u);
    const uint32_t *act = active ? active + (long long)ev * 8 : nullptr;
    uint32_t pl[9];
#pragma unroll
    for (int q = 0; q < 9; q++) pl[q] = 0u;
    auto add_votes = [&](uint32_t mk) {
#pragma unroll
        for (int q = 0; q < 9; q++) {
            const uint32_t cy = pl[q] & mk;
            pl[q] ^= mk;
            mk = cy;
        }
    };
    unsigned n_pre = 0, n_tail = 0;
    for (int h = 0; h < nh; h++) {
        if (act && !((act[h >> 5] >> (h & 31)) & 1u)) continue;
        if (wguard) { add_votes(all); continue; }
        Hit<double> hh = load_hit<double>(hs + h * 80);
        if (mir) mirror_hit(hh);
        MidPre pre = mid_prefix(c, m, hh);
        n_pre++;
        if (pre.guard) { add_votes(all); continue; }
        uint32_t v = 0;
#pragma unroll 1
        for (int l = 0; l < Bl; l++)
            if (mid_tail(pre, Lc[l], hh, c.W)) v |= 1u << l;
        n_tail += Bl;
        add_votes(v);
    }
    const long long ncell = (long long)Bd * Bp * Bw * Bz * Bl;
    int32_t *vo = votes + (long long)e * ncell;
    for (int l = 0; l < Bl; l++) {
        int v = 0;
#pragma unroll
        for (int q = 0; q < 9; q++) v |= (int)((pl[q] >> l) & 1u) << q;
        long long lin = d + (long long)Bd * (p + (long long)Bp * (w + (long long)Bw * (z + (long long)Bz * l)));
        vo[lin] = v;
        atomicAdd(&hist_s[v], 1u);
    }
    __syncthreads();
    for (int i = tid; i < kHistBins; i += nthr)
        if (hist_s[i]) atomicAdd(&hist[(long long)e * kHistBins + i], hist_s[i]);
    if (ctr) {   // work counters (diagnostics): midpoint prefixes / tails in the FP64 slots
        unsigned long long v[2] = {n_pre, n_tail};
#pragma unroll
        for (int i = 0; i < 2; i++) {
            unsigned long long x = v[i];
            if ((int)blockDim.x - (tid & ~31) >= 32) {   // a full warp: reduce, one add per warp
                for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
                if ((tid & 31) == 0 && x) atomicAdd(&ctr[1 + i], x);
            } else if (x) {                               // a partial last warp
                atomicAdd(&ctr[1 + i], x);
            }
        }
    }
}

// Midpoint form on explicit cells: given keys, or the 32 children of each parent key (in
// the order of k_vote_cells).  One cell per thread, all hits of its event.
__global__ void __launch_bounds__(256)
k_vote_cells_mid(DevGeom g, const HitRecD *hd, const int32_t *n_hits, const uint32_t *active, int level,
                 const uint64_t *keys, const uint64_t *parents, long long n_per_ev, uint64_t *out_keys,
                 int32_t *out_votes, unsigned *status) {
    extern __shared__ __align__(16) unsigned char smem[];
    unsigned char *hs = smem;
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + kHitCap * 80);
    const int ev = blockIdx.y;
    int nh = n_hits[ev];
    if (nh < 0) nh = 0;
    bool ok = stage_to_smem(hs, hd + (long long)ev * kHitCap, (unsigned)nh * 80u, nullptr, nullptr, 0u,
                            bar, status);
    __syncthreads();
    if (!ok) nh = 0;
    const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n_per_ev) return;
    uint64_t key;
    if (parents) {
        uint64_t pk = parents[(long long)ev * (n_per_ev / 32) + j / 32];
        int idx[5], b = (int)(j % 32);
        unpack_key(g, pk, idx);
#pragma unroll
        for (int a = 0; a < 5; a++) idx[a] = 2 * idx[a] + ((b >> a) & 1);
        key = pack_key(g, idx);
    } else {
        key = keys[(long long)ev * n_per_ev + j];
    }
    int idx[5];
    unpack_key(g, key, idx);
    const long long o = (long long)ev * n_per_ev + j;
    bool valid = true;
#pragma unroll
    for (int a = 0; a < 5; a++) valid = valid && idx[a] < (g.bins[a] << level);
    if (!valid) {   // a key outside the grid of this level: no lookup, vote count -1
        out_votes[o] = -1;
        if (out_keys) out_keys[o] = key;
        return;
    }
    const IV<double> Le = edge(g, 4, level, idx[4]);
    const Cell<double> c{edge(g, 0, level, idx[0]), sin_phi0(g, level, idx[1]), cos_phi0(g, level, idx[1]),
                         edge(g, 2, level, idx[2]), edge(g, 3, level, idx[3]), Le};
    MidCentre m;
    sincos_phi0_centre(g, level, idx[1], m.S0, m.C0);
    m.D = pt::centre(c.D);
    m.W = pt::centre(c.W);
    m.Z = pt::centre(c.Z);
    const double Lm = pt::centre(Le);
    const uint32_t *act = active ? active + (long long)ev * 8 : nullptr;
    int v = 0;
    for (int h = 0; h < nh; h++) {
        if (act && !((act[h >> 5] >> (h & 31)) & 1u)) continue;
        v += mid_vote_pair(c, m, Lm, load_hit<double>(hs + h * 80)) ? 1 : 0;
    }
    out_votes[o] = v;
    if (out_keys) out_keys[o] = key;
}

static void launch_coarse_mid(const DevGeom &g, int ev0, int n_ev, const HitRecD *hd, const int32_t *n_hits,
                              const uint32_t *active, int32_t *votes, uint32_t *hist, unsigned *status,
                              cudaStream_t s, unsigned long long *ctr) {
    dim3 grid(g.bins[1] * g.bins[2], n_ev);
    k_vote_coarse_mid<<<grid, g.bins[0] * g.bins[3], MidSmem::total(g.bins[4]), s>>>(
        g, ev0, hd, n_hits, active, votes, hist, status, ctr);
}

static void launch_cells_mid(const DevGeom &g, int n_ev, const HitRecD *hd, const int32_t *n_hits,
                             const uint32_t *active, int level, const uint64_t *keys,
                             const uint64_t *parents, long long n_per_ev, uint64_t *out_keys,
                             int32_t *out_votes, unsigned *status, cudaStream_t s, int block) {
    dim3 grid((unsigned)((n_per_ev + block - 1) / block), n_ev);
    k_vote_cells_mid<<<grid, block, kHitCap * 80 + 16, s>>>(g, hd, n_hits, active, level, keys, parents,
                                                            n_per_ev, out_keys, out_votes, status);
}

// Raises the dynamic shared-memory limit of a kernel once per process (the attribute is a
// property of the function; setting it outside any stream capture keeps captures clean).
static bool g_attr_coarse[4] = {false, false, false, false}, g_attr_cells[4] = {false, false, false, false},
            g_attr_children[4] = {false, false, false, false};

template <typename K> static void smem_limit_once(K kernel, bool &flag) {
    if (!flag) {
        cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024);
        flag = true;
    }
}

template <int MODE> static void launch_coarse_mode(const DevGeom &g, int ev0, int n_ev, const HitRecD *hd,
                                                  const HitRecF *hf, const int32_t *n_hits,
                                                  const uint32_t *active, int32_t *votes,
                                                  uint32_t *hist, unsigned *status, cudaStream_t s,
                                                  unsigned long long *ctr, uint64_t *cand_k,
                                                  int32_t *cand_v, int K) {
    smem_limit_once(k_vote_coarse<MODE>, g_attr_coarse[MODE]);
    constexpr int split = CoarseShape<MODE>::split;
    dim3 grid(g.bins[1] * g.bins[2] * split, n_ev);
    const int nthr = (g.bins[0] * g.bins[3] + split - 1) / split;
    size_t sm = CoarseSmem<MODE>::total(g.bins[4], nthr);
    k_vote_coarse<MODE><<<grid, nthr, sm, s>>>(g, ev0, hd, hf, n_hits, active, votes, hist, status, ctr,
                                                cand_k, cand_v, K);
}

int coarse_lists(const DevGeom &g, int prec) {
    const int split = (prec == APO_F32 || prec == APO_F64_MID) ? CoarseShape<kModeF32>::split
                                                                : CoarseShape<kModeF64>::split;
    return g.bins[1] * g.bins[2] * split;
}

void launch_vote_coarse(const DevGeom &g, int prec, int ev0, int n_ev, const HitRecD *hd,
                        const HitRecF *hf, const int32_t *n_hits, int32_t *votes, uint32_t *hist,
                        unsigned *status, cudaStream_t s, unsigned long long *ctr,
                        const uint32_t *active, uint64_t *cand_k, int32_t *cand_v, int K) {
    if (n_ev <= 0) return;
    if (prec == APO_F64_MID)
        launch_coarse_mid(g, ev0, n_ev, hd, n_hits, active, votes, hist, status, s, ctr);
    else if (prec == APO_F64_EXACT)
        launch_coarse_mode<kModeF64Exact>(g, ev0, n_ev, hd, hf, n_hits, active, votes, hist, status, s, ctr,
                                              cand_k, cand_v, K);
    else if (prec == APO_F32)
        launch_coarse_mode<kModeF32>(g, ev0, n_ev, hd, hf, n_hits, active, votes, hist, status, s, ctr,
                                              cand_k, cand_v, K);
    else if (prec == APO_F64_FILTERED)
        launch_coarse_mode<kModeF64Filtered>(g, ev0, n_ev, hd, hf, n_hits, active, votes, hist, status, s, ctr,
                                              cand_k, cand_v, K);
    else
        launch_coarse_mode<kModeF64>(g, ev0, n_ev, hd, hf, n_hits, active, votes, hist, status, s, ctr,
                                              cand_k, cand_v, K);
}

// ---------------------------------------------------------------------------------------
// Voting of explicit cells: either given keys (keys != nullptr, n_per_ev per event) or the
// 32 children of each parent key (parents != nullptr).  Thread = one cell, looping over
// all hits of its event; child keys are written out when parents are given.
// ---------------------------------------------------------------------------------------
template <int MODE>
__global__ void __launch_bounds__(256)
k_vote_cells(DevGeom g, const HitRecD *hd, const HitRecF *hf, const int32_t *n_hits,
             const uint32_t *active, int level, const uint64_t *keys, const uint64_t *parents,
             long long n_per_ev, uint64_t *out_keys, int32_t *out_votes, unsigned *status) {
    constexpr bool k64 = ModeOf<MODE>::k64, k32 = ModeOf<MODE>::k32;
    extern __shared__ __align__(16) unsigned char smem[];
    unsigned char *h64s = smem;
    unsigned char *h32s = smem + (k64 ? kHitCap * 80 : 0);
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + (k64 ? kHitCap * 80 : 0) + (k32 ? kHitCap * 80 : 0));
    const int ev = blockIdx.y;
    int nh = n_hits[ev];
    if (nh < 0) nh = 0;
    const unsigned bytes = (unsigned)nh * 80u;
    bool ok = stage_to_smem(h64s, hd + (long long)ev * kHitCap, k64 ? bytes : 0u, h32s,
                            hf + (long long)ev * kHitCap, k32 ? bytes : 0u, bar, status);
    __syncthreads();
    if (!ok) nh = 0;
    long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n_per_ev) return;
    uint64_t key;
    if (parents) {
        uint64_t pk = parents[(long long)ev * (n_per_ev / 32) + j / 32];
        int idx[5], b = (int)(j % 32);
        unpack_key(g, pk, idx);
#pragma unroll
        for (int a = 0; a < 5; a++) idx[a] = 2 * idx[a] + ((b >> a) & 1);
        key = pack_key(g, idx);
    } else if (keys) {
        key = keys[(long long)ev * n_per_ev + j];
    } else {   // the level-0 grid in linear order (d0 fastest)
        int idx[5];
        long long r = j;
#pragma unroll
        for (int a = 0; a < 5; a++) { idx[a] = (int)(r % g.bins[a]); r /= g.bins[a]; }
        key = pack_key(g, idx);
    }
    int idx[5];
    unpack_key(g, key, idx);
    long long o = (long long)ev * n_per_ev + j;
    bool valid = true;
#pragma unroll
    for (int a = 0; a < 5; a++) valid = valid && idx[a] < (g.bins[a] << level);
    if (!valid) {   // a key outside the grid of this level: no lookup, vote count -1
        out_votes[o] = -1;
        if (out_keys) out_keys[o] = key;
        return;
    }
    Cell<double> c{edge(g, 0, level, idx[0]), sin_phi0(g, level, idx[1]), cos_phi0(g, level, idx[1]),
                   edge(g, 2, level, idx[2]), edge(g, 3, level, idx[3]), edge(g, 4, level, idx[4])};
    Cell<float> c32{to_prec<float>(c.D), to_prec<float>(c.S0), to_prec<float>(c.C0),
                    to_prec<float>(c.W), to_prec<float>(c.Z), to_prec<float>(c.L)};
    const SeriesConsts &k = g.k;
    const uint32_t *act = active ? active + (long long)ev * 8 : nullptr;
    int v = 0;
    for (int h = 0; h < nh; h++) {
        if (act && !((act[h >> 5] >> (h & 31)) & 1u)) continue;
        bool vt = true;
        if (k32) vt = vote_pair<float>(c32, load_hit<float>(h32s + h * 80), k);
        if (k64 && vt)
            vt = ModeOf<MODE>::exact ? vote_pair_exact(c, load_hit<double>(h64s + h * 80), k)
                                     : vote_pair<double>(c, load_hit<double>(h64s + h * 80), k);
        v += vt ? 1 : 0;
    }
    out_votes[o] = v;
    if (out_keys) out_keys[o] = key;
}

// Children of kept cells, two per thread: the children 2 idx + bit of a parent that differ
// only in the tan(lambda) bit share every tan(lambda)-free step of the program, so one
// prefix per hit serves both tails (same operations as evaluating them apart).
// One thread's pair j of an event: children 2 idx + bit of parent j / 16 for the bit pattern
// b = j % 16 on d0 .. z0, with tan(lambda) bit 0 and 1 (slots 32 (j / 16) + b and + 16 of the
// event's outputs).  h64s / h32s: the event's hits staged in shared memory; parents_e,
// out_keys_e, out_votes_e: the event's arrays.
template <int MODE>
__device__ __forceinline__ void children_pair(const DevGeom &g, const unsigned char *h64s,
                                              const unsigned char *h32s, int nh, const uint32_t *act,
                                              int level, const uint64_t *parents_e, long long j,
                                              uint64_t *out_keys_e, int32_t *out_votes_e) {
    constexpr bool k64 = ModeOf<MODE>::k64, k32 = ModeOf<MODE>::k32;
    const int b = (int)(j % 16);
    int idx[5];
    unpack_key(g, parents_e[j / 16], idx);
#pragma unroll
    for (int a = 0; a < 4; a++) idx[a] = 2 * idx[a] + ((b >> a) & 1);
    const int l0 = 2 * idx[4];                    // tan(lambda) bit 0 / 1 of the pair
    idx[4] = l0;
    const uint64_t key0 = pack_key(g, idx);
    const uint64_t key1 = key0 + (1ULL << g.key_shift[4]);
    Cell<double> c{edge(g, 0, level, idx[0]), sin_phi0(g, level, idx[1]), cos_phi0(g, level, idx[1]),
                   edge(g, 2, level, idx[2]), edge(g, 3, level, idx[3]), edge(g, 4, level, l0)};
    const IV<double> L1 = edge(g, 4, level, l0 + 1);
    Cell<float> c32{to_prec<float>(c.D), to_prec<float>(c.S0), to_prec<float>(c.C0),
                    to_prec<float>(c.W), to_prec<float>(c.Z), to_prec<float>(c.L)};
    const IV<float> L1f = to_prec<float>(L1);
    const bool mir = mirror_cell(c);
    mirror_cell(c32);
    const bool wguard = !gt0(c.W.lo) || !gt0(c32.W.lo);
    const IV<double> R = recip(c.W);
    const IV<float> R32 = recip(c32.W);
    const SeriesConsts &k = g.k;
    int v0 = 0, v1 = 0;
    for (int h = 0; h < nh; h++) {
        if (act && !((act[h >> 5] >> (h & 31)) & 1u)) continue;
        if (wguard) { v0++; v1++; continue; }
        unsigned lm = 3u;
        if (k32) {
            Hit<float> h32 = load_hit<float>(h32s + h * 80);
            if (mir) mirror_hit(h32);
            Pre<float> p32 = prefix<float>(c32, h32, k);
            if (p32.novote) {
                lm = 0u;
            } else if (!p32.guard) {
                lm = (tail<float>(p32, c32.L, h32, R32, c32.W, k) ? 1u : 0u) |
                     (tail<float>(p32, L1f, h32, R32, c32.W, k) ? 2u : 0u);
            }
            if (!k64) { v0 += lm & 1u; v1 += lm >> 1; continue; }
            if (!lm) continue;
        }
        Hit<double> h64 = load_hit<double>(h64s + h * 80);
        if (mir) mirror_hit(h64);
        Pre<double> p64 = prefix<double>(c, h64, k);
        if (p64.novote) continue;
        if (p64.guard) { v0++; v1++; continue; }
        if (ModeOf<MODE>::exact) {
            if ((lm & 1u) && tail_exact(p64, c.L, h64, R, c.W, k)) v0++;
            if ((lm & 2u) && tail_exact(p64, L1, h64, R, c.W, k)) v1++;
        } else {
            if ((lm & 1u) && tail<double>(p64, c.L, h64, R, c.W, k)) v0++;
            if ((lm & 2u) && tail<double>(p64, L1, h64, R, c.W, k)) v1++;
        }
    }
    // output order: child b at 32 j' + b, child b + 16 at 32 j' + b + 16 (j' = parent)
    const long long o = (j / 16) * 32 + b;
    out_keys_e[o] = key0;
    out_votes_e[o] = v0;
    out_keys_e[o + 16] = key1;
    out_votes_e[o + 16] = v1;
}

// NT: threads per block, 256 or 128; the 128-thread form asks for three resident blocks
// per SM (12 warps), which the FP64 modes' register count otherwise limits to 8 warps.
template <int MODE, int NT>
__global__ void __launch_bounds__(NT, NT == 128 ? 3 : 1)
k_vote_children(DevGeom g, const HitRecD *hd, const HitRecF *hf, const int32_t *n_hits,
                const uint32_t *active, int level, const uint64_t *parents, int n_par,
                const int32_t *n_valid, uint64_t *out_keys, int32_t *out_votes, unsigned *status) {
    constexpr bool k64 = ModeOf<MODE>::k64, k32 = ModeOf<MODE>::k32;
    extern __shared__ __align__(16) unsigned char smem[];
    unsigned char *h64s = smem;
    unsigned char *h32s = smem + (k64 ? kHitCap * 80 : 0);
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + (k64 ? kHitCap * 80 : 0) + (k32 ? kHitCap * 80 : 0));
    const int ev = blockIdx.y;
    // n_valid (may be null): parents 0 .. n_valid[ev] - 1 of the event's n_par slots are
    // real; a block past them has nothing to do (the condition is uniform in the block)
    const long long n_here = n_valid ? (long long)n_valid[ev] : (long long)n_par;
    if ((long long)blockIdx.x * blockDim.x >= n_here * 16) return;
    int nh = n_hits[ev];
    if (nh < 0) nh = 0;
    const unsigned bytes = (unsigned)nh * 80u;
    bool ok = stage_to_smem(h64s, hd + (long long)ev * kHitCap, k64 ? bytes : 0u, h32s,
                            hf + (long long)ev * kHitCap, k32 ? bytes : 0u, bar, status);
    __syncthreads();
    if (!ok) nh = 0;
    const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n_here * 16) return;
    children_pair<MODE>(g, h64s, h32s, nh, active ? active + (long long)ev * 8 : nullptr, level,
                        parents + (long long)ev * n_par, j, out_keys + (long long)ev * n_par * 32,
                        out_votes + (long long)ev * n_par * 32);
}

template <int MODE>
static void launch_cells_mode(const DevGeom &g, int n_ev, const HitRecD *hd, const HitRecF *hf,
                              const int32_t *n_hits, const uint32_t *active, int level,
                              const uint64_t *keys, const uint64_t *parents, long long n_per_ev,
                              uint64_t *out_keys, int32_t *out_votes, unsigned *status, cudaStream_t s,
                              int block) {
    smem_limit_once(k_vote_cells<MODE>, g_attr_cells[MODE]);
    size_t sm = (ModeOf<MODE>::k64 ? kHitCap * 80 : 0) + (ModeOf<MODE>::k32 ? kHitCap * 80 : 0) + 16;
    dim3 grid((unsigned)((n_per_ev + block - 1) / block), n_ev);
    k_vote_cells<MODE><<<grid, block, sm, s>>>(g, hd, hf, n_hits, active, level, keys, parents, n_per_ev,
                                                out_keys, out_votes, status);
}

static void launch_cells(const DevGeom &g, int prec, int n_ev, const HitRecD *hd, const HitRecF *hf,
                         const int32_t *n_hits, const uint32_t *active, int level,
                         const uint64_t *keys, const uint64_t *parents, long long n_per_ev,
                         uint64_t *out_keys, int32_t *out_votes, unsigned *status, cudaStream_t s,
                         int block = 256) {
    if (block != 128) block = 256;
    if (prec == APO_F64_MID)
        launch_cells_mid(g, n_ev, hd, n_hits, active, level, keys, parents, n_per_ev, out_keys, out_votes,
                         status, s, block);
    else if (prec == APO_F64_EXACT)
        launch_cells_mode<kModeF64Exact>(g, n_ev, hd, hf, n_hits, active, level, keys, parents, n_per_ev,
                                         out_keys, out_votes, status, s, block);
    else if (prec == APO_F32)
        launch_cells_mode<kModeF32>(g, n_ev, hd, hf, n_hits, active, level, keys, parents, n_per_ev,
                                    out_keys, out_votes, status, s, block);
    else if (prec == APO_F64_FILTERED)
        launch_cells_mode<kModeF64Filtered>(g, n_ev, hd, hf, n_hits, active, level, keys, parents,
                                            n_per_ev, out_keys, out_votes, status, s, block);
    else
        launch_cells_mode<kModeF64>(g, n_ev, hd, hf, n_hits, active, level, keys, parents, n_per_ev,
                                    out_keys, out_votes, status, s, block);
}

void launch_vote_keys(const DevGeom &g, int prec, int n_ev, const HitRecD *hd, const HitRecF *hf,
                      const int32_t *n_hits, int level, const uint64_t *keys, long long n_per_ev,
                      int32_t *votes, cudaStream_t s, const uint32_t *active) {
    if (n_ev <= 0 || n_per_ev <= 0) return;
    launch_cells(g, prec, n_ev, hd, hf, n_hits, active, level, keys, nullptr, n_per_ev, nullptr, votes,
                 nullptr, s);
}

template <int MODE>
static void launch_children_mode(const DevGeom &g, int n_ev, const HitRecD *hd, const HitRecF *hf,
                                 const int32_t *n_hits, const uint32_t *active, int level,
                                 const uint64_t *parents, int n_par, const int32_t *n_valid,
                                 uint64_t *out_keys, int32_t *out_votes, cudaStream_t s, int block) {
    size_t sm = (ModeOf<MODE>::k64 ? kHitCap * 80 : 0) + (ModeOf<MODE>::k32 ? kHitCap * 80 : 0) + 16;
    dim3 grid((unsigned)(((long long)n_par * 16 + block - 1) / block), n_ev);
    if (block == 128) {
        k_vote_children<MODE, 128><<<grid, 128, sm, s>>>(g, hd, hf, n_hits, active, level, parents, n_par,
                                                         n_valid, out_keys, out_votes, nullptr);
    } else {
        k_vote_children<MODE, 256><<<grid, 256, sm, s>>>(g, hd, hf, n_hits, active, level, parents, n_par,
                                                         n_valid, out_keys, out_votes, nullptr);
    }
}

void launch_vote_children(const DevGeom &g, int prec, int n_ev, const HitRecD *hd,
                          const HitRecF *hf, const int32_t *n_hits, int child_level,
                          const uint64_t *parents, int n_par, uint64_t *child_keys,
                          int32_t *child_votes, cudaStream_t s, const uint32_t *active, int block,
                          const int32_t *n_valid) {
    if (n_ev <= 0 || n_par <= 0) return;
    if (block != 128) block = 256;
    if (prec == APO_F64_MID) {   // children in the order of k_vote_children: 32 per parent
        launch_cells_mid(g, n_ev, hd, n_hits, active, child_level, nullptr, parents, (long long)n_par * 32,
                         child_keys, child_votes, nullptr, s, block);
        return;
    }
    if (prec == APO_F64_EXACT)
        launch_children_mode<kModeF64Exact>(g, n_ev, hd, hf, n_hits, active, child_level, parents, n_par,
                                            n_valid, child_keys, child_votes, s, block);
    else if (prec == APO_F32)
        launch_children_mode<kModeF32>(g, n_ev, hd, hf, n_hits, active, child_level, parents, n_par,
                                       n_valid, child_keys, child_votes, s, block);
    else if (prec == APO_F64_FILTERED)
        launch_children_mode<kModeF64Filtered>(g, n_ev, hd, hf, n_hits, active, child_level, parents, n_par,
                                               n_valid, child_keys, child_votes, s, block);
    else
        launch_children_mode<kModeF64>(g, n_ev, hd, hf, n_hits, active, child_level, parents, n_par,
                                       n_valid, child_keys, child_votes, s, block);
}

// Sets every vote kernel's dynamic shared-memory limit now, outside any stream capture.
void init_kernel_attributes() {
    const int lim = 96 * 1024;   // on the current device, every time a geometry is created there
    cudaFuncSetAttribute(k_vote_coarse<kModeF32>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    cudaFuncSetAttribute(k_vote_coarse<kModeF64>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    cudaFuncSetAttribute(k_vote_coarse<kModeF64Filtered>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    cudaFuncSetAttribute(k_vote_cells<kModeF32>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    cudaFuncSetAttribute(k_vote_cells<kModeF64>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    cudaFuncSetAttribute(k_vote_cells<kModeF64Filtered>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    cudaFuncSetAttribute(k_vote_children<kModeF32, 256>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    cudaFuncSetAttribute(k_vote_children<kModeF32, 128>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    cudaFuncSetAttribute(k_vote_children<kModeF64, 256>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    cudaFuncSetAttribute(k_vote_children<kModeF64, 128>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    cudaFuncSetAttribute(k_vote_children<kModeF64Filtered, 256>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    cudaFuncSetAttribute(k_vote_children<kModeF64Filtered, 128>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    cudaFuncSetAttribute(k_vote_coarse<kModeF64Exact>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    cudaFuncSetAttribute(k_vote_cells<kModeF64Exact>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    cudaFuncSetAttribute(k_vote_children<kModeF64Exact, 256>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    cudaFuncSetAttribute(k_vote_children<kModeF64Exact, 128>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    for (int i = 0; i < 4; i++) g_attr_coarse[i] = g_attr_cells[i] = g_attr_children[i] = true;
}

// ---------------------------------------------------------------------------------------
// Coarse top-K: threshold from the vote histogram, then an order-preserving compaction.
// Keeps every cell with votes above the threshold v* and the lowest-key cells at v*, so the
// kept set is the K best by (votes desc, key asc).  From the histogram: A = #(v > v*) < K
// and need = K - A.  One pass over the event's votes in key order, 4096 cells per tile,
// each thread 4 consecutive cells (one 16-byte load where aligned); cells above v* go to
// slot (rank among them), cells at v* to slot A + (rank among them) while that is < K.
// A tile with nothing to keep costs one barrier; the pass ends once all A cells and
// `need` tied cells are placed.  Votes are clamped to [0, kHitCap] as the histogram does.
// ---------------------------------------------------------------------------------------
constexpr int kSelThreads = 1024;
constexpr int kSelTile = 4 * kSelThreads;

// One event's selection by one block of any multiple-of-32 size (tiles of 4 cells per
// thread): vo = the event's level-0 votes, hist_e its histogram, ok_ / ov its K outputs.
__device__ __forceinline__ void select_coarse_block(const DevGeom &g, const int32_t *vo, const uint32_t *hist_e,
                                                    int K, uint64_t *ok_, int32_t *ov) {
    __shared__ int s_vstar, s_need, s_above;
    __shared__ int s_warp[32];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nwarps = blockDim.x >> 5;
    const long long tile = 4LL * blockDim.x;
    const long long n = (long long)g.bins[0] * g.bins[1] * g.bins[2] * g.bins[3] * g.bins[4];
    if (tid == 0) {
        long long cum = 0;
        int vstar = -1, need = 0;
        for (int v = kHistBins - 1; v >= 0; v--) {
            long long h = hist_e[v];
            if (cum + h >= K) { vstar = v; need = (int)(K - cum); break; }
            cum += h;
        }
        s_vstar = vstar;
        s_need = need;
        s_above = (int)cum;
    }
    __syncthreads();
    const int vstar = s_vstar, need = s_need, above = s_above;
    const bool vec = (n % 4 == 0) && ((reinterpret_cast<uintptr_t>(vo) & 15) == 0);
    int runA = 0, runB = 0;   // cells above v* / at v* in the tiles before this one
    for (long long t0 = 0; t0 < n; t0 += tile) {
        if (runA >= above && runB >= need) break;
        const long long j0 = t0 + 4LL * tid;
        int v[4];
        if (vec && j0 + 3 < n) {
            int4 q = __ldcs(reinterpret_cast<const int4 *>(vo + j0));
            v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
        } else {
#pragma unroll
            for (int r = 0; r < 4; r++) v[r] = j0 + r < n ? __ldcs(vo + j0 + r) : INT_MIN;
        }
        int a = 0, b = 0;
#pragma unroll
        for (int r = 0; r < 4; r++) {
            if (v[r] != INT_MIN) v[r] = v[r] < 0 ? 0 : (v[r] > kHitCap ? kHitCap : v[r]);
            a += v[r] > vstar;
            b += v[r] == vstar;
        }
        if (!__syncthreads_or(a > 0 || (b > 0 && runB < need))) continue;
        // block exclusive scan of (a, b) packed as a + (b << 16); a tile holds < 2^16 cells
        const int x = a + (b << 16);
        int inc = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += y;
        }
        if (lane == 31) s_warp[wid] = inc;
        __syncthreads();
        int w = lane < nwarps ? s_warp[lane] : 0;
        int winc = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, winc, o);
            if (lane >= o) winc += y;
        }
        const int wpre = __shfl_sync(0xffffffffu, winc - w, wid);
        const int total = __shfl_sync(0xffffffffu, winc, 31);
        const int pre = wpre + inc - x;
        int pa = runA + (pre & 0xffff), pb = runB + (pre >> 16);
#pragma unroll
        for (int r = 0; r < 4; r++) {
            const bool ka = v[r] > vstar, kb = v[r] == vstar;
            int pos = -1;
            if (ka) pos = pa++;
            else if (kb) { if (pb < need) pos = above + pb; pb++; }
            if (pos >= 0 && pos < K) {
                long long rr = j0 + r;
                int idx[5];
                for (int q = 0; q < 5; q++) { idx[q] = (int)(rr % g.bins[q]); rr /= g.bins[q]; }
                ok_[pos] = pack_key(g, idx);
                ov[pos] = v[r];
            }
        }
        runA += total & 0xffff;
        runB += total >> 16;
        __syncthreads();   // s_warp is rewritten by the next scanned tile
    }
    __syncthreads();
}

__global__ void __launch_bounds__(kSelThreads)
k_select_coarse(DevGeom g, int ev0, const int32_t *votes, const uint32_t *hist, int K,
                uint64_t *out_keys, int32_t *out_votes) {
    const int e = blockIdx.x, ev = ev0 + e;
    const long long n = (long long)g.bins[0] * g.bins[1] * g.bins[2] * g.bins[3] * g.bins[4];
    select_coarse_block(g, votes + (long long)e * n, hist + (long long)e * kHistBins, K,
                        out_keys + (long long)ev * K, out_votes + (long long)ev * K);
}

// Top-K of level 0 from the coarse blocks' candidates (see launch_vote_coarse): the same v*
// and need from the event's histogram as k_select_coarse; every candidate above v* is kept
// (there are exactly `above` of them), then the `need` lowest keys at v*.  In each block's
// list the candidates at v* come in key order, so the lowest keys overall come from a
// merge: `need` rounds, each taking the smallest head over the lists.
__global__ void __launch_bounds__(kSelThreads)
k_select_candidates(int ev0, const uint64_t *cand_k, const int32_t *cand_v, int n_lists,
                    const uint32_t *hist, int K, uint64_t *out_keys, int32_t *out_votes) {
    extern __shared__ int s_head[];          // n_lists heads
    __shared__ int s_vstar, s_need, s_above, s_nA;
    __shared__ unsigned long long s_red[32];
    const int e = blockIdx.x, ev = ev0 + e, tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const uint64_t *ck = cand_k + (long long)e * n_lists * K;
    const int32_t *cv = cand_v + (long long)e * n_lists * K;
    uint64_t *ok_ = out_keys + (long long)ev * K;
    int32_t *ov = out_votes + (long long)ev * K;
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
        s_above = (int)cum;
        s_nA = 0;
    }
    __syncthreads();
    const int vstar = s_vstar, need = s_need, above = s_above;
    for (long long i = tid; i < (long long)n_lists * K; i += blockDim.x) {
        const int v = cv[i];
        if (v > vstar) {
            const int pos = atomicAdd(&s_nA, 1);
            if (pos < K) { ok_[pos] = ck[i]; ov[pos] = v; }
        }
    }
    for (int t = tid; t < n_lists; t += blockDim.x) {
        int j = 0;
        while (j < K && cv[(long long)t * K + j] != vstar) j++;
        s_head[t] = j;
    }
    __syncthreads();
    const int nwarps = blockDim.x >> 5;
    for (int r = 0; r < need; r++) {
        unsigned long long best = ~0ULL;   // (key << 13) | list: keys of at most 50 bits
        for (int t = tid; t < n_lists; t += blockDim.x) {
            const int j = s_head[t];
            if (j < K) {
                const unsigned long long x = (ck[(long long)t * K + j] << 13) | (unsigned long long)t;
                best = x < best ? x : best;
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long y = __shfl_down_sync(0xffffffffu, best, o);
            best = y < best ? y : best;
        }
        if (lane == 0) s_red[wid] = best;
        __syncthreads();
        if (tid == 0) {
            unsigned long long b = ~0ULL;
            for (int q = 0; q < nwarps; q++) b = s_red[q] < b ? s_red[q] : b;
            const int t = (int)(b & 8191ULL);
            ok_[above + r] = b >> 13;
            ov[above + r] = vstar;
            int j = s_head[t] + 1;
            while (j < K && cv[(long long)t * K + j] != vstar) j++;
            s_head[t] = j;
        }
        __syncthreads();
    }
}

void launch_select_candidates(const DevGeom &, int ev0, int n_ev, const uint64_t *cand_k,
                              const int32_t *cand_v, int n_lists, const uint32_t *hist, int K,
                              uint64_t *out_keys, int32_t *out_votes, cudaStream_t s) {
    if (n_ev <= 0) return;
    k_select_candidates<<<n_ev, kSelThreads, sizeof(int) * (size_t)n_lists, s>>>(
        ev0, cand_k, cand_v, n_lists, hist, K, out_keys, out_votes);
}

void launch_select_coarse(const DevGeom &g, int ev0, int n_ev, const int32_t *votes,
                          const uint32_t *hist, int K, uint64_t *out_keys, int32_t *out_votes,
                          cudaStream_t s) {
    if (n_ev <= 0) return;
    k_select_coarse<<<n_ev, kSelThreads, 0, s>>>(g, ev0, votes, hist, K, out_keys, out_votes);
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

// One event's top-K by one block: s = shared scratch of pow2_ge(n_in) entries.
__device__ __forceinline__ void topk_block(const uint64_t *keys_e, const int32_t *votes_e, int n_in, int K,
                                           uint64_t *out_keys_e, int32_t *out_votes_e, uint64_t *s) {
    int np2 = pow2_ge(n_in);
    load_sorted(s, keys_e, votes_e, n_in, np2);
    for (int i = threadIdx.x; i < K; i += blockDim.x) {
        uint64_t x = i < n_in ? s[i] : ~0ULL;
        out_keys_e[i] = x & kKeyMask;
        out_votes_e[i] = i < n_in ? 1023 - (int)(x >> 50) : 0;
    }
    __syncthreads();
}

__global__ void __launch_bounds__(1024)
k_topk(const uint64_t *keys, const int32_t *votes, int n_in, int K, uint64_t *out_keys,
       int32_t *out_votes) {
    __shared__ uint64_t s[kSortMax];
    const int e = blockIdx.x;
    topk_block(keys + (long long)e * n_in, votes + (long long)e * n_in, n_in, K, out_keys + (long long)e * K,
               out_votes + (long long)e * K, s);
}

void launch_topk(int n_ev, const uint64_t *keys, const int32_t *votes, int n_in, int K,
                 uint64_t *out_keys, int32_t *out_votes, cudaStream_t s) {
    if (n_ev <= 0) return;
    k_topk<<<n_ev, 1024, 0, s>>>(keys, votes, n_in, K, out_keys, out_votes);
}

// ---------------------------------------------------------------------------------------
// Final estimate (Section 3.3) and, for multi-track extraction, hit masking.  Per event
// (one block) in round `round`: stop (done) if no hit is active or the best final vote
// count is below min_votes; otherwise write track `round`: over the maximum-vote cells in
// ascending key order, the mean of the cell centres and the half-extent of their union per
// axis, in round-to-nearest.  Then deactivate every active hit that votes (FP64) for at
// least one maximum-vote cell with its drift widened to [max(rd(d - width), 0),
// ru(d + width)] (the paper's hit finding with a widened box, Section 3.3).
// ---------------------------------------------------------------------------------------
constexpr int kEstChunk = 256;

// One event's estimate and hit masking by one block (any multiple of 32 threads, at least
// 64): keys_e / votes_e the last level's cells, active_e its 8 mask words, done_e its flag,
// hd_e its staged hits, te its max_tracks records, n_tracks_e its count, a0 its first hit
// in the batch (for hit_track).  s: shared scratch of kSortMax entries; s_cen: of
// kEstChunk x 5.
__device__ __forceinline__ void estimate_mask_block(const DevGeom &g, const uint64_t *keys_e, const int32_t *votes_e,
                                                    int n_in, int level, int nh, uint32_t *active_e,
                                                    int32_t *done_e, const HitRecD *hd_e, int round,
                                                    int max_tracks, int min_votes, double width,
                                                    apo_track *te, int32_t *n_tracks_e, int a0,
                                                    int32_t *hit_track, uint64_t *s, double *s_cen) {
    __shared__ long long s_lo[5], s_hi[5];
    __shared__ uint32_t act0[8], act1[8];
    __shared__ int s_m;
    const int tid = threadIdx.x;
    if (*done_e) return;
    if (round == 0) {
        if (tid < max_tracks) {
            for (int a = 0; a < 5; a++) { te[tid].p[a] = 0.0; te[tid].w[a] = 0.0; }
            te[tid].votes = (tid == 0 && nh < 0) ? nh : 0;
            te[tid].n_hits = nh < 0 ? 0 : nh;
        }
        if (tid == 0) *n_tracks_e = 0;
    }
    if (nh < 0) {
        __syncthreads();
        if (tid == 0) *done_e = 1;
        __syncthreads();
        return;
    }
    if (tid < 8) act0[tid] = act1[tid] = active_e[tid];
    __syncthreads();
    int na = 0;
    for (int i = 0; i < 8; i++) na += __popc(act0[i]);
    if (na == 0) {
        __syncthreads();
        if (tid == 0) *done_e = 1;
        __syncthreads();
        return;
    }
    if (tid == 0) s_m = 0;
    if (tid < 5) { s_lo[tid] = okey(1e300); s_hi[tid] = okey(-1e300); }
    int np2 = pow2_ge(n_in);
    load_sorted(s, keys_e, votes_e, n_in, np2);
    // the maximum-vote cells are s[0, m) after the sort
    const uint64_t top = s[0] >> 50;
    const int vmax = 1023 - (int)top;
    {
        int cnt = 0;
        for (int i = tid; i < n_in; i += blockDim.x) cnt += (s[i] >> 50) == top;
        if (cnt) atomicAdd(&s_m, cnt);
    }
    __syncthreads();
    const int m = s_m;
    if (vmax < min_votes) {
        if (tid == 0) *done_e = 1;
        __syncthreads();
        return;
    }
    // Centres of the m cells, staged per chunk by all threads; thread a < 5 then adds axis
    // a's centres in key order (the same round-to-nearest sequence as a serial loop).  The
    // union's ends are order-free: min / max through atomics on value-ordered keys.
    double sum = 0.0;
    for (int c0 = 0; c0 < m; c0 += kEstChunk) {
        const int cn = m - c0 < kEstChunk ? m - c0 : kEstChunk;
        for (int q = tid; q < cn * 5; q += blockDim.x) {
            const int j = q / 5, a = q - 5 * j;
            int idx[5];
            unpack_key(g, s[c0 + j] & kKeyMask, idx);
            IV<double> ed = edge(g, a, level, idx[a]);
            s_cen[q] = __dmul_rn(__dadd_rn(ed.lo, ed.hi), 0.5);
            atomicMin(&s_lo[a], okey(ed.lo));
            atomicMax(&s_hi[a], okey(ed.hi));
        }
        __syncthreads();
        if (tid < 5)
            for (int j = 0; j < cn; j++) sum = __dadd_rn(sum, s_cen[5 * j + tid]);
        __syncthreads();
    }
    if (tid < 5) {
        apo_track &t = te[round];
        const double lo_min = __longlong_as_double(okey_inv(s_lo[tid]));
        const double hi_max = __longlong_as_double(okey_inv(s_hi[tid]));
        t.p[tid] = __ddiv_rn(sum, (double)m);
        t.w[tid] = __dmul_rn(__dsub_rn(hi_max, lo_min), 0.5);
        if (tid == 0) {
            t.votes = vmax;
            t.n_hits = nh;
            *n_tracks_e = round + 1;
        }
    }
    const bool last = round + 1 >= max_tracks;
    if (last && !hit_track) {   // no later round needs the masks
        if (tid == 0) *done_e = 1;
        __syncthreads();
        return;
    }
    const SeriesConsts &k = g.k;
    const long long pairs = (long long)m * nh;
    for (long long q = tid; q < pairs; q += blockDim.x) {
        const int j = (int)(q / nh), i = (int)(q % nh);
        if (!((act0[i >> 5] >> (i & 31)) & 1u)) continue;
        if (!((act1[i >> 5] >> (i & 31)) & 1u)) continue;   // already masked by another cell
        int idx[5];
        unpack_key(g, s[j] & kKeyMask, idx);
        Cell<double> c{edge(g, 0, level, idx[0]), sin_phi0(g, level, idx[1]), cos_phi0(g, level, idx[1]),
                       edge(g, 2, level, idx[2]), edge(g, 3, level, idx[3]), edge(g, 4, level, idx[4])};
        Hit<double> h = load_hit<double>(hd_e + i);
        const double d = h.d.lo;
        const double dlo = __dsub_rd(d, width);
        h.d = {gt0(dlo) ? dlo : 0.0, __dadd_ru(d, width)};
        if (vote_pair<double>(c, h, k)) atomicAnd(&act1[i >> 5], ~(1u << (i & 31)));
    }
    __syncthreads();
    if (tid < 8) active_e[tid] = act1[tid];
    if (hit_track) {   // the hits this track took: active before, masked now
        for (int i = tid; i < nh; i += blockDim.x)
            if (((act0[i >> 5] & ~act1[i >> 5]) >> (i & 31)) & 1u) hit_track[a0 + i] = round;
    }
    if (tid == 0) {
        int left = 0;
        for (int i = 0; i < 8; i++) left += __popc(act1[i]);
        if (left == 0 || last) *done_e = 1;
    }
    __syncthreads();
}

__global__ void __launch_bounds__(256)
k_estimate_mask(DevGeom g, const uint64_t *keys, const int32_t *votes, int n_in, int level,
                const int32_t *n_hits, uint32_t *active, int32_t *done, const HitRecD *hd,
                int round, int max_tracks, int min_votes, double width, apo_track *out,
                int32_t *n_tracks, const int32_t *offsets, int32_t *hit_track) {
    __shared__ uint64_t s[kSortMax];
    __shared__ double s_cen[kEstChunk * 5];
    const int e = blockIdx.x;
    estimate_mask_block(g, keys + (long long)e * n_in, votes + (long long)e * n_in, n_in, level, n_hits[e],
                        active + (long long)e * 8, done + e, hd + (long long)e * kHitCap, round, max_tracks,
                        min_votes, width, out + (long long)e * max_tracks, n_tracks + e,
                        hit_track ? offsets[e] : 0, hit_track, s, s_cen);
}

void launch_estimate_mask(const DevGeom &g, int n_ev, const uint64_t *keys, const int32_t *votes,
                          int n_in, int level, const int32_t *n_hits, uint32_t *active, int32_t *done,
                          const HitRecD *hd, int round, int max_tracks, int min_votes, double width,
                          apo_track *out, int32_t *n_tracks, cudaStream_t s, const int32_t *offsets,
                          int32_t *hit_track) {
    if (n_ev <= 0) return;
    k_estimate_mask<<<n_ev, 256, 0, s>>>(g, keys, votes, n_in, level, n_hits, active, done, hd, round,
                                          max_tracks, min_votes, width, out, n_tracks, offsets,
                                          hit_track);
}

// ---------------------------------------------------------------------------------------
// Persistent batch search (top-K schedule, multi-track rounds).  One launch of as many
// blocks as the GPU holds at once.  Each block pulls the next event from a device counter
// and runs that event's whole search: per round the level-0 tiles (with the parent-cell
// test), the top-K selection, every bisection level with its top-K, and the estimate with
// the hit masking of Section 3.3; then the next round or the next event.  The steps are
// the device functions of the per-level kernels above (same operations, same results);
// only their scheduling differs.  Events are independent, so no block ever waits on
// another: uneven events (10-200 hits) simply keep their block longer while the others
// pull new ones, and no launch boundary waits for the slowest event of a level.  The only
// device waits are the bounded waits of the hit staging.
// ---------------------------------------------------------------------------------------
template <int MODE> __device__ __noinline__ void persist_coarse(const DevGeom &g, const PersistArgs &A, int e,
                                                                   int32_t *vo, uint32_t *hist_b,
                                                                   unsigned char *smem) {
    const int split = (g.bins[0] * g.bins[3] + blockDim.x - 1) / blockDim.x;
    const int ntiles = g.bins[1] * g.bins[2] * split;
    for (int t = 0; t < ntiles; t++) {
        const int part = t % split, pw = t / split;
        coarse_block<MODE>(g, e, split, part, pw % g.bins[1], pw / g.bins[1], A.hd, A.hf, A.n_hits,
                           A.active, vo, hist_b, A.status, nullptr, smem);
    }
}

template <int MODE> __device__ __noinline__ void persist_children(const DevGeom &g, const PersistArgs &A, int e,
                                                                     int level, unsigned char *smem) {
    constexpr bool k64 = ModeOf<MODE>::k64, k32 = ModeOf<MODE>::k32;
    unsigned char *h64s = smem;
    unsigned char *h32s = smem + (k64 ? kHitCap * 80 : 0);
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + (k64 ? kHitCap * 80 : 0) + (k32 ? kHitCap * 80 : 0));
    int nh = A.n_hits[e];
    if (nh < 0) nh = 0;
    const unsigned bytes = (unsigned)nh * 80u;
    bool ok = stage_to_smem(h64s, A.hd + (long long)e * kHitCap, k64 ? bytes : 0u, h32s,
                            A.hf + (long long)e * kHitCap, k32 ? bytes : 0u, bar, A.status);
    __syncthreads();
    if (threadIdx.x == 0) mbar_inval(bar);
    if (!ok) nh = 0;
    const int K = g.topk;
    const uint32_t *act = A.active + (long long)e * 8;
    for (long long j = threadIdx.x; j < (long long)K * 16; j += blockDim.x)
        children_pair<MODE>(g, h64s, h32s, nh, act, level, A.fk + (long long)e * K, j,
                            A.ck + (long long)e * K * 32, A.cv + (long long)e * K * 32);
    __syncthreads();
}

__global__ void __launch_bounds__(128, 3) k_solve_persistent(DevGeom g, PersistArgs A) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_e;
    const int lv = g.levels, K = g.topk;
    const long long ncell = (long long)g.bins[0] * g.bins[1] * g.bins[2] * g.bins[3] * g.bins[4];
    int32_t *vo = A.votes + (long long)blockIdx.x * ncell;        // this block's level-0 votes
    uint32_t *hist_b = A.hist + (long long)blockIdx.x * kHistBins;
    uint64_t *s_sort = reinterpret_cast<uint64_t *>(smem);
    double *s_cen = reinterpret_cast<double *>(smem + kSortMax * sizeof(uint64_t));
    for (;;) {
        if (threadIdx.x == 0) s_e = atomicAdd(A.next_event, 1);
        __syncthreads();
        const int e = s_e;
        __syncthreads();
        if (e >= A.n_events) break;
        for (int round = 0; round < A.max_tracks; round++) {
            if (A.done[e]) break;
            for (int i = threadIdx.x; i < kHistBins; i += blockDim.x) hist_b[i] = 0u;
            __syncthreads();
            switch (A.mode[0]) {
                case kModeF32: persist_coarse<kModeF32>(g, A, e, vo, hist_b, smem); break;
                case kModeF64Filtered: persist_coarse<kModeF64Filtered>(g, A, e, vo, hist_b, smem); break;
                default: persist_coarse<kModeF64>(g, A, e, vo, hist_b, smem); break;
            }
            __threadfence_block();
            __syncthreads();
            select_coarse_block(g, vo, hist_b, K, A.fk + (long long)e * K, A.fv + (long long)e * K);
            for (int lev = 1; lev <= lv; lev++) {
                switch (A.mode[lev]) {
                    case kModeF32: persist_children<kModeF32>(g, A, e, lev, smem); break;
                    case kModeF64Filtered: persist_children<kModeF64Filtered>(g, A, e, lev, smem); break;
                    default: persist_children<kModeF64>(g, A, e, lev, smem); break;
                }
                topk_block(A.ck + (long long)e * K * 32, A.cv + (long long)e * K * 32, K * 32, K,
                           A.fk + (long long)e * K, A.fv + (long long)e * K, s_sort);
            }
            estimate_mask_block(g, A.ck + (long long)e * K * 32, A.cv + (long long)e * K * 32, K * 32, lv,
                                A.n_hits[e], A.active + (long long)e * 8, A.done + e,
                                A.hd + (long long)e * kHitCap, round, A.max_tracks, A.min_votes, A.width,
                                A.tracks + (long long)e * A.max_tracks, A.n_tracks + e,
                                A.hit_track ? A.offsets[e] : 0, A.hit_track, s_sort, s_cen);
        }
    }
}

static_assert(kPersistF32 == kModeF32 && kPersistF64 == kModeF64 && kPersistF64Filtered == kModeF64Filtered,
              "persistent launch modes");

size_t persist_smem_bytes(const DevGeom &g) {
    size_t a = CoarseSmem<kModeF64Filtered>::total(g.bins[4], 128);
    size_t b = 2 * kHitCap * 80 + 16;
    size_t c = kSortMax * sizeof(uint64_t) + kEstChunk * 5 * sizeof(double);
    size_t m = a > b ? a : b;
    return m > c ? m : c;
}

int persist_blocks(const DevGeom &g) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaFuncSetAttribute(k_solve_persistent, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_solve_persistent, 128, persist_smem_bytes(g));
    if (per_sm < 1) per_sm = 1;
    return sms * per_sm;
}

void launch_solve_persistent(const DevGeom &g, int blocks, const PersistArgs &A, cudaStream_t s) {
    if (A.n_events <= 0 || blocks <= 0) return;
    k_solve_persistent<<<blocks, 128, persist_smem_bytes(g), s>>>(g, A);
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
__global__ void k_children(DevGeom g, const uint64_t *keys, long long n, uint64_t *out) {
    long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n * 32) return;
    int idx[5], b = (int)(j % 32);
    unpack_key(g, keys[j / 32], idx);
#pragma unroll
    for (int a = 0; a < 5; a++) idx[a] = 2 * idx[a] + ((b >> a) & 1);
    out[j] = pack_key(g, idx);
}

void launch_children(const DevGeom &g, const uint64_t *keys, long long n, uint64_t *out, cudaStream_t s) {
    if (n <= 0) return;
    k_children<<<(unsigned)((n * 32 + 255) / 256), 256, 0, s>>>(g, keys, n, out);
}

}  // namespace apo
