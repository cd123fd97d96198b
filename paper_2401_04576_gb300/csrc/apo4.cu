// The paper's own 4-D search on the GPU (include/apo4.h; arXiv:2401.04576 Sections 3.1-3.3,
// Tables tabGridDef and HelixParametes): voxel voting in the midpoint form behind the disk
// pre-filter, the per-event maximum-vote statistics, the estimate, hit finding and the
// reference-point update, all queued on the caller's stream without host round trips.
#include <cuda_runtime.h>

#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <vector>

#include "../../include/apo4.h"
#include "fourd.cuh"
#include "kernels.cuh"

using namespace apo;

struct apo4_chamber {
    DevGeom dg;      // only the wire table and n_wires are set (for the hit staging)
    int device;
    std::vector<void *> allocs;
};

namespace {

int fail4(int code, const char *fmt, ...) {
    char msg[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(msg, sizeof(msg), fmt, ap);
    va_end(ap);
    set_last_error(msg);
    return code;
}

#define CU4(call)                                                                       \
    do {                                                                                \
        cudaError_t e_ = (call);                                                        \
        if (e_ != cudaSuccess)                                                          \
            return fail4(APO_ECUDA, "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, \
                         __LINE__);                                                     \
    } while (0)

size_t al256(size_t x) { return (x + 255) & ~size_t(255); }

// One iteration's grid shape and the constants of the search, by value to the kernels.
struct Iter4 {
    double w[4];
    int n[4];
    long long ncol, nvox;
    double p_gev, b_tesla, disk_radius, hit_factor;
};

// Maximum-vote statistics of one event: count, index sums, index extent per axis.
struct Stats4 {
    unsigned long long cnt, sum[4];
    int mn[4], mx[4];
};

struct Layout4 {
    size_t status, nh, hd, hf, active, done, lo, ref, vmax, stats, lo2, ref2, active2, stats2, votes, end;
    int chunk;
    long long max_nvox;
};

Layout4 layout4(const apo4_opts *o, int ne) {
    Layout4 L{};
    long long mv = 1;
    for (int k = 0; k < 3; k++) {
        long long v = 1;
        for (int a = 0; a < 4; a++) v *= o->n[k][a];
        if (k < o->n_iter && v > mv) mv = v;
    }
    L.max_nvox = mv;
    long long c = (1LL << 30) / (8 * mv);
    L.chunk = (int)(c < 1 ? 1 : (c > ne ? (ne > 0 ? ne : 1) : c));
    size_t n = (size_t)(ne > 0 ? ne : 1);
    size_t off = 0;
    L.status = off; off += 256;
    L.nh = off; off += al256(sizeof(int32_t) * n);
    L.hd = off; off += al256(sizeof(HitRecD) * n * kHitCap);
    L.hf = off; off += al256(sizeof(HitRecF) * n * kHitCap);
    L.active = off; off += al256(sizeof(uint32_t) * n * 8);
    L.done = off; off += al256(sizeof(int32_t) * n);
    L.lo = off; off += al256(sizeof(double) * n * 4);
    L.ref = off; off += al256(sizeof(double) * n * 2);
    L.vmax = off; off += al256(sizeof(int32_t) * n * 2);
    L.stats = off; off += al256(sizeof(Stats4) * n);
    // per-sign state of iteration 3 (sign-major: sign s of event e at s n + e)
    L.lo2 = off; off += al256(sizeof(double) * 2 * n * 4);
    L.ref2 = off; off += al256(sizeof(double) * 2 * n * 2);
    L.active2 = off; off += al256(sizeof(uint32_t) * 2 * n * 8);
    L.stats2 = off; off += al256(sizeof(Stats4) * 2 * n);
    L.votes = off; off += al256(sizeof(int32_t) * 2 * (size_t)mv * (size_t)L.chunk);
    L.end = off;
    return L;
}

int check_opts(const apo4_opts *o) {
    if (!o) return fail4(APO_EINVAL, "opts is NULL");
    if (o->n_iter < 1 || o->n_iter > 3) return fail4(APO_EINVAL, "n_iter must be 1..3");
    if (o->precision != APO_F64 && o->precision != APO_F32)
        return fail4(APO_EINVAL, "precision must be APO_F64 or APO_F32");
    if (o->per_sign != 0 && o->per_sign != 1) return fail4(APO_EINVAL, "per_sign must be 0 or 1");
    if (!(o->p_gev > 0) || !(o->b_tesla > 0) || !(o->disk_radius >= 0) || !(o->hit_factor >= 0))
        return fail4(APO_EINVAL, "p_gev, b_tesla > 0 and disk_radius, hit_factor >= 0 required");
    for (int k = 0; k < o->n_iter; k++) {
        long long v = 1;
        for (int a = 0; a < 4; a++) {
            if (o->n[k][a] < 1 || o->n[k][a] > 4096) return fail4(APO_EINVAL, "n[%d][%d] out of range", k, a);
            if (!(o->w[k][a] > 0)) return fail4(APO_EINVAL, "w[%d][%d] must be > 0", k, a);
            v *= o->n[k][a];
        }
        if (o->n[k][3] > 32) return fail4(APO_EINVAL, "n[%d][3] (z0 voxels) must be <= 32", k);
        if (v > (1LL << 28)) return fail4(APO_EINVAL, "iteration %d has more than 2^28 voxels", k);
    }
    return APO_OK;
}

Iter4 iter4(const apo4_opts *o, int k) {
    Iter4 it{};
    for (int a = 0; a < 4; a++) { it.w[a] = o->w[k][a]; it.n[a] = o->n[k][a]; }
    it.ncol = (long long)it.n[0] * it.n[1] * it.n[2];
    it.nvox = it.ncol * it.n[3];
    it.p_gev = o->p_gev;
    it.b_tesla = o->b_tesla;
    it.disk_radius = o->disk_radius;
    it.hit_factor = o->hit_factor;
    return it;
}

}  // namespace

namespace apo {

// ---- precision helpers: FP64 end points as intervals / points of T ----
template <typename T> __device__ __forceinline__ IV<T> box_iv(double lo, double hi);
template <> __device__ __forceinline__ IV<double> box_iv<double>(double lo, double hi) { return {lo, hi}; }
template <> __device__ __forceinline__ IV<float> box_iv<float>(double lo, double hi) {
    return {__double2float_rd(lo), __double2float_ru(hi)};
}
template <typename T> __device__ __forceinline__ T rn(double x);
template <> __device__ __forceinline__ double rn<double>(double x) { return x; }
template <> __device__ __forceinline__ float rn<float>(double x) { return __double2float_rn(x); }
template <typename T> __device__ __forceinline__ T up(double x);   // rd of the disk radius
template <> __device__ __forceinline__ double up<double>(double x) { return x; }
template <> __device__ __forceinline__ float up<float>(double x) { return __double2float_ru(x); }

template <typename T> __device__ __forceinline__ HitP<T> hit_point(const HitRecD &r) {
    return {rn<T>(r.v[0]), rn<T>(r.v[1]), rn<T>(r.v[2]), rn<T>(r.v[3]), rn<T>(r.v[4]), rn<T>(r.v[5]),
            rn<T>(r.v[6]), rn<T>(r.v[7]), rn<T>(r.v[8])};
}
template <typename T> __device__ __forceinline__ HitI<T> hit_iv(const HitRecD &r) {
    return {box_iv<T>(r.v[0], r.v[0]), box_iv<T>(r.v[1], r.v[1]), box_iv<T>(r.v[5], r.v[5]),
            box_iv<T>(r.v[6], r.v[6])};
}

// voxel edge lo + i w (round to nearest)
__device__ __forceinline__ double edge4(double lo, int i, double w) { return __dadd_rn(lo, __dmul_rn((double)i, w)); }
__device__ __forceinline__ double mid4(double a, double b) { return __dmul_rn(__dadd_rn(a, b), 0.5); }

// ---------------------------------------------------------------------------------------
// Voting.  Block: a tile of kTile4 voxel columns (x_c, y_c, R) of one event.  First the
// block tests every column of its tile against the disk pre-filter (Eq. ApoVoteDisk) and
// the centre's validity, writes zero votes for the columns that fail, and lists the rest
// in shared memory.  Then its 128 threads share out the listed columns: each runs every
// active hit over its column's z0 voxels and both signs of tan(lambda), sharing the z0-
// and sign-free part per hit, with vote counters bit-sliced over the z0 voxels.  Listing
// first keeps the lanes of a warp on columns that all do the work; on the first
// iteration's wide grid most warps would otherwise mix passing and failing columns.
// ---------------------------------------------------------------------------------------
constexpr int kTile4 = 512;

template <typename T> struct Col4 {
    IV<T> X, Y, Rv;
    Ctr4<T> m;
};

template <typename T>
__device__ __forceinline__ Col4<T> column4(const Iter4 &it, const double *le, const double *rf,
                                           long long col) {
    const int ix = (int)(col % it.n[0]);
    const int iy = (int)((col / it.n[0]) % it.n[1]);
    const int iR = (int)(col / ((long long)it.n[0] * it.n[1]));
    const double xl = edge4(le[0], ix, it.w[0]), xh = edge4(le[0], ix + 1, it.w[0]);
    const double yl = edge4(le[1], iy, it.w[1]), yh = edge4(le[1], iy + 1, it.w[1]);
    const double rl = edge4(le[2], iR, it.w[2]), rh = edge4(le[2], iR + 1, it.w[2]);
    Col4<T> c;
    c.X = box_iv<T>(xl, xh);
    c.Y = box_iv<T>(yl, yh);
    c.Rv = box_iv<T>(rl, rh);
    c.m = centre4<T>(rn<T>(mid4(xl, xh)), rn<T>(mid4(yl, yh)), rn<T>(mid4(rl, rh)),
                     rn<T>(it.p_gev), rn<T>(it.b_tesla), rn<T>(rf[0]), rn<T>(rf[1]));
    return c;
}

template <typename T>
__global__ void __launch_bounds__(128, sizeof(T) == 8 ? 3 : 5)
k4_vote(Iter4 it, int ev0, const int32_t *n_hits, const HitRecD *hd, const uint32_t *active,
        const double *lo, const double *ref, int32_t *votes, int32_t *vmax, int sign_only) {
    __shared__ HitP<T> s_h[kHitCap];
    __shared__ HitI<T> s_w[kHitCap];
    __shared__ T s_zc[32];
    __shared__ IV<T> s_z[32];
    __shared__ short s_col[kTile4];
    __shared__ int s_n, s_np, s_vmax[2];
    const int el = blockIdx.y, e = ev0 + el, tid = threadIdx.x;
    int nh = n_hits[e];
    if (nh < 0) nh = 0;
    if (tid == 0) { s_n = 0; s_np = 0; s_vmax[0] = s_vmax[1] = 0; }
    __syncthreads();
    const uint32_t *act = active + (long long)e * 8;
    for (int i = tid; i < nh; i += blockDim.x) {
        if (!((act[i >> 5] >> (i & 31)) & 1u)) continue;
        const HitRecD r = hd[(long long)e * kHitCap + i];
        const int j = atomicAdd(&s_n, 1);
        s_h[j] = hit_point<T>(r);
        s_w[j] = hit_iv<T>(r);
    }
    const double *le = lo + (long long)e * 4;
    for (int iz = tid; iz < it.n[3]; iz += blockDim.x) {
        const double zl = edge4(le[3], iz, it.w[3]), zh = edge4(le[3], iz + 1, it.w[3]);
        s_zc[iz] = rn<T>(mid4(zl, zh));
        s_z[iz] = box_iv<T>(zl, zh);
    }
    const double *rf = ref + (long long)e * 2;
    const int nz = it.n[3];
    int32_t *vo = votes + (long long)el * 2 * it.nvox;
    const long long col0 = (long long)blockIdx.x * kTile4;
    // disk pre-filter of the tile; failing columns get zero votes
    for (int k = tid; k < kTile4; k += blockDim.x) {
        const long long col = col0 + k;
        if (col >= it.ncol) break;
        const Col4<T> c = column4<T>(it, le, rf, col);
        if (disk4<T>(c.X, c.Y, c.Rv, up<T>(it.disk_radius)) && c.m.valid) {
            s_col[atomicAdd(&s_np, 1)] = (short)k;
        } else {
            for (int s = 0; s < 2; s++)
                if (sign_only < 0 || s == sign_only)
                    for (int iz = 0; iz < nz; iz++) vo[(long long)s * it.nvox + col + it.ncol * iz] = 0;
        }
    }
    __syncthreads();
    const int na = s_n, np = s_np;
    int mx[2] = {0, 0};
    for (int i = tid; i < np; i += blockDim.x) {
        const long long col = col0 + s_col[i];
        const Col4<T> c = column4<T>(it, le, rf, col);
        uint32_t pl[2][9];
#pragma unroll
        for (int s = 0; s < 2; s++)
#pragma unroll
            for (int q = 0; q < 9; q++) pl[s][q] = 0u;
        auto add_votes = [&](int s, uint32_t m) {
#pragma unroll
            for (int q = 0; q < 9; q++) {
                const uint32_t cy = pl[s][q] & m;
                pl[s][q] ^= m;
                m = cy;
            }
        };
        for (int j = 0; j < na; j++) {
            const HitP<T> h = s_h[j];
            const HitI<T> wi = s_w[j];
            uint32_t b0 = 0, b1 = 0;
            for (int iz = 0; iz < nz; iz++) {
                const Pre4<T> pre = prefix4<T>(c.m, s_zc[iz], h);
                if (pre.guard) { b0 |= 1u << iz; b1 |= 1u << iz; continue; }
                const IV<T> A2 = a2_4<T>(c.X, c.Y, s_z[iz], wi);
                if (sign_only != 1 && pair4<T>(c.m, pre, 1, h, A2, c.Rv)) b0 |= 1u << iz;
                if (sign_only != 0 && pair4<T>(c.m, pre, -1, h, A2, c.Rv)) b1 |= 1u << iz;
            }
            add_votes(0, b0);
            add_votes(1, b1);
        }
        for (int s = 0; s < 2; s++) {
            if (sign_only >= 0 && s != sign_only) continue;
            for (int iz = 0; iz < nz; iz++) {
                int v = 0;
#pragma unroll
                for (int q = 0; q < 9; q++) v |= (int)((pl[s][q] >> iz) & 1u) << q;
                vo[(long long)s * it.nvox + col + it.ncol * iz] = v;
                mx[s] = v > mx[s] ? v : mx[s];
            }
        }
    }
    if (mx[0] > 0) atomicMax(&s_vmax[0], mx[0]);
    if (mx[1] > 0) atomicMax(&s_vmax[1], mx[1]);
    __syncthreads();
    if (tid < 2 && s_vmax[tid] > 0) atomicMax(&vmax[(long long)e * 2 + tid], s_vmax[tid]);
}

// Statistics of the maximum-vote voxels of the accumulator with the larger maximum (force
// >= 0: of that sign's accumulator).
__global__ void __launch_bounds__(256)
k4_stats(Iter4 it, int ev0, const int32_t *votes, const int32_t *vmax, Stats4 *st, int force) {
    __shared__ unsigned long long s_cnt, s_sum[4];
    __shared__ int s_mn[4], s_mx[4];
    const int el = blockIdx.y, e = ev0 + el, tid = threadIdx.x;
    if (tid == 0) {
        s_cnt = 0;
        for (int a = 0; a < 4; a++) { s_sum[a] = 0; s_mn[a] = 1 << 30; s_mx[a] = -1; }
    }
    __syncthreads();
    const int s = force >= 0 ? force : (vmax[(long long)e * 2] >= vmax[(long long)e * 2 + 1] ? 0 : 1);
    const int vm = vmax[(long long)e * 2 + s];
    const int32_t *vo = votes + ((long long)el * 2 + s) * it.nvox;
    unsigned long long cnt = 0, sum[4] = {0, 0, 0, 0};
    int mn[4] = {1 << 30, 1 << 30, 1 << 30, 1 << 30}, mx[4] = {-1, -1, -1, -1};
    for (long long j = (long long)blockIdx.x * blockDim.x + tid; j < it.nvox; j += (long long)gridDim.x * blockDim.x) {
        if (__ldcs(vo + j) != vm) continue;
        long long r = j;
        int idx[4];
        for (int a = 0; a < 4; a++) { idx[a] = (int)(r % it.n[a]); r /= it.n[a]; }
        cnt++;
        for (int a = 0; a < 4; a++) {
            sum[a] += (unsigned long long)idx[a];
            mn[a] = idx[a] < mn[a] ? idx[a] : mn[a];
            mx[a] = idx[a] > mx[a] ? idx[a] : mx[a];
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        cnt += __shfl_down_sync(0xffffffffu, cnt, o);
        for (int a = 0; a < 4; a++) {
            sum[a] += __shfl_down_sync(0xffffffffu, sum[a], o);
            const int a1 = __shfl_down_sync(0xffffffffu, mn[a], o), b1 = __shfl_down_sync(0xffffffffu, mx[a], o);
            mn[a] = a1 < mn[a] ? a1 : mn[a];
            mx[a] = b1 > mx[a] ? b1 : mx[a];
        }
    }
    if ((tid & 31) == 0 && cnt) {
        atomicAdd(&s_cnt, cnt);
        for (int a = 0; a < 4; a++) {
            atomicAdd(&s_sum[a], sum[a]);
            atomicMin(&s_mn[a], mn[a]);
            atomicMax(&s_mx[a], mx[a]);
        }
    }
    __syncthreads();
    if (tid == 0 && s_cnt) {
        Stats4 &g = st[e];
        atomicAdd(&g.cnt, s_cnt);
        for (int a = 0; a < 4; a++) {
            atomicAdd(&g.sum[a], s_sum[a]);
            atomicMin(&g.mn[a], s_mn[a]);
            atomicMax(&g.mx[a], s_mx[a]);
        }
    }
}

// Active-hit bits from one byte per hit (CSR order), restricted to the staged valid hits.
__global__ void k4_active_bytes(const int32_t *offsets, const int32_t *n_hits, const uint8_t *in,
                                uint32_t *active) {
    const int e = blockIdx.x, wd = threadIdx.x;
    if (wd >= 8) return;
    const int n = n_hits[e] < 0 ? 0 : n_hits[e], a0 = offsets[e];
    uint32_t m = 0u;
    for (int b = 0; b < 32; b++) {
        const int i = 32 * wd + b;
        if (i < n && in[a0 + i]) m |= 1u << b;
    }
    active[(long long)e * 8 + wd] &= m;
}

__global__ void k4_reset_stats(int n, Stats4 *st, int32_t *vmax) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    Stats4 &g = st[e];
    g.cnt = 0;
    for (int a = 0; a < 4; a++) { g.sum[a] = 0; g.mn[a] = 1 << 30; g.mx[a] = -1; }
    if (vmax) vmax[2 * e] = vmax[2 * e + 1] = 0;
}

// Iteration 1 state: the global corner and the origin as reference point.
__global__ void k4_init(int n, double g0, double g1, double g2, double g3, double *lo, double *ref) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    lo[4 * e + 0] = g0; lo[4 * e + 1] = g1; lo[4 * e + 2] = g2; lo[4 * e + 3] = g3;
    ref[2 * e] = ref[2 * e + 1] = 0.0;
}

// Estimate, hit finding, and the next iteration's reference point and grid corner.
// One block per event.  k: this iteration; nxt (null after the last): the next one's
// shape; glo: the global corner.  Per-sign iteration 3 (lo2 / ref2 / active2: sign-major
// state of ne events):
//   force = s >= 0 (after iteration 2): the estimate of sign s's accumulator (st holds its
//     statistics), its hit finding into active2, its next reference point and corner into
//     ref2 / lo2; no record, no selection;
//   force < 0 with lo2 set (iteration 3): this iteration's corner and reference point are
//     those of the chosen sign in lo2 / ref2.
template <typename T>
__global__ void __launch_bounds__(256)
k4_finish(Iter4 it, int k, int n_iter, bool has_next, Iter4 nxt, double g0, double g1, double g2, double g3,
          const int32_t *offsets, const int32_t *n_hits, const HitRecD *hd, const int32_t *vmax,
          const Stats4 *st, double *lo, double *ref, uint32_t *active, apo4_iter *out, uint8_t *selected,
          int force, int ne, double *lo2, double *ref2, uint32_t *active2) {
    __shared__ double s_val[4], s_err[4];
    __shared__ int s_sign, s_cnt;
    __shared__ uint32_t s_act[8];
    __shared__ apo4_iter s_rec;   // the record of a forced-sign pass (not stored)
    const int e = blockIdx.x, tid = threadIdx.x;
    const int nh_raw = n_hits[e];
    const int nh = nh_raw < 0 ? 0 : nh_raw;
    const int sc = force >= 0 ? force : (vmax[2 * e] >= vmax[2 * e + 1] ? 0 : 1);
    const long long es = (long long)sc * ne + e;   // sign-major index
    apo4_iter &o = force >= 0 ? s_rec : out[(long long)e * n_iter + k];
    const double *le = (force < 0 && lo2) ? lo2 + es * 4 : lo + (long long)e * 4;
    const double *rf = (force < 0 && lo2) ? ref2 + es * 2 : ref + (long long)e * 2;
    double *le_out = force >= 0 ? lo2 + es * 4 : lo + (long long)e * 4;
    double *rf_out = force >= 0 ? ref2 + es * 2 : ref + (long long)e * 2;
    uint32_t *act_out = force >= 0 ? active2 + es * 8 : active + (long long)e * 8;
    if (force >= 0) selected = nullptr;
    if (tid == 0) {
        const int s = sc;
        const Stats4 g = st[e];
        const double m = (double)g.cnt;
        for (int a = 0; a < 4; a++) {
            const double mu = __ddiv_rn((double)g.sum[a], m);
            s_val[a] = __dadd_rn(le[a], __dmul_rn(it.w[a], __dadd_rn(mu, 0.5)));
            s_err[a] = __dmul_rn(__dmul_rn(it.w[a], (double)(g.mx[a] + 1 - g.mn[a])), 0.5);
            o.value[a] = s_val[a];
            o.err[a] = s_err[a];
        }
        o.ref[0] = rf[0];
        o.ref[1] = rf[1];
        s_sign = s == 0 ? 1 : -1;
        o.sign = s_sign;
        o.vmax = nh_raw < 0 ? nh_raw : vmax[2 * e + s];
        o.n_max = (int)g.cnt;
        s_cnt = 0;
    }
    if (tid < 8) s_act[tid] = 0u;
    __syncthreads();
    // hit finding on value +- hit_factor * error, every hit of the event
    double blo[4], bhi[4], c[4];
    for (int a = 0; a < 4; a++) {
        const double r = __dmul_rn(it.hit_factor, s_err[a]);
        blo[a] = __dsub_rn(s_val[a], r);
        bhi[a] = __dadd_rn(s_val[a], r);
        c[a] = mid4(blo[a], bhi[a]);
    }
    const Ctr4<T> m = centre4<T>(rn<T>(c[0]), rn<T>(c[1]), rn<T>(c[2]), rn<T>(it.p_gev), rn<T>(it.b_tesla),
                                 rn<T>(rf[0]), rn<T>(rf[1]));
    const IV<T> X = box_iv<T>(blo[0], bhi[0]), Y = box_iv<T>(blo[1], bhi[1]), Rv = box_iv<T>(blo[2], bhi[2]);
    const IV<T> Z = box_iv<T>(blo[3], bhi[3]);
    const int a0 = offsets[e], nseg = offsets[e + 1] - a0;
    for (int i = tid; i < nh; i += blockDim.x) {
        const HitRecD r = hd[(long long)e * kHitCap + i];
        bool v = false;
        if (m.valid) {
            const HitP<T> h = hit_point<T>(r);
            const Pre4<T> pre = prefix4<T>(m, rn<T>(c[3]), h);
            v = pre.guard || pair4<T>(m, pre, s_sign, h, a2_4<T>(X, Y, Z, hit_iv<T>(r)), Rv);
        }
        if (v) {
            atomicOr(&s_act[i >> 5], 1u << (i & 31));
            atomicAdd(&s_cnt, 1);
        }
        if (selected && !has_next) selected[a0 + i] = v ? 1 : 0;
    }
    if (selected && !has_next && nh_raw < 0 && a0 >= 0 && nseg >= 0 && nseg <= kHitCap)
        for (int i = tid; i < nseg; i += blockDim.x) selected[a0 + i] = 0;
    __syncthreads();
    if (tid < 8) act_out[tid] = s_act[tid];
    if (tid != 0) return;
    o.n_sel = s_cnt;
    if (!has_next) return;
    // next reference point: the selected hit's waist point nearest to the found circle
    double r0 = rf[0], r1 = rf[1], best = __longlong_as_double(0x7ff0000000000000LL);   // +inf
    for (int i = 0; i < nh; i++) {
        if (!((s_act[i >> 5] >> (i & 31)) & 1u)) continue;
        const HitRecD &r = hd[(long long)e * kHitCap + i];
        const double dx = __dsub_rn(r.v[0], s_val[0]), dy = __dsub_rn(r.v[1], s_val[1]);
        const double dist = fabs(__dsub_rn(__dsqrt_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy))), s_val[2]));
        if (dist < best) { best = dist; r0 = r.v[0]; r1 = r.v[1]; }
    }
    if (k + 1 == 1) {
        le_out[0] = g0; le_out[1] = g1; le_out[2] = g2; le_out[3] = g3;
    } else {
        // z0 moved from the old reference point to the new one: z0 + tan(lambda) R dpsi,
        // dpsi the difference of their phases from the direction of the origin
        const double xc = s_val[0], yc = s_val[1], R = s_val[2];
        const double ox = -xc, oy = -yc;
        const double on = __dsqrt_rn(__dadd_rn(__dmul_rn(ox, ox), __dmul_rn(oy, oy)));
        bool bad = !(on > 0.0);
        const double ax = __dsub_rn(rf[0], xc), ay = __dsub_rn(rf[1], yc);
        const double bx = __dsub_rn(r0, xc), by = __dsub_rn(r1, yc);
        const double pa = bad ? 0.0 : phase4<double>(ox, oy, on, ax, ay,
                                                     __dsqrt_rn(__dadd_rn(__dmul_rn(ax, ax), __dmul_rn(ay, ay))), bad);
        const double pb = bad ? 0.0 : phase4<double>(ox, oy, on, bx, by,
                                                     __dsqrt_rn(__dadd_rn(__dmul_rn(bx, bx), __dmul_rn(by, by))), bad);
        const double dpsi = bad ? 0.0 : __dsub_rn(pb, pa);
        const double ratio = __ddiv_rn(it.p_gev, __dmul_rn(__dmul_rn(0.3, it.b_tesla), R));
        const double aL = ratio > 1.0 ? __dsqrt_rn(__dsub_rn(__dmul_rn(ratio, ratio), 1.0)) : 0.0;
        const double L = s_sign > 0 ? aL : -aL;
        const double c3 = __dadd_rn(s_val[3], __dmul_rn(L, __dmul_rn(R, dpsi)));
        const double cc[4] = {s_val[0], s_val[1], s_val[2], c3};
        for (int a = 0; a < 4; a++)
            le_out[a] = __dsub_rn(cc[a], __dmul_rn(__dmul_rn((double)nxt.n[a], nxt.w[a]), 0.5));
    }
    rf_out[0] = r0;
    rf_out[1] = r1;
}

}  // namespace apo

namespace {

template <typename T>
void launch_vote4(const Iter4 &it, int ev0, int n, const int32_t *nh, const HitRecD *hd,
                  const uint32_t *active, const double *lo, const double *ref, int32_t *votes,
                  int32_t *vmax, cudaStream_t s, int sign_only = -1) {
    dim3 grid((unsigned)((it.ncol + kTile4 - 1) / kTile4), n);
    k4_vote<T><<<grid, 128, 0, s>>>(it, ev0, nh, hd, active, lo, ref, votes, vmax, sign_only);
}

void launch_stats4(const Iter4 &it, int ev0, int n, const int32_t *votes, const int32_t *vmax,
                   Stats4 *st, cudaStream_t s, int force = -1) {
    long long b = (it.nvox + 256LL * 8 - 1) / (256LL * 8);
    dim3 grid((unsigned)(b < 1 ? 1 : (b > 1024 ? 1024 : b)), n);
    k4_stats<<<grid, 256, 0, s>>>(it, ev0, votes, vmax, st, force);
}

template <typename T>
void launch_finish4(const Iter4 &it, int k, const apo4_opts *o, bool has_next, const Iter4 &nxt,
                    const apo_hits *hits, const int32_t *nh, const HitRecD *hd, const int32_t *vmax,
                    const Stats4 *st, double *lo, double *ref, uint32_t *active, apo4_iter *out,
                    uint8_t *selected, int force, int ne, double *lo2, double *ref2, uint32_t *active2,
                    cudaStream_t s) {
    k4_finish<T><<<ne, 256, 0, s>>>(it, k, o->n_iter, has_next, nxt, o->glo[0], o->glo[1], o->glo[2], o->glo[3],
                                    hits->offsets, nh, hd, vmax, st, lo, ref, active, out, selected, force, ne,
                                    lo2, ref2, active2);
}

int check_hits4(const apo_hits *h) {
    if (!h) return fail4(APO_EINVAL, "hits is NULL");
    if (h->n_events < 0) return fail4(APO_EINVAL, "n_events < 0");
    if (h->n_events > 0 && (!h->offsets || !h->wire_id || !h->drift))
        return fail4(APO_EINVAL, "hits arrays must be non-NULL");
    return APO_OK;
}

int check_chamber(const apo4_chamber *c) {
    if (!c) return fail4(APO_EINVAL, "chamber is NULL");
    int dev = -1;
    CU4(cudaGetDevice(&dev));
    if (dev != c->device) return fail4(APO_EINVAL, "chamber lives on device %d, current is %d", c->device, dev);
    return APO_OK;
}

int check_ws4(const apo4_opts *o, int ne, void *ws, size_t bytes, Layout4 &L) {
    L = layout4(o, ne);
    if (!ws) return fail4(APO_EINVAL, "workspace is NULL");
    if (reinterpret_cast<uintptr_t>(ws) % 256) return fail4(APO_EINVAL, "workspace must be 256-byte aligned");
    if (bytes < L.end) return fail4(APO_ENOMEM, "workspace too small: %zu < %zu bytes", bytes, L.end);
    return APO_OK;
}

template <typename P> P *at4(void *ws, size_t off) { return reinterpret_cast<P *>(static_cast<unsigned char *>(ws) + off); }

}  // namespace

extern "C" {

void apo4_opts_default(apo4_opts *o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->p_gev = 0.105;
    o->b_tesla = 1.0;
    o->disk_radius = 0.10;
    o->hit_factor = 5.0;
    const double glo[4] = {-0.45, -0.45, 0.225, -0.75};
    const double w[3][4] = {{0.018, 0.018, 0.00375, 0.075}, {0.010, 0.010, 0.00375, 0.075},
                            {0.001, 0.001, 0.001, 0.040}};
    const int n[3][4] = {{50, 50, 40, 20}, {90, 90, 40, 20}, {50, 50, 50, 20}};
    for (int a = 0; a < 4; a++) o->glo[a] = glo[a];
    for (int k = 0; k < 3; k++)
        for (int a = 0; a < 4; a++) { o->w[k][a] = w[k][a]; o->n[k][a] = n[k][a]; }
    o->precision = APO_F64;
    o->n_iter = 3;
    o->per_sign = 1;
}

int apo4_chamber_create(const apo_wires *w, apo4_chamber **out) {
    if (!out) return fail4(APO_EINVAL, "out is NULL");
    *out = nullptr;
    if (!w || w->n_wires <= 0) return fail4(APO_EINVAL, "wires missing");
    const double *wa[8] = {w->x0, w->y0, w->sin_phis, w->cos_phis, w->tan_tau, w->sphi_t, w->cphi_t, w->t2};
    for (int i = 0; i < 8; i++)
        if (!wa[i]) return fail4(APO_EINVAL, "wire array %d is NULL", i);
    apo4_chamber *c = new apo4_chamber();
    std::memset(&c->dg, 0, sizeof(c->dg));
    CU4(cudaGetDevice(&c->device));
    c->dg.n_wires = w->n_wires;
    for (int i = 0; i < 8; i++) {
        void *p = nullptr;
        cudaError_t e = cudaMalloc(&p, sizeof(double) * (size_t)w->n_wires);
        if (e == cudaSuccess) {
            c->allocs.push_back(p);
            e = cudaMemcpy(p, wa[i], sizeof(double) * (size_t)w->n_wires, cudaMemcpyHostToDevice);
        }
        if (e != cudaSuccess) {
            apo4_chamber_destroy(c);
            return fail4(APO_ECUDA, "wire upload: %s", cudaGetErrorString(e));
        }
        c->dg.wire[i] = static_cast<const double *>(p);
    }
    *out = c;
    return APO_OK;
}

void apo4_chamber_destroy(apo4_chamber *c) {
    if (!c) return;
    for (void *p : c->allocs) cudaFree(p);
    delete c;
}

int apo4_workspace_bytes(const apo4_chamber *c, int32_t n_events, const apo4_opts *o, size_t *bytes) {
    int rc;
    if (!c || !bytes) return fail4(APO_EINVAL, "NULL argument");
    if ((rc = check_opts(o))) return rc;
    if (n_events < 0) return fail4(APO_EINVAL, "n_events < 0");
    *bytes = layout4(o, n_events).end;
    return APO_OK;
}

int apo4_solve_batch(const apo4_chamber *c, const apo_hits *hits, const apo4_opts *o, apo4_iter *out,
                     uint8_t *selected, void *ws, size_t ws_bytes, void *stream) {
    int rc;
    if ((rc = check_chamber(c)) || (rc = check_hits4(hits)) || (rc = check_opts(o))) return rc;
    const int ne = hits->n_events;
    if (ne > 0 && !out) return fail4(APO_EINVAL, "out is NULL");
    Layout4 L;
    if ((rc = check_ws4(o, ne, ws, ws_bytes, L))) return rc;
    if (ne == 0) return APO_OK;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    unsigned *status = at4<unsigned>(ws, L.status);
    int32_t *nh = at4<int32_t>(ws, L.nh);
    HitRecD *hd = at4<HitRecD>(ws, L.hd);
    HitRecF *hf = at4<HitRecF>(ws, L.hf);
    uint32_t *active = at4<uint32_t>(ws, L.active);
    int32_t *done = at4<int32_t>(ws, L.done);
    double *lo = at4<double>(ws, L.lo);
    double *ref = at4<double>(ws, L.ref);
    int32_t *vmax = at4<int32_t>(ws, L.vmax);
    Stats4 *st = at4<Stats4>(ws, L.stats);
    double *lo2 = at4<double>(ws, L.lo2);
    double *ref2 = at4<double>(ws, L.ref2);
    uint32_t *active2 = at4<uint32_t>(ws, L.active2);
    Stats4 *st2 = at4<Stats4>(ws, L.stats2);
    int32_t *votes = at4<int32_t>(ws, L.votes);
    // per-sign iteration 3: after iteration 2 each sign's accumulator gets its own estimate,
    // hit finding, reference point and box; iteration 3 votes sign s on box s
    const bool ps = o->per_sign && o->n_iter == 3;
    const bool f32 = o->precision == APO_F32;
    CU4(cudaMemsetAsync(status, 0, 256, s));
    launch_stage(c->dg, ne, hits->offsets, hits->wire_id, hits->drift, hd, hf, nh, active, done, status, s);
    k4_init<<<(ne + 127) / 128, 128, 0, s>>>(ne, o->glo[0], o->glo[1], o->glo[2], o->glo[3], lo, ref);
    CU4(cudaGetLastError());
    for (int k = 0; k < o->n_iter; k++) {
        const Iter4 it = iter4(o, k);
        const bool has_next = k + 1 < o->n_iter;
        const Iter4 nxt = has_next ? iter4(o, k + 1) : it;
        const bool split_stats = ps && k == 1, split_vote = ps && k == 2;
        k4_reset_stats<<<(ne + 127) / 128, 128, 0, s>>>(ne, st, vmax);
        if (split_stats) k4_reset_stats<<<(2 * ne + 127) / 128, 128, 0, s>>>(2 * ne, st2, nullptr);
        for (int e0 = 0; e0 < ne; e0 += L.chunk) {
            const int n = ne - e0 < L.chunk ? ne - e0 : L.chunk;
            for (int sg = split_vote ? 0 : -1; sg < (split_vote ? 2 : 0); sg++) {
                const uint32_t *ac = sg < 0 ? active : active2 + (size_t)sg * ne * 8;
                const double *lc = sg < 0 ? lo : lo2 + (size_t)sg * ne * 4;
                const double *rc = sg < 0 ? ref : ref2 + (size_t)sg * ne * 2;
                if (f32) launch_vote4<float>(it, e0, n, nh, hd, ac, lc, rc, votes, vmax, s, sg);
                else launch_vote4<double>(it, e0, n, nh, hd, ac, lc, rc, votes, vmax, s, sg);
            }
            launch_stats4(it, e0, n, votes, vmax, st, s);
            if (split_stats)
                for (int sg = 0; sg < 2; sg++) launch_stats4(it, e0, n, votes, vmax, st2 + (size_t)sg * ne, s, sg);
        }
        if (split_stats)   // before the chosen sign's pass, which moves lo / ref on
            for (int sg = 0; sg < 2; sg++) {
                if (f32)
                    launch_finish4<float>(it, k, o, has_next, nxt, hits, nh, hd, vmax, st2 + (size_t)sg * ne, lo, ref,
                                          active, out, nullptr, sg, ne, lo2, ref2, active2, s);
                else
                    launch_finish4<double>(it, k, o, has_next, nxt, hits, nh, hd, vmax, st2 + (size_t)sg * ne, lo,
                                           ref, active, out, nullptr, sg, ne, lo2, ref2, active2, s);
            }
        if (f32)
            launch_finish4<float>(it, k, o, has_next, nxt, hits, nh, hd, vmax, st, lo, ref, active, out, selected, -1,
                                  ne, split_vote ? lo2 : nullptr, split_vote ? ref2 : nullptr, active2, s);
        else
            launch_finish4<double>(it, k, o, has_next, nxt, hits, nh, hd, vmax, st, lo, ref, active, out, selected,
                                   -1, ne, split_vote ? lo2 : nullptr, split_vote ? ref2 : nullptr, active2, s);
        CU4(cudaGetLastError());
    }
    return APO_OK;
}

int apo4_vote(const apo4_chamber *c, const apo_hits *hits, const apo4_opts *o, int32_t iter, const double *lo,
              const double *ref, const uint8_t *active_in, int32_t *votes_out, void *ws, size_t ws_bytes,
              void *stream) {
    int rc;
    if ((rc = check_chamber(c)) || (rc = check_hits4(hits)) || (rc = check_opts(o))) return rc;
    if (iter < 0 || iter >= o->n_iter) return fail4(APO_EINVAL, "iter out of range");
    const int ne = hits->n_events;
    if (ne > 0 && (!lo || !ref || !votes_out)) return fail4(APO_EINVAL, "lo, ref and votes must be non-NULL");
    Layout4 L;
    if ((rc = check_ws4(o, ne, ws, ws_bytes, L))) return rc;
    if (ne == 0) return APO_OK;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    unsigned *status = at4<unsigned>(ws, L.status);
    int32_t *nh = at4<int32_t>(ws, L.nh);
    HitRecD *hd = at4<HitRecD>(ws, L.hd);
    HitRecF *hf = at4<HitRecF>(ws, L.hf);
    uint32_t *active = at4<uint32_t>(ws, L.active);
    int32_t *done = at4<int32_t>(ws, L.done);
    int32_t *vmax = at4<int32_t>(ws, L.vmax);
    Stats4 *st = at4<Stats4>(ws, L.stats);
    CU4(cudaMemsetAsync(status, 0, 256, s));
    launch_stage(c->dg, ne, hits->offsets, hits->wire_id, hits->drift, hd, hf, nh, active, done, status, s);
    if (active_in) k4_active_bytes<<<ne, 32, 0, s>>>(hits->offsets, nh, active_in, active);
    k4_reset_stats<<<(ne + 127) / 128, 128, 0, s>>>(ne, st, vmax);
    const Iter4 it = iter4(o, iter);
    // the caller's array holds every event: vote all of them in one launch
    if (o->precision == APO_F32) launch_vote4<float>(it, 0, ne, nh, hd, active, lo, ref, votes_out, vmax, s);
    else launch_vote4<double>(it, 0, ne, nh, hd, active, lo, ref, votes_out, vmax, s);
    CU4(cudaGetLastError());
    return APO_OK;
}

}  // extern "C"
