// Host side of the C ABI declared in include/apo.h: geometry upload, workspace layout and
// the coarse-to-fine pipeline (arXiv:2401.04576, Sections 3.1 and 3.3) queued on the
// caller's stream.
#include <cuda_runtime.h>

#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/apo.h"
#include "../../include/apo_diag.h"
#include "kernels.cuh"

using namespace apo;

namespace {

thread_local char g_err[512] = "";

int fail(int code, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return code;
}

#define CU(call)                                                                        \
    do {                                                                                \
        cudaError_t e_ = (call);                                                        \
        if (e_ != cudaSuccess)                                                          \
            return fail(APO_ECUDA, "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, \
                        __LINE__);                                                      \
    } while (0)

int check_launch(const char *what) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(APO_ECUDA, "%s launch: %s", what, cudaGetErrorString(e));
    return APO_OK;
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace

// A recorded search: replayed when apo_solve_batch is called again with the same key.
struct GraphEntry {
    unsigned char key[256];
    size_t key_len;
    cudaGraphExec_t exec;
};

struct apo_geometry {
    DevGeom dg;
    int device;
    long long n_coarse;
    int persist_blocks = 0;              // blocks of the persistent launch (all resident)
    std::vector<void *> allocs;
    std::mutex graph_mu;                 // guards the two members below
    std::vector<GraphEntry> graphs;
    cudaStream_t capture_stream = nullptr;
};

namespace {

// Workspace regions for a batch of n_events.
struct Layout {
    size_t status, n_hits, hd, hf, votes, hist, fk, fv, ck, cv, mask, done, ntr, tune_tracks;
    size_t ms_front, ms_count, ms_stop, ms_ck, ms_cv, ms_ts, ms_tcnt, p_votes, p_hist, p_next, cand_k, cand_v,
        end;
    int chunk, ms_chunk;
};

// Events per chunk of the max-set schedule: its children arrays hold max_keep x 32 cells per
// event; a chunk keeps them within 2 GiB (and within the level-0 chunk).
int maxset_chunk(const Layout &L, int max_keep) {
    long long per = (long long)max_keep * 32 * (sizeof(uint64_t) + sizeof(int32_t));
    long long c = (2LL << 30) / (per > 0 ? per : 1);
    if (c < 1) c = 1;
    if (c > L.chunk) c = L.chunk;
    return (int)c;
}

Layout layout(const apo_geometry *g, int n_events, const apo_solve_opts *opts = nullptr) {
    Layout L;
    const int K = g->dg.topk;
    long long chunk = (1LL << 28) / (g->n_coarse > 0 ? g->n_coarse : 1);
    if (chunk < 1) chunk = 1;
    if (chunk > n_events) chunk = n_events > 0 ? n_events : 1;
    L.chunk = (int)chunk;
    size_t o = 0;
    L.status = o; o += 256;
    L.n_hits = o; o = align256(o + sizeof(int32_t) * (size_t)n_events);
    L.hd = o; o = align256(o + sizeof(HitRecD) * (size_t)n_events * kHitCap);
    L.hf = o; o = align256(o + sizeof(HitRecF) * (size_t)n_events * kHitCap);
    // level 0 keeps every cell's vote only for the max-set schedule and the midpoint form;
    // otherwise each coarse block keeps its K best cells (candidates).  Without options the
    // layout holds both, so it serves any options.
    const bool maxset = opts && opts->schedule == APO_SCHED_MAXSET;
    const bool full_votes = !opts || maxset || (opts->precision[0] & ~APO_OUTGOING) == APO_F64_MID ||
                            opts->tune.coarse_full;
    L.votes = o; o = align256(o + (full_votes ? sizeof(int32_t) * (size_t)chunk * (size_t)g->n_coarse : 0));
    const size_t n_lists = (size_t)g->dg.bins[1] * g->dg.bins[2] * 2;   // the larger split
    L.cand_k = o; o = align256(o + (maxset ? 0 : sizeof(uint64_t) * (size_t)chunk * n_lists * K));
    L.cand_v = o; o = align256(o + (maxset ? 0 : sizeof(int32_t) * (size_t)chunk * n_lists * K));
    L.hist = o; o = align256(o + sizeof(uint32_t) * (size_t)chunk * kHistBins);
    L.fk = o; o = align256(o + sizeof(uint64_t) * (size_t)n_events * K);
    L.fv = o; o = align256(o + sizeof(int32_t) * (size_t)n_events * K);
    L.ck = o; o = align256(o + sizeof(uint64_t) * (size_t)n_events * K * 32);
    L.cv = o; o = align256(o + sizeof(int32_t) * (size_t)n_events * K * 32);
    L.mask = o; o = align256(o + sizeof(uint32_t) * (size_t)n_events * (kHitCap / 32));
    L.done = o; o = align256(o + sizeof(int32_t) * (size_t)n_events);
    L.ntr = o; o = align256(o + sizeof(int32_t) * (size_t)n_events);
    L.tune_tracks = o; o = align256(o + sizeof(apo_track) * (size_t)n_events * APO_MAX_TRACKS);
    L.ms_chunk = 0;
    L.ms_front = L.ms_count = L.ms_stop = L.ms_ck = L.ms_cv = L.ms_ts = L.ms_tcnt = o;
    L.p_votes = L.p_hist = L.p_next = o;
    if (opts && opts->schedule == APO_SCHED_TOPK && opts->tune.persistent) {
        const size_t B = (size_t)(g->persist_blocks > 0 ? g->persist_blocks : 1);
        L.p_votes = o; o = align256(o + sizeof(int32_t) * B * (size_t)g->n_coarse);
        L.p_hist = o; o = align256(o + sizeof(uint32_t) * B * kHistBins);
        L.p_next = o; o = align256(o + sizeof(int32_t));
    }
    if (opts && opts->schedule == APO_SCHED_MAXSET && opts->max_keep > 0) {
        const size_t K = (size_t)opts->max_keep;
        const int c = maxset_chunk(L, opts->max_keep);
        L.ms_chunk = c;
        L.ms_front = o; o = align256(o + sizeof(uint64_t) * (size_t)c * K);
        L.ms_count = o; o = align256(o + sizeof(int32_t) * (size_t)c);
        L.ms_stop = o; o = align256(o + sizeof(int32_t) * (size_t)c);
        L.ms_ck = o; o = align256(o + sizeof(uint64_t) * (size_t)c * K * 32);
        L.ms_cv = o; o = align256(o + sizeof(int32_t) * (size_t)c * K * 32);
        if (opts->max_tracks > 1) {   // the multi-track rounds' track step
            L.ms_ts = o; o = align256(o + sizeof(TrackStep) * (size_t)c);
            L.ms_tcnt = o; o = align256(o + maxset_smem_bytes(g->dg) * (size_t)c);
        }
    }
    L.end = o;
    return L;
}

template <typename P> P *at(void *ws, size_t off) {
    return reinterpret_cast<P *>(static_cast<unsigned char *>(ws) + off);
}

// A level precision the geometry can evaluate.
int check_precision(const apo_geometry *g, int p_code, const char *what) {
    const int p = p_code & ~APO_OUTGOING;
    if ((p_code & ~(APO_OUTGOING | 7)) != 0 ||
        (p != APO_F64 && p != APO_F32 && p != APO_F64_FILTERED && p != APO_F64_MID && p != APO_F64_EXACT))
        return fail(APO_EINVAL, "bad %s", what);
    if (p == APO_F64_MID && (p_code & APO_OUTGOING))
        return fail(APO_EINVAL, "APO_OUTGOING does not apply to APO_F64_MID");
    if (p == APO_F64_MID && !g->dg.sincos_mid)
        return fail(APO_EINVAL, "APO_F64_MID needs the grid's sincos_mid table");
    return APO_OK;
}

// The device tables for one precision code: the geometry's, with the direction flag set.
DevGeom geom_for(const apo_geometry *g, int p_code) {
    DevGeom d = g->dg;
    d.k.outgoing = (p_code & APO_OUTGOING) ? 1 : 0;
    return d;
}

int key_bits_total(const DevGeom &d) {
    int t = 0;
    for (int a = 0; a < 5; a++) t += d.key_bits[a];
    return t;
}

int check_geom(const apo_geometry *g) {
    if (!g) return fail(APO_EINVAL, "geometry is NULL");
    int dev = -1;
    CU(cudaGetDevice(&dev));
    if (dev != g->device)
        return fail(APO_EINVAL, "geometry lives on device %d, current device is %d", g->device, dev);
    return APO_OK;
}

int check_hits(const apo_hits *h) {
    if (!h) return fail(APO_EINVAL, "hits is NULL");
    if (h->n_events < 0) return fail(APO_EINVAL, "n_events < 0");
    if (h->n_events > 0 && (!h->offsets || !h->wire_id || !h->drift))
        return fail(APO_EINVAL, "hits arrays must be non-NULL");
    return APO_OK;
}

int check_ws(const apo_geometry *g, int n_events, void *ws, size_t bytes, Layout &L,
             const apo_solve_opts *opts = nullptr) {
    L = layout(g, n_events, opts);
    if (!ws) return fail(APO_EINVAL, "workspace is NULL");
    if (reinterpret_cast<uintptr_t>(ws) % 256)
        return fail(APO_EINVAL, "workspace must be 256-byte aligned");
    if (bytes < L.end)
        return fail(APO_ENOMEM, "workspace too small: %zu < %zu bytes", bytes, L.end);
    return APO_OK;
}

}  // namespace

namespace apo {
const DevGeom *geometry_device_tables(const apo_geometry *g, int *device) {
    if (device) *device = g ? g->device : -1;
    return g ? &g->dg : nullptr;
}
void set_last_error(const char *msg) { std::snprintf(g_err, sizeof(g_err), "%s", msg); }
}  // namespace apo

extern "C" {

const char *apo_last_error(void) { return g_err; }

void apo_solve_opts_default(apo_solve_opts *o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    for (int i = 0; i <= APO_MAX_LEVELS; i++) o->precision[i] = APO_F64;
    o->max_tracks = 1;
    o->min_votes = 0;
    o->mask_sigma = 150e-6;
    o->tune.cells_filter = 1;   // measured faster on bisected cells, identical votes
    o->schedule = APO_SCHED_TOPK;
    o->max_keep = 32768;
    o->slack = 0;
}

int apo_geometry_create(const apo_wires *w, const apo_grid *gr, apo_geometry **out) {
    if (!out) return fail(APO_EINVAL, "out is NULL");
    *out = nullptr;
    if (!w || !gr) return fail(APO_EINVAL, "wires / grid is NULL");
    if (w->n_wires <= 0) return fail(APO_EINVAL, "n_wires must be > 0");
    const double *wa[8] = {w->x0, w->y0, w->sin_phis, w->cos_phis, w->tan_tau, w->sphi_t, w->cphi_t, w->t2};
    for (int i = 0; i < 8; i++)
        if (!wa[i]) return fail(APO_EINVAL, "wire array %d is NULL", i);
    if (gr->levels < 0 || gr->levels > APO_MAX_LEVELS) return fail(APO_EINVAL, "levels out of range");
    if (gr->topk < 1 || gr->topk * 32 > 4096) return fail(APO_EINVAL, "topk must be in [1, 128]");
    long long n0 = 1;
    int kbits[5], kshift[5], ktot = 0;
    for (int a = 0; a < 5; a++) {
        if (gr->bins[a] < 1 || ((long long)gr->bins[a] << gr->levels) > 65536)
            return fail(APO_EINVAL, "bins[%d] << levels must be in [1, 65536]", a);
        if (!gr->lo_edge[a] || !gr->hi_edge[a]) return fail(APO_EINVAL, "edge table %d is NULL", a);
        n0 *= gr->bins[a];
        int b = 10;
        while ((1LL << b) < ((long long)gr->bins[a] << gr->levels)) b++;
        kbits[a] = b;
        kshift[a] = ktot;
        ktot += b;
    }
    if (ktot > 64) return fail(APO_EINVAL, "cell keys need %d > 64 bits", ktot);
    if (!gr->sincos) return fail(APO_EINVAL, "sincos table is NULL");
    if (gr->bins[0] * gr->bins[3] > 256)
        return fail(APO_EINVAL, "bins[0] * bins[3] must be <= 256 (one thread each in a block)");
    if (gr->bins[4] > 32) return fail(APO_EINVAL, "bins[4] must be <= 32 (one bit each in a vote mask)");
    if (n0 < gr->topk) return fail(APO_EINVAL, "fewer level-0 cells than topk");
    // omega cells must not contain 0
    {
        int nf = gr->bins[2] << gr->levels;
        for (int i = 0; i < nf; i++)
            if (!(gr->hi_edge[2][i] < 0.0 || gr->lo_edge[2][i] > 0.0))
                return fail(APO_EINVAL, "omega cell %d contains 0", i);
    }
    int dev = 0;
    CU(cudaGetDevice(&dev));
    init_kernel_attributes();
    init_maxset_attributes();
    apo_geometry *g = new apo_geometry();
    g->device = dev;
    g->n_coarse = n0;
    DevGeom &d = g->dg;
    std::memset(&d, 0, sizeof(d));
    for (int a = 0; a < 5; a++) d.bins[a] = gr->bins[a];
    d.levels = gr->levels;
    d.topk = gr->topk;
    d.n_wires = w->n_wires;
    for (int a = 0; a < 5; a++) { d.key_bits[a] = kbits[a]; d.key_shift[a] = kshift[a]; }
    auto upload = [&](const double *src, size_t n, const double **dst) -> int {
        void *p = nullptr;
        cudaError_t e = cudaMalloc(&p, n * sizeof(double));
        if (e != cudaSuccess) return fail(APO_ECUDA, "cudaMalloc: %s", cudaGetErrorString(e));
        g->allocs.push_back(p);
        e = cudaMemcpy(p, src, n * sizeof(double), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return fail(APO_ECUDA, "cudaMemcpy: %s", cudaGetErrorString(e));
        *dst = static_cast<const double *>(p);
        return APO_OK;
    };
    int rc = APO_OK;
    for (int i = 0; i < 8 && rc == APO_OK; i++) rc = upload(wa[i], (size_t)w->n_wires, &d.wire[i]);
    for (int a = 0; a < 5 && rc == APO_OK; a++) {
        size_t nf = (size_t)gr->bins[a] << gr->levels;
        rc = upload(gr->lo_edge[a], nf, &d.lo_edge[a]);
        if (rc == APO_OK) rc = upload(gr->hi_edge[a], nf, &d.hi_edge[a]);
    }
    long long rows = 0;
    for (int L = 0; L <= gr->levels; L++) {
        d.sincos_off[L] = rows;
        rows += (long long)gr->bins[1] << L;
    }
    if (rc == APO_OK) rc = upload(gr->sincos, (size_t)rows * 4, &d.sincos);
    if (rc == APO_OK && gr->sincos_mid) rc = upload(gr->sincos_mid, (size_t)rows * 2, &d.sincos_mid);
    if (rc == APO_OK) {
        SeriesConsts *dk = nullptr;
        cudaError_t e = cudaMalloc(&dk, sizeof(SeriesConsts));
        if (e == cudaSuccess) {
            launch_series_consts(dk, 0);
            e = cudaGetLastError();
            if (e == cudaSuccess) e = cudaMemcpy(&d.k, dk, sizeof(SeriesConsts), cudaMemcpyDeviceToHost);
            d.k.outgoing = 0;
            g->persist_blocks = persist_blocks(d);
            cudaFree(dk);
        }
        if (e != cudaSuccess) rc = fail(APO_ECUDA, "series constants: %s", cudaGetErrorString(e));
    }
    if (rc != APO_OK) {
        apo_geometry_destroy(g);
        return rc;
    }
    *out = g;
    return APO_OK;
}

void apo_geometry_destroy(apo_geometry *g) {
    if (!g) return;
    for (GraphEntry &e : g->graphs) cudaGraphExecDestroy(e.exec);
    if (g->capture_stream) cudaStreamDestroy(g->capture_stream);
    for (void *p : g->allocs) cudaFree(p);
    delete g;
}

int64_t apo_coarse_cells(const apo_geometry *g) { return g ? g->n_coarse : 0; }

int apo_workspace_bytes(const apo_geometry *g, int32_t n_events, const apo_solve_opts *opts, size_t *bytes) {
    if (!g || !bytes) return fail(APO_EINVAL, "NULL argument");
    if (n_events < 0) return fail(APO_EINVAL, "n_events < 0");
    *bytes = layout(g, n_events, opts).end;
    return APO_OK;
}

size_t apo_host_extra_bytes(int32_t n_events, int64_t n_hits) {
    return align256(sizeof(int32_t) * (size_t)(n_events + 1)) + align256(sizeof(int32_t) * (size_t)n_hits) +
           align256(sizeof(double) * (size_t)n_hits) + align256(sizeof(apo_track) * (size_t)n_events * APO_MAX_TRACKS) +
           align256(sizeof(int32_t) * (size_t)n_events) + 256;
}

int apo_vote(const apo_geometry *g, const apo_hits *hits, const uint64_t *cell_keys,
             int64_t n_cells_per_event, int32_t level, int32_t precision, int32_t *votes_out,
             void *ws, size_t ws_bytes, void *stream) {
    int rc;
    if ((rc = check_geom(g)) || (rc = check_hits(hits))) return rc;
    if ((rc = check_precision(g, precision, "precision"))) return rc;
    if (level < 0 || level > g->dg.levels) return fail(APO_EINVAL, "level out of range");
    if (!votes_out) return fail(APO_EINVAL, "votes_out is NULL");
    if (!cell_keys && (level != 0 || n_cells_per_event != g->n_coarse))
        return fail(APO_EINVAL, "full-grid voting needs level 0 and n_cells = apo_coarse_cells");
    if (n_cells_per_event < 0) return fail(APO_EINVAL, "n_cells < 0");
    Layout L;
    if ((rc = check_ws(g, hits->n_events, ws, ws_bytes, L))) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int ne = hits->n_events;
    if (ne == 0 || n_cells_per_event == 0) return APO_OK;
    unsigned *status = at<unsigned>(ws, L.status);
    int32_t *nh = at<int32_t>(ws, L.n_hits);
    HitRecD *hd = at<HitRecD>(ws, L.hd);
    HitRecF *hf = at<HitRecF>(ws, L.hf);
    CU(cudaMemsetAsync(status, 0, 256, s));
    launch_stage(g->dg, ne, hits->offsets, hits->wire_id, hits->drift, hd, hf, nh,
                 at<uint32_t>(ws, L.mask), at<int32_t>(ws, L.done), status, s);
    if ((rc = check_launch("stage"))) return rc;
    const DevGeom dg = geom_for(g, precision);
    const int prec = precision & ~APO_OUTGOING;
    if (!cell_keys) {
        uint32_t *hist = at<uint32_t>(ws, L.hist);
        for (int e0 = 0; e0 < ne; e0 += L.chunk) {
            int n = ne - e0 < L.chunk ? ne - e0 : L.chunk;
            CU(cudaMemsetAsync(hist, 0, sizeof(uint32_t) * (size_t)n * kHistBins, s));
            launch_vote_coarse(dg, prec, e0, n, hd, hf, nh, votes_out + (size_t)e0 * g->n_coarse,
                               hist, status, s);
            if ((rc = check_launch("vote_coarse"))) return rc;
        }
    } else {
        launch_vote_keys(dg, prec, ne, hd, hf, nh, level, cell_keys, n_cells_per_event,
                         votes_out, s);
        if ((rc = check_launch("vote_keys"))) return rc;
    }
    return APO_OK;
}

int apo_refine(const apo_geometry *g, const apo_hits *hits, const uint64_t *keys_in,
               const int32_t *votes_in, int64_t n_in, int32_t level, uint64_t *kept_keys,
               int32_t *kept_votes, uint64_t *children_out, void *ws, size_t ws_bytes, void *stream) {
    int rc;
    if ((rc = check_geom(g)) || (rc = check_hits(hits))) return rc;
    if (level < 0 || level >= g->dg.levels) return fail(APO_EINVAL, "level must be in [0, levels)");
    if (!votes_in || !children_out) return fail(APO_EINVAL, "votes_in / children_out is NULL");
    if (!keys_in && (level != 0 || n_in != g->n_coarse))
        return fail(APO_EINVAL, "implicit keys need level 0 and n_in = apo_coarse_cells");
    if (keys_in && (n_in < 1 || n_in > 4096)) return fail(APO_EINVAL, "n_in must be in [1, 4096]");
    if (key_bits_total(g->dg) > 50) return fail(APO_EINVAL, "top-K selection needs keys of at most 50 bits");
    Layout L;
    if ((rc = check_ws(g, hits->n_events, ws, ws_bytes, L))) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int ne = hits->n_events, K = g->dg.topk;
    if (ne == 0) return APO_OK;
    uint64_t *fk = at<uint64_t>(ws, L.fk);
    int32_t *fv = at<int32_t>(ws, L.fv);
    if (!keys_in) {
        uint32_t *hist = at<uint32_t>(ws, L.hist);
        for (int e0 = 0; e0 < ne; e0 += L.chunk) {
            int n = ne - e0 < L.chunk ? ne - e0 : L.chunk;
            CU(cudaMemsetAsync(hist, 0, sizeof(uint32_t) * (size_t)n * kHistBins, s));
            launch_hist(n, votes_in + (size_t)e0 * g->n_coarse, g->n_coarse, hist, s);
            launch_select_coarse(g->dg, e0, n, votes_in + (size_t)e0 * g->n_coarse, hist, K, fk, fv, s);
            if ((rc = check_launch("select_coarse"))) return rc;
        }
    } else {
        launch_topk(ne, keys_in, votes_in, (int)n_in, K, fk, fv, s);
        if ((rc = check_launch("topk"))) return rc;
    }
    if (kept_keys) CU(cudaMemcpyAsync(kept_keys, fk, sizeof(uint64_t) * (size_t)ne * K, cudaMemcpyDeviceToDevice, s));
    if (kept_votes) CU(cudaMemcpyAsync(kept_votes, fv, sizeof(int32_t) * (size_t)ne * K, cudaMemcpyDeviceToDevice, s));
    launch_children(g->dg, fk, (long long)ne * K, children_out, s);
    return check_launch("children");
}

static int trace_copy(const apo_solve_opts *o, const apo_geometry *g, int e0, int n, int level,
                      const uint64_t *keys, const int32_t *votes, cudaStream_t s) {
    if (!o->trace_keys && !o->trace_votes) return APO_OK;
    const int K = g->dg.topk, lv = g->dg.levels;
    if (o->trace_keys)
        CU(cudaMemcpy2DAsync(o->trace_keys + ((size_t)e0 * (lv + 1) + level) * K, sizeof(uint64_t) * K * (lv + 1),
                             keys, sizeof(uint64_t) * K, sizeof(uint64_t) * K, n, cudaMemcpyDeviceToDevice, s));
    if (o->trace_votes)
        CU(cudaMemcpy2DAsync(o->trace_votes + ((size_t)e0 * (lv + 1) + level) * K, sizeof(int32_t) * K * (lv + 1),
                             votes, sizeof(int32_t) * K, sizeof(int32_t) * K, n, cudaMemcpyDeviceToDevice, s));
    return APO_OK;
}

}  // extern "C"

namespace {

int validate_solve(const apo_geometry *g, const apo_hits *hits, const apo_solve_opts *o,
                   const apo_track *tracks_out, void *ws, size_t ws_bytes, Layout &L) {
    int rc;
    if ((rc = check_geom(g)) || (rc = check_hits(hits))) return rc;
    const int lv = g->dg.levels;
    if (lv < 1) return fail(APO_EINVAL, "apo_solve_batch needs levels >= 1");
    for (int i = 0; i <= lv; i++)
        if ((rc = check_precision(g, o->precision[i], "precision[level]"))) return rc;
    if (o->max_tracks < 1 || o->max_tracks > APO_MAX_TRACKS)
        return fail(APO_EINVAL, "max_tracks must be in [1, %d]", APO_MAX_TRACKS);
    if (!(o->mask_sigma >= 0.0 && o->mask_sigma < 1.0)) return fail(APO_EINVAL, "mask_sigma out of range");
    if (o->tune.cells_block != 0 && o->tune.cells_block != 128 && o->tune.cells_block != 256)
        return fail(APO_EINVAL, "tune.cells_block must be 0, 128 or 256");
    if (o->tune.chunk_events < 0) return fail(APO_EINVAL, "tune.chunk_events < 0");
    if (!tracks_out && hits->n_events > 0) return fail(APO_EINVAL, "tracks_out is NULL");
    if (o->schedule == APO_SCHED_MAXSET) {
        if (o->max_tracks > 1) {
            if (o->trace_count) return fail(APO_EINVAL, "APO_SCHED_MAXSET with max_tracks > 1 writes no trace");
            for (int i = 0; i <= lv; i++)
                if ((o->precision[i] & ~APO_OUTGOING) == APO_F64_MID)
                    return fail(APO_EINVAL, "APO_SCHED_MAXSET with max_tracks > 1 takes no APO_F64_MID level");
        } else if (o->hit_track) {
            return fail(APO_EINVAL, "APO_SCHED_MAXSET takes hit_track only with max_tracks > 1");
        }
        if (o->max_keep < 1 || o->max_keep > (1 << 20)) return fail(APO_EINVAL, "max_keep must be in [1, 2^20]");
        if (o->slack < 0) return fail(APO_EINVAL, "slack < 0");
        if (maxset_smem_bytes(g->dg) > 64 * 1024)
            return fail(APO_EINVAL, "APO_SCHED_MAXSET needs sum_a bins[a] << levels <= 16384");
    } else if (o->schedule == APO_SCHED_TOPK) {
        if (key_bits_total(g->dg) > 50) return fail(APO_EINVAL, "APO_SCHED_TOPK needs keys of at most 50 bits");
        if ((long long)g->dg.bins[1] * g->dg.bins[2] * 2 > 8192)
            return fail(APO_EINVAL, "APO_SCHED_TOPK needs bins[1] * bins[2] <= 4096");
        if (o->tune.persistent) {
            for (int i = 0; i <= lv; i++) {
                const int p = o->precision[i] & ~APO_OUTGOING;
                if (p != APO_F64 && p != APO_F32 && p != APO_F64_FILTERED)
                    return fail(APO_EINVAL, "the persistent launch takes APO_F64, APO_F32 or APO_F64_FILTERED");
                if ((o->precision[i] & APO_OUTGOING) != (o->precision[0] & APO_OUTGOING))
                    return fail(APO_EINVAL, "the persistent launch needs one APO_OUTGOING setting for all levels");
            }
            if (o->trace_keys || o->trace_votes) return fail(APO_EINVAL, "the persistent launch writes no trace");
            if (g->dg.topk * 32 > 4096) return fail(APO_EINVAL, "topk too large for the persistent launch");
        }
        if (o->trace_count || o->final_level || o->n_final)
            return fail(APO_EINVAL, "trace_count / final_level / n_final belong to APO_SCHED_MAXSET");
    } else {
        return fail(APO_EINVAL, "bad schedule");
    }
    return check_ws(g, hits->n_events, ws, ws_bytes, L, o);
}

// NVTX range for the host-side queueing of one phase (visible in Nsight timelines).
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
};

// The max-set schedule (APO_SCHED_MAXSET) for every chunk of events: level-0 voting of the
// whole grid (one thread per cell), then per level the selection of whole vote groups and
// the voting of the kept cells' children, until each event's search has ended.
template <typename PrecAt>
int enqueue_maxset(const apo_geometry *g, const apo_hits *hits, const apo_solve_opts *o, const DevGeom *gl,
                   PrecAt prec_at, apo_track *tracks_out, int32_t *n_tracks_out, void *ws, const Layout &L,
                   cudaStream_t s) {
    int rc;
    const int lv = g->dg.levels, K = o->max_keep, ne = hits->n_events, mt = o->max_tracks;
    unsigned *status = at<unsigned>(ws, L.status);
    int32_t *nh = at<int32_t>(ws, L.n_hits);
    HitRecD *hd = at<HitRecD>(ws, L.hd);
    HitRecF *hf = at<HitRecF>(ws, L.hf);
    int32_t *votes = at<int32_t>(ws, L.votes);
    uint64_t *front = at<uint64_t>(ws, L.ms_front);
    int32_t *count = at<int32_t>(ws, L.ms_count);
    int32_t *stop = at<int32_t>(ws, L.ms_stop);
    uint64_t *ck = at<uint64_t>(ws, L.ms_ck);
    int32_t *cv = at<int32_t>(ws, L.ms_cv);
    uint32_t *active = at<uint32_t>(ws, L.mask);
    int32_t *done = at<int32_t>(ws, L.done);
    int32_t *ntr = n_tracks_out ? n_tracks_out : at<int32_t>(ws, L.ntr);
    const int block = o->tune.cells_block ? o->tune.cells_block : 256;
    const int chunk = (o->tune.chunk_events > 0 && o->tune.chunk_events < L.ms_chunk) ? o->tune.chunk_events
                                                                                      : L.ms_chunk;
    CU(cudaMemsetAsync(status, 0, 256, s));
    launch_stage(g->dg, ne, hits->offsets, hits->wire_id, hits->drift, hd, hf, nh, active, done, status, s,
                 mt > 1 ? o->hit_track : nullptr);
    if ((rc = check_launch("stage"))) return rc;
    for (int e0 = 0; e0 < ne; e0 += chunk) {
        NvtxRange range_chunk("apo max-set chunk");
        const int n = ne - e0 < chunk ? ne - e0 : chunk;
        const HitRecD *hde = hd + (size_t)e0 * kHitCap;
        const HitRecF *hfe = hf + (size_t)e0 * kHitCap;
        const int32_t *nhe = nh + e0;
        // multi-track rounds search the hits still active; one track per event: every hit
        uint32_t *act = mt > 1 ? active + (size_t)e0 * 8 : nullptr;
        MaxsetArgs A{};
        A.levels = lv;
        A.max_keep = K;
        A.slack = o->slack;
        A.min_votes = o->min_votes;
        A.n_coarse = g->n_coarse;
        A.front = front;
        A.count_out = count;
        A.stop = stop;
        A.n_hits = nhe;
        A.tracks = tracks_out + (size_t)e0 * mt;
        A.n_tracks = ntr + e0;
        A.final_level = o->final_level ? o->final_level + (size_t)e0 * mt : nullptr;
        A.n_final = o->n_final ? o->n_final + (size_t)e0 * mt : nullptr;
        A.trace_keys = o->trace_count && o->trace_keys ? o->trace_keys + (size_t)e0 * (lv + 1) * K : nullptr;
        A.trace_votes = o->trace_count && o->trace_votes ? o->trace_votes + (size_t)e0 * (lv + 1) * K : nullptr;
        A.trace_count = o->trace_count ? o->trace_count + (size_t)e0 * (lv + 1) : nullptr;
        A.max_tracks = mt;
        A.width = 3.0 * o->mask_sigma;
        A.active = act;
        A.done = mt > 1 ? done + e0 : nullptr;
        A.hd = hde;
        A.hf = hfe;
        A.offsets = hits->offsets + e0;
        A.hit_track = mt > 1 ? o->hit_track : nullptr;
        A.ts = mt > 1 ? at<TrackStep>(ws, L.ms_ts) : nullptr;
        A.tcnt = mt > 1 ? at<uint32_t>(ws, L.ms_tcnt) : nullptr;
        A.cnt_stride = (int)(maxset_smem_bytes(g->dg) / sizeof(uint32_t));
        if (mt > 1) {   // no pending step, counters zero
            CU(cudaMemsetAsync(A.ts, 0, sizeof(TrackStep) * (size_t)n, s));
            CU(cudaMemsetAsync(A.tcnt, 0, maxset_smem_bytes(g->dg) * (size_t)n, s));
        }
        if (A.trace_count) CU(cudaMemsetAsync(A.trace_count, 0, sizeof(int32_t) * (size_t)n * (lv + 1), s));
        for (int r = 0; r < mt; r++) {
            A.round = r;
            CU(cudaMemsetAsync(stop, 0, sizeof(int32_t) * (size_t)n, s));
            // level 0: every cell of the grid, one thread each, in linear (= key) order
            launch_vote_keys(gl[0], prec_at(0), n, hde, hfe, nhe, 0, nullptr, g->n_coarse, votes, s, act);
            if ((rc = check_launch("vote_coarse_cells"))) return rc;
            A.level = 0;
            A.prec = prec_at(0) & ~APO_OUTGOING;
            A.votes = votes;
            A.keys = nullptr;
            A.count_in = nullptr;
            A.stride = g->n_coarse;
            launch_maxset_select(gl[0], n, A, s);
            if ((rc = check_launch("maxset_select"))) return rc;
            if (mt > 1) {
                launch_track_step(gl[0], n, A, s);
                if ((rc = check_launch("track_step"))) return rc;
            }
            for (int lev = 1; lev <= lv; lev++) {
                launch_vote_children(gl[lev], prec_at(lev), n, hde, hfe, nhe, lev, front, K, ck, cv, s, act,
                                     block, count);
                if ((rc = check_launch("vote_children"))) return rc;
                A.level = lev;
                A.prec = prec_at(lev) & ~APO_OUTGOING;
                A.votes = cv;
                A.keys = ck;
                A.count_in = count;
                A.stride = (long long)K * 32;
                launch_maxset_select(gl[lev], n, A, s);
                if ((rc = check_launch("maxset_select"))) return rc;
                if (mt > 1) {
                    launch_track_step(gl[lev], n, A, s);
                    if ((rc = check_launch("track_step"))) return rc;
                }
            }
        }
    }
    return APO_OK;
}

// Queues the whole search on stream s (no host synchronisation, capturable).
int enqueue_solve(const apo_geometry *g, const apo_hits *hits, const apo_solve_opts *o,
                  apo_track *tracks_out, int32_t *n_tracks_out, void *ws, const Layout &L,
                  cudaStream_t s) {
    int rc;
    const int lv = g->dg.levels, K = g->dg.topk;
    const int ne = hits->n_events;
    if (ne == 0) return APO_OK;
    unsigned *status = at<unsigned>(ws, L.status);
    int32_t *nh = at<int32_t>(ws, L.n_hits);
    HitRecD *hd = at<HitRecD>(ws, L.hd);
    HitRecF *hf = at<HitRecF>(ws, L.hf);
    int32_t *votes = at<int32_t>(ws, L.votes);
    uint32_t *hist = at<uint32_t>(ws, L.hist);
    uint64_t *fk = at<uint64_t>(ws, L.fk);
    int32_t *fv = at<int32_t>(ws, L.fv);
    uint64_t *ck = at<uint64_t>(ws, L.ck);
    int32_t *cv = at<int32_t>(ws, L.cv);
    uint32_t *active = at<uint32_t>(ws, L.mask);
    int32_t *done = at<int32_t>(ws, L.done);
    int32_t *ntr = n_tracks_out ? n_tracks_out : at<int32_t>(ws, L.ntr);
    uint64_t *cand_k = at<uint64_t>(ws, L.cand_k);
    int32_t *cand_v = at<int32_t>(ws, L.cand_v);
    const double width = 3.0 * o->mask_sigma;   // round-to-nearest, as the oracle
    const int chunk = (o->tune.chunk_events > 0 && o->tune.chunk_events < L.chunk) ? o->tune.chunk_events : L.chunk;
    const int block = o->tune.cells_block ? o->tune.cells_block : 256;
    auto prec_at = [&](int lev) {
        int p = o->precision[lev] & ~APO_OUTGOING;
        bool filt = lev == 0 ? o->tune.coarse_filter != 0 : o->tune.cells_filter != 0;
        return (p == APO_F64 && filt) ? (int)APO_F64_FILTERED : p;
    };
    DevGeom gl[APO_MAX_LEVELS + 1];   // per level: the geometry with that level's direction flag
    for (int lev = 0; lev <= lv; lev++) gl[lev] = geom_for(g, o->precision[lev]);
    if (o->schedule == APO_SCHED_MAXSET)
        return enqueue_maxset(g, hits, o, gl, prec_at, tracks_out, n_tracks_out, ws, L, s);
    if (o->tune.persistent) {
        CU(cudaMemsetAsync(status, 0, 256, s));
        launch_stage(g->dg, ne, hits->offsets, hits->wire_id, hits->drift, hd, hf, nh, active, done, status, s,
                     o->hit_track);
        if ((rc = check_launch("stage"))) return rc;
        CU(cudaMemsetAsync(at<int32_t>(ws, L.p_next), 0, sizeof(int32_t), s));
        PersistArgs A{};
        A.n_events = ne;
        A.max_tracks = o->max_tracks;
        A.min_votes = o->min_votes;
        A.width = width;
        auto mode_of = [](int p) {
            return p == APO_F32 ? kPersistF32 : (p == APO_F64_FILTERED ? kPersistF64Filtered : kPersistF64);
        };
        for (int lev = 0; lev <= lv; lev++) A.mode[lev] = mode_of(prec_at(lev));
        A.hd = hd;
        A.hf = hf;
        A.n_hits = nh;
        A.offsets = hits->offsets;
        A.active = active;
        A.done = done;
        A.next_event = at<int32_t>(ws, L.p_next);
        A.status = status;
        A.votes = at<int32_t>(ws, L.p_votes);
        A.hist = at<uint32_t>(ws, L.p_hist);
        A.fk = fk;
        A.fv = fv;
        A.ck = ck;
        A.cv = cv;
        A.tracks = tracks_out;
        A.n_tracks = ntr;
        A.hit_track = o->hit_track;
        launch_solve_persistent(gl[0], g->persist_blocks, A, s);
        return check_launch("solve_persistent");
    }
    CU(cudaMemsetAsync(status, 0, 256, s));
    launch_stage(g->dg, ne, hits->offsets, hits->wire_id, hits->drift, hd, hf, nh, active, done, status, s,
                 o->hit_track);
    if ((rc = check_launch("stage"))) return rc;
    for (int e0 = 0; e0 < ne; e0 += chunk) {
        const int n = ne - e0 < chunk ? ne - e0 : chunk;
        uint64_t *fke = fk + (size_t)e0 * K;
        int32_t *fve = fv + (size_t)e0 * K;
        uint64_t *cke = ck + (size_t)e0 * K * 32;
        int32_t *cve = cv + (size_t)e0 * K * 32;
        const HitRecD *hde = hd + (size_t)e0 * kHitCap;
        const HitRecF *hfe = hf + (size_t)e0 * kHitCap;
        const int32_t *nhe = nh + e0;
        uint32_t *acte = active + (size_t)e0 * 8;
        // one round per track: search the active hits, record, mask the track's hits
        for (int round = 0; round < o->max_tracks; round++) {
            NvtxRange range_round("apo search round");
            CU(cudaMemsetAsync(hist, 0, sizeof(uint32_t) * (size_t)n * kHistBins, s));
            if (prec_at(0) == APO_F64_MID || o->tune.coarse_full) {   // every cell's vote, then the selection
                launch_vote_coarse(gl[0], prec_at(0), e0, n, hd, hf, nh, votes, hist, status, s, nullptr, active);
                if ((rc = check_launch("vote_coarse"))) return rc;
                launch_select_coarse(g->dg, e0, n, votes, hist, K, fk, fv, s);
                if ((rc = check_launch("select_coarse"))) return rc;
            } else {   // each block's K best cells, then the selection among them
                launch_vote_coarse(gl[0], prec_at(0), e0, n, hd, hf, nh, nullptr, hist, status, s, nullptr, active,
                                   cand_k, cand_v, K);
                if ((rc = check_launch("vote_coarse"))) return rc;
                launch_select_candidates(g->dg, e0, n, cand_k, cand_v, coarse_lists(gl[0], prec_at(0)), hist, K,
                                         fk, fv, s);
                if ((rc = check_launch("select_candidates"))) return rc;
            }
            if (round == 0 && (rc = trace_copy(o, g, e0, n, 0, fke, fve, s))) return rc;
            for (int lev = 1; lev <= lv; lev++) {
                launch_vote_children(gl[lev], prec_at(lev), n, hde, hfe, nhe, lev, fke, K, cke, cve, s, acte,
                                     block);
                if ((rc = check_launch("vote_children"))) return rc;
                launch_topk(n, cke, cve, K * 32, K, fke, fve, s);
                if ((rc = check_launch("topk"))) return rc;
                if (round == 0 && (rc = trace_copy(o, g, e0, n, lev, fke, fve, s))) return rc;
            }
            launch_estimate_mask(gl[lv], n, cke, cve, K * 32, lv, nhe, acte, done + e0, hde, round,
                                 o->max_tracks, o->min_votes, width,
                                 tracks_out + (size_t)e0 * o->max_tracks, ntr + e0, s,
                                 hits->offsets + e0, o->hit_track);
            if ((rc = check_launch("estimate_mask"))) return rc;
        }
    }
    return APO_OK;
}

// Key of a recorded search: every argument that the queued work depends on.
size_t graph_key(unsigned char *k, const apo_hits *h, const apo_solve_opts *o, const apo_track *t,
                 const int32_t *nt, const void *ws, size_t ws_bytes) {
    size_t n = 0;
    auto put = [&](const void *p, size_t b) { std::memcpy(k + n, p, b); n += b; };
    put(h, sizeof(*h));
    apo_solve_opts oc = *o;
    oc.use_graph = 0;
    put(&oc, sizeof(oc));
    put(&t, sizeof(t));
    put(&nt, sizeof(nt));
    put(&ws, sizeof(ws));
    put(&ws_bytes, sizeof(ws_bytes));
    return n;
}

}  // namespace

extern "C" {

int apo_solve_batch(const apo_geometry *g, const apo_hits *hits, const apo_solve_opts *opts,
                    apo_track *tracks_out, int32_t *n_tracks_out, void *ws, size_t ws_bytes, void *stream) {
    apo_solve_opts def;
    apo_solve_opts_default(&def);
    const apo_solve_opts *o = opts ? opts : &def;
    Layout L;
    int rc = validate_solve(g, hits, o, tracks_out, ws, ws_bytes, L);
    if (rc) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (!o->use_graph || hits->n_events == 0)
        return enqueue_solve(g, hits, o, tracks_out, n_tracks_out, ws, L, s);
    static_assert(sizeof(apo_hits) + sizeof(apo_solve_opts) + 4 * sizeof(void *) <= sizeof(GraphEntry::key),
                  "graph key size");
    apo_geometry *gm = const_cast<apo_geometry *>(g);
    GraphEntry ent;
    ent.key_len = graph_key(ent.key, hits, o, tracks_out, n_tracks_out, ws, ws_bytes);
    std::lock_guard<std::mutex> lk(gm->graph_mu);
    for (GraphEntry &e : gm->graphs)
        if (e.key_len == ent.key_len && std::memcmp(e.key, ent.key, ent.key_len) == 0) {
            CU(cudaGraphLaunch(e.exec, s));
            return APO_OK;
        }
    if (!gm->capture_stream) CU(cudaStreamCreateWithFlags(&gm->capture_stream, cudaStreamNonBlocking));
    cudaStream_t cap = gm->capture_stream;
    CU(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
    rc = enqueue_solve(g, hits, o, tracks_out, n_tracks_out, ws, L, cap);
    cudaGraph_t graph = nullptr;
    cudaError_t ce = cudaStreamEndCapture(cap, &graph);
    if (rc != APO_OK) {
        if (graph) cudaGraphDestroy(graph);
        return rc;
    }
    if (ce != cudaSuccess) return fail(APO_ECUDA, "stream capture: %s", cudaGetErrorString(ce));
    ce = cudaGraphInstantiate(&ent.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ce != cudaSuccess) return fail(APO_ECUDA, "graph instantiate: %s", cudaGetErrorString(ce));
    gm->graphs.push_back(ent);
    CU(cudaGraphLaunch(ent.exec, s));
    return APO_OK;
}

int apo_autotune(const apo_geometry *g, const apo_hits *hits, const apo_solve_opts *opts, void *ws,
                 size_t ws_bytes, void *stream, apo_tune *best, float *best_ms) {
    if (!best) return fail(APO_EINVAL, "best is NULL");
    apo_solve_opts def;
    apo_solve_opts_default(&def);
    apo_solve_opts o = opts ? *opts : def;
    o.use_graph = 0;
    o.trace_keys = nullptr;
    o.trace_votes = nullptr;
    o.trace_count = nullptr;
    o.final_level = nullptr;
    o.n_final = nullptr;
    std::memset(&o.tune, 0, sizeof(o.tune));
    Layout L;
    apo_track *tt = nullptr;
    int rc = check_ws(g, hits ? hits->n_events : 0, ws, ws_bytes, L, &o);
    if (rc) return rc;
    tt = at<apo_track>(ws, L.tune_tracks);
    if ((rc = validate_solve(g, hits, &o, tt, ws, ws_bytes, L))) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    *best = o.tune;
    float best_t = 1e30f;
    cudaEvent_t e0, e1;
    CU(cudaEventCreate(&e0));
    CU(cudaEventCreate(&e1));
    const int chunks[2] = {0, L.chunk > 4 ? L.chunk / 4 : 0};
    // the persistent launch is a candidate when the options allow it (and the workspace
    // holds its per-block scratch)
    bool try_persistent = false;
    {
        apo_solve_opts op = o;
        op.tune.persistent = 1;
        Layout Lp;
        char keep[sizeof(g_err)];
        std::memcpy(keep, g_err, sizeof(g_err));
        try_persistent = validate_solve(g, hits, &op, tt, ws, ws_bytes, Lp) == APO_OK;
        std::memcpy(g_err, keep, sizeof(g_err));
    }
    for (int full = 0; full < 2; full++)
    for (int ps = 0; ps < 2; ps++)
    for (int cf = 0; cf < 2; cf++)
        for (int lf = 0; lf < 2; lf++)
            for (int bs = 0; bs < 2; bs++)
                for (int ch = 0; ch < 2; ch++) {
                    if (ch == 1 && chunks[1] == 0) continue;
                    if (ps == 1 && (!try_persistent || bs == 1 || ch == 1 || full == 1)) continue;
                    if (full == 1 && o.schedule != APO_SCHED_TOPK) continue;
                    apo_tune t{cf, lf, bs ? 128 : 256, chunks[ch], full, ps};
                    o.tune = t;
                    if (layout(g, hits->n_events, &o).end > ws_bytes) continue;   // needs more workspace
                    float ms = 0.f;
                    Layout Lt = layout(g, hits->n_events, &o);
                    for (int rep = 0; rep < 2 && rc == APO_OK; rep++) {   // warm-up, then timed
                        if (rep == 1) cudaEventRecord(e0, s);
                        rc = enqueue_solve(g, hits, &o, tt, nullptr, ws, Lt, s);
                        if (rep == 1) cudaEventRecord(e1, s);
                    }
                    if (rc != APO_OK) break;
                    if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
                        rc = fail(APO_ECUDA, "autotune timing failed");
                        break;
                    }
                    if (ms < best_t) { best_t = ms; *best = t; }
                }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != APO_OK) return rc;
    if (best_ms) *best_ms = best_t;
    return APO_OK;
}

int apo_diag_vote_coarse_counts(const apo_geometry *g, const apo_hits *hits, int32_t precision,
                                int32_t *votes_out, unsigned long long *counts, void *ws,
                                size_t ws_bytes, void *stream) {
    int rc;
    if ((rc = check_geom(g)) || (rc = check_hits(hits))) return rc;
    if ((rc = check_precision(g, precision, "precision"))) return rc;
    if (!votes_out && (precision & ~APO_OUTGOING) == APO_F64_MID)
        return fail(APO_EINVAL, "the midpoint form keeps every vote: votes_out is needed");
    Layout L;
    if ((rc = check_ws(g, hits->n_events, ws, ws_bytes, L))) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int ne = hits->n_events;
    if (counts) CU(cudaMemsetAsync(counts, 0, 8 * sizeof(unsigned long long), s));
    if (ne == 0) return APO_OK;
    unsigned *status = at<unsigned>(ws, L.status);
    int32_t *nh = at<int32_t>(ws, L.n_hits);
    HitRecD *hd = at<HitRecD>(ws, L.hd);
    HitRecF *hf = at<HitRecF>(ws, L.hf);
    uint32_t *hist = at<uint32_t>(ws, L.hist);
    CU(cudaMemsetAsync(status, 0, 256, s));
    launch_stage(g->dg, ne, hits->offsets, hits->wire_id, hits->drift, hd, hf, nh,
                 at<uint32_t>(ws, L.mask), at<int32_t>(ws, L.done), status, s);
    unsigned long long launches = 0;
    for (int e0 = 0; e0 < ne; e0 += L.chunk) {
        int n = ne - e0 < L.chunk ? ne - e0 : L.chunk;
        CU(cudaMemsetAsync(hist, 0, sizeof(uint32_t) * (size_t)n * kHistBins, s));
        const DevGeom dg = geom_for(g, precision);
        const int prec = precision & ~APO_OUTGOING;
        if (votes_out)
            launch_vote_coarse(dg, prec, e0, n, hd, hf, nh, votes_out + (size_t)e0 * g->n_coarse, hist, status, s,
                               counts);
        else   // the search's form: each block keeps its topk best cells
            launch_vote_coarse(dg, prec, e0, n, hd, hf, nh, nullptr, hist, status, s, counts, nullptr,
                               at<uint64_t>(ws, L.cand_k), at<int32_t>(ws, L.cand_v), g->dg.topk);
        if ((rc = check_launch("vote_coarse"))) return rc;
        launches++;
    }
    if (counts) CU(cudaMemcpyAsync(counts + 3, &launches, sizeof(launches), cudaMemcpyHostToDevice, s));
    CU(cudaStreamSynchronize(s));
    return APO_OK;
}

int32_t apo_diag_coarse_launches(const apo_geometry *g, int32_t n_events) {
    if (!g || n_events <= 0) return 0;
    Layout L = layout(g, n_events);
    return (n_events + L.chunk - 1) / L.chunk;
}

int apo_diag_wait_timeout(int32_t limit_polls) {
    unsigned *st = nullptr;
    CU(cudaMalloc(&st, sizeof(unsigned)));
    unsigned h = 0;
    cudaError_t e = cudaMemset(st, 0, sizeof(unsigned));
    if (e == cudaSuccess) {
        launch_wait_never(limit_polls > 0 ? limit_polls : 1, st, 0);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(&h, st, sizeof(unsigned), cudaMemcpyDeviceToHost);
    cudaFree(st);
    if (e != cudaSuccess) return fail(APO_ECUDA, "wait test: %s", cudaGetErrorString(e));
    if (h & ST_TIMEOUT) return fail(APO_ETIMEOUT, "device wait ran out of its poll limit");
    return APO_OK;
}

int apo_workspace_status(const apo_geometry *g, int32_t n_events, const void *ws, void *stream) {
    int rc;
    if ((rc = check_geom(g))) return rc;
    if (!ws) return fail(APO_EINVAL, "workspace is NULL");
    Layout L = layout(g, n_events);
    unsigned h = 0;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    CU(cudaMemcpyAsync(&h, static_cast<const unsigned char *>(ws) + L.status, sizeof(unsigned),
                       cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    if (h & ST_TIMEOUT) return fail(APO_ETIMEOUT, "a device wait ran out of its poll limit");
    return APO_OK;
}

int apo_diag_pipe_peak(int32_t precision, int32_t op, double *ops_per_s) {
    if (!ops_per_s) return fail(APO_EINVAL, "ops_per_s is NULL");
    if (precision != APO_F64 && precision != APO_F32) return fail(APO_EINVAL, "bad precision");
    double r = pipe_peak(precision, op);
    if (r <= 0) return fail(APO_ECUDA, "pipe microbenchmark failed");
    *ops_per_s = r;
    return APO_OK;
}

int apo_diag_dops(int32_t op, const double *x, double *out, int64_t n, void *stream) {
    if (op < 0 || op > 17) return fail(APO_EINVAL, "bad op");
    if (n < 0 || (n > 0 && (!x || !out))) return fail(APO_EINVAL, "bad arguments");
    if (op >= 12 && op <= 17 && (n & 1)) return fail(APO_EINVAL, "quotients need an even n");
    if (launch_dops(op, x, out, n, static_cast<cudaStream_t>(stream)))
        return fail(APO_ECUDA, "dops launch failed");
    return APO_OK;
}

int apo_diag_vote_pair_ends(const apo_geometry *g, int32_t precision, const double *cells,
                            const double *hits, double *out, int64_t n, void *stream) {
    int rc;
    if ((rc = check_geom(g))) return rc;
    const int base = precision & ~APO_OUTGOING;
    if ((base != APO_F64 && base != APO_F32) || (precision & ~(APO_OUTGOING | 7)))
        return fail(APO_EINVAL, "bad precision");
    if (n < 0 || (n > 0 && (!cells || !hits || !out))) return fail(APO_EINVAL, "bad arguments");
    if (launch_pair_ends(geom_for(g, precision).k, base == APO_F64 ? 0 : 1, cells, hits, out, n,
                         static_cast<cudaStream_t>(stream)))
        return fail(APO_ECUDA, "pair-ends launch failed");
    return APO_OK;
}

int apo_solve_batch_host(const apo_geometry *g, int32_t n_events, const int32_t *offsets,
                         const int32_t *wire_id, const double *drift, const apo_solve_opts *opts,
                         apo_track *tracks_out, int32_t *n_tracks_out, void *ws, size_t ws_bytes,
                         void *stream) {
    int rc;
    if ((rc = check_geom(g))) return rc;
    if (n_events < 0 || (n_events > 0 && (!offsets || !tracks_out))) return fail(APO_EINVAL, "bad arguments");
    const int64_t n_hits = n_events > 0 ? offsets[n_events] : 0;
    if (n_hits < 0) return fail(APO_EINVAL, "offsets[n_events] < 0");
    if (n_hits > 0 && (!wire_id || !drift)) return fail(APO_EINVAL, "hit arrays are NULL");
    apo_solve_opts def;
    apo_solve_opts_default(&def);
    const apo_solve_opts *o = opts ? opts : &def;
    if (o->hit_track) return fail(APO_EINVAL, "apo_solve_batch_host takes no hit_track (device output)");
    if (o->final_level || o->n_final || o->trace_count || o->trace_keys || o->trace_votes)
        return fail(APO_EINVAL, "apo_solve_batch_host takes no device traces or per-event outputs");
    Layout L = layout(g, n_events, o);
    const size_t need = L.end + apo_host_extra_bytes(n_events, n_hits);
    if (!ws || ws_bytes < need) return fail(APO_ENOMEM, "workspace too small: %zu < %zu", ws_bytes, need);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    size_t off = L.end;
    int32_t *d_off = at<int32_t>(ws, off); off += align256(sizeof(int32_t) * (size_t)(n_events + 1));
    int32_t *d_wid = at<int32_t>(ws, off); off += align256(sizeof(int32_t) * (size_t)n_hits);
    double *d_dr = at<double>(ws, off); off += align256(sizeof(double) * (size_t)n_hits);
    apo_track *d_tr = at<apo_track>(ws, off); off += align256(sizeof(apo_track) * (size_t)n_events * APO_MAX_TRACKS);
    int32_t *d_nt = at<int32_t>(ws, off);
    CU(cudaMemcpyAsync(d_off, offsets, sizeof(int32_t) * (size_t)(n_events + 1), cudaMemcpyHostToDevice, s));
    if (n_hits > 0) {
        CU(cudaMemcpyAsync(d_wid, wire_id, sizeof(int32_t) * (size_t)n_hits, cudaMemcpyHostToDevice, s));
        CU(cudaMemcpyAsync(d_dr, drift, sizeof(double) * (size_t)n_hits, cudaMemcpyHostToDevice, s));
    }
    apo_hits h{n_events, d_off, d_wid, d_dr};
    if ((rc = apo_solve_batch(g, &h, o, d_tr, d_nt, ws, L.end, stream))) return rc;
    CU(cudaMemcpyAsync(tracks_out, d_tr, sizeof(apo_track) * (size_t)n_events * o->max_tracks,
                       cudaMemcpyDeviceToHost, s));
    if (n_tracks_out)
        CU(cudaMemcpyAsync(n_tracks_out, d_nt, sizeof(int32_t) * (size_t)n_events, cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    unsigned st = 0;
    CU(cudaMemcpy(&st, at<unsigned>(ws, L.status), sizeof(unsigned), cudaMemcpyDeviceToHost));
    if (st & ST_TIMEOUT) return fail(APO_ETIMEOUT, "a device wait ran out of its poll limit");
    return APO_OK;
}

}  // extern "C"
