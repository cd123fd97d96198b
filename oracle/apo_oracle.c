/* Plain CPU oracle of interval-arithmetic Apollonius voting over the 5-D helix parameter
 * space (arXiv:2401.04576, Sections 3.1 and 3.3, Appendix A).
 *
 * TEST INFRASTRUCTURE.  Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline /
 * reference leg load this library.  It shares no code with the CUDA path.
 *
 * It is slow on purpose: every cell is evaluated against every hit with the full interval
 * program of vote_program.inc, one directed operation at a time, under fesetround
 * (FE_DOWNWARD, upward results by exact negation).  OpenMP only splits the loop over
 * cells; it changes no result.
 *
 * Build: cc -O1 -frounding-math -ffp-contract=off -fno-fast-math -fopenmp -shared -fPIC
 * (no FMA contraction: every product and sum is rounded on its own).
 */
#include <fenv.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#pragma STDC FENV_ACCESS ON

#define REAL double
#define SFX _d
#define SQRT sqrt
#define NEXTUP(x) nextafter((x), INFINITY)
#include "vote_program.inc"
#include "midpoint.inc"
#include "exactphi.inc"
#include "fourd.inc"
#undef REAL
#undef SFX
#undef SQRT
#undef NEXTUP

#define REAL float
#define SFX _f
#define SQRT sqrtf
#define NEXTUP(x) nextafterf((x), INFINITY)
#include "vote_program.inc"
#include "fourd.inc"
#undef REAL
#undef SFX
#undef SQRT
#undef NEXTUP

/* ------------------------------------------------------------------------------------ */
/* Inputs                                                                                */
/* ------------------------------------------------------------------------------------ */
typedef struct {
    int32_t n_wires;
    const double *x0, *y0, *sin_phis, *cos_phis, *tan_tau, *sphi_t, *cphi_t, *t2;
} or_wires;

typedef struct {
    int32_t bins[5];
    int32_t levels;
    int32_t topk;
    const double *lo_edge[5];     /* finest-level cell edges, bins[a] << levels each */
    const double *hi_edge[5];
    const double *sincos;         /* rows of (sin lo, sin hi, cos lo, cos hi) */
    const int64_t *sincos_offset; /* first row of level L */
    const double *sincos_mid;     /* rows of (sin, cos) of each phi0 cell's centre, same
                                     offsets; needed by the midpoint form only */
} or_grid;

/* One cell of `level` as 6 FP64 intervals: D, S0, C0, W, Z, L (lo, hi each). */
static void cell_intervals(const or_grid *g, int level, const int32_t idx[5], double c[12]) {
    int sh = g->levels - level;
    double lo[5], hi[5];
    for (int a = 0; a < 5; a++) {
        int64_t i = idx[a];
        lo[a] = g->lo_edge[a][i << sh];
        hi[a] = g->hi_edge[a][((i + 1) << sh) - 1];
    }
    const double *sc = g->sincos + 4 * (g->sincos_offset[level] + idx[1]);
    c[0] = lo[0]; c[1] = hi[0];
    c[2] = sc[0]; c[3] = sc[1];
    c[4] = sc[2]; c[5] = sc[3];
    c[6] = lo[2]; c[7] = hi[2];
    c[8] = lo[3]; c[9] = hi[3];
    c[10] = lo[4]; c[11] = hi[4];
}

static void hit_constants(const or_wires *w, int32_t wid, double drift, double h[9]) {
    h[0] = w->x0[wid]; h[1] = w->y0[wid]; h[2] = w->sin_phis[wid]; h[3] = w->cos_phis[wid];
    h[4] = w->tan_tau[wid]; h[5] = w->sphi_t[wid]; h[6] = w->cphi_t[wid]; h[7] = w->t2[wid];
    h[8] = drift;
}

/* FP32 inputs: each FP64 end point rounded outward (lo down, hi up). */
static float rd32(double x) { volatile float r = (float)x; return r; }   /* FE_DOWNWARD */
static float ru32(double x) { volatile float r = (float)(-x); return -r; }

/* Flag bit of a precision code: apply the direction condition of the vote program (the
 * hit lies on the outgoing arc, downstream of the POCA). */
#define OR_OUTGOING 16
/* vote-count bins of the max-set schedule's histogram (counts are at most the hit cap) */
#define APO_OR_HIST 257

/* The vote of one (cell, hit) pair.  prec 0: FP64 intervals, 1: FP32 intervals, 4: FP64
 * intervals with the exact phase (exactphi.inc); optionally | OR_OUTGOING. */
static int vote_pair(const double c[12], const double h[9], int prec_code, double *out) {
    const int og = (prec_code & OR_OUTGOING) != 0, prec = prec_code & ~OR_OUTGOING;
    if (prec == 4) {
        iv_d C[6], H[9];
        for (int i = 0; i < 6; i++) C[i] = mk_d(c[2 * i], c[2 * i + 1]);
        for (int i = 0; i < 9; i++) H[i] = mk_d(h[i], h[i]);
        return exact_vote_program_d(C[0], C[1], C[2], C[3], C[4], C[5], H[0], H[1], H[2], H[3],
                                    H[4], H[5], H[6], H[7], H[8], og, out);
    }
    if (prec == 0) {
        iv_d C[6], H[9];
        for (int i = 0; i < 6; i++) C[i] = mk_d(c[2 * i], c[2 * i + 1]);
        for (int i = 0; i < 9; i++) H[i] = mk_d(h[i], h[i]);
        return vote_program_d(C[0], C[1], C[2], C[3], C[4], C[5], H[0], H[1], H[2], H[3],
                              H[4], H[5], H[6], H[7], H[8], og, out);
    } else {
        iv_f C[6], H[9];
        for (int i = 0; i < 6; i++) C[i] = mk_f(rd32(c[2 * i]), ru32(c[2 * i + 1]));
        for (int i = 0; i < 9; i++) H[i] = mk_f(rd32(h[i]), ru32(h[i]));
        return vote_program_f(C[0], C[1], C[2], C[3], C[4], C[5], H[0], H[1], H[2], H[3],
                              H[4], H[5], H[6], H[7], H[8], og, out);
    }
}

/* ------------------------------------------------------------------------------------ */
/* Exported: one pair                                                                    */
/* ------------------------------------------------------------------------------------ */
int or_vote_pair(const double cell[12], const double hit[9], int prec, double out[9]) {
    int old = fegetround();
    fesetround(FE_DOWNWARD);
    int v = vote_pair(cell, hit, prec, out);
    fesetround(old);
    return v;
}

/* One pair in the midpoint form: scm = sin, cos of the phi0 centre; out[7] as in
 * mid_vote_program. */
int or_vote_pair_mid(const double cell[12], const double scm[2], const double hit[9], double out[7]) {
    int old = fegetround();
    fesetround(FE_DOWNWARD);
    int v = mid_vote_program(cell, scm, hit, out);
    fesetround(old);
    return v;
}

/* ------------------------------------------------------------------------------------ */
/* Cell keys                                                                             */
/* ------------------------------------------------------------------------------------ */
/* Key layout: idx_a occupies bits_a = max(10, ceil(log2(bins_a << levels))) bits starting
 * at s_a = bits_0 + ... + bits_(a-1), d0 lowest; g = NULL means 10 bits per axis. */
static void key_layout(const or_grid *g, int sh[5], uint64_t mk[5]) {
    int s = 0;
    for (int a = 0; a < 5; a++) {
        int bits = 10;
        if (g) {
            int64_t n = (int64_t)g->bins[a] << g->levels;
            while (((int64_t)1 << bits) < n) bits++;
        }
        sh[a] = s;
        mk[a] = ((uint64_t)1 << bits) - 1;
        s += bits;
    }
}
static void key_to_idx(const or_grid *g, uint64_t key, int32_t idx[5]) {
    int sh[5];
    uint64_t mk[5];
    key_layout(g, sh, mk);
    for (int a = 0; a < 5; a++) idx[a] = (int32_t)((key >> sh[a]) & mk[a]);
}
static uint64_t idx_to_key(const or_grid *g, const int32_t idx[5]) {
    int sh[5];
    uint64_t mk[5];
    key_layout(g, sh, mk);
    uint64_t k = 0;
    for (int a = 0; a < 5; a++) k |= (uint64_t)idx[a] << sh[a];
    return k;
}

/* sin, cos of the phi0 centre of cell idx at `level` */
static void centre_sincos(const or_grid *g, int level, const int32_t idx[5], double scm[2]) {
    const double *r = g->sincos_mid + 2 * (g->sincos_offset[level] + idx[1]);
    scm[0] = r[0];
    scm[1] = r[1];
}

/* votes of n cells of `level` (given by key) for one event's hits: Eq. (ApoVote) summed
 * over hits, one vote per (cell, hit) whichever drift sign passes (Section 3.1).
 * prec 0: FP64 intervals, 1: FP32 intervals, 3: the FP64 midpoint form, 4: FP64 intervals
 * with the exact phase; | OR_OUTGOING (not with 3) adds the direction condition. */
void or_vote_cells(const or_grid *g, const or_wires *w, int32_t n_hits, const int32_t *wire_id,
                   const double *drift, int32_t level, int32_t prec, const uint64_t *keys,
                   int64_t n, int32_t *votes) {
    #pragma omp parallel
    {
        int old = fegetround();
        fesetround(FE_DOWNWARD);
        const int base = prec & ~OR_OUTGOING;   /* the midpoint form takes no direction flag */
        #pragma omp for schedule(dynamic, 256)
        for (int64_t j = 0; j < n; j++) {
            int32_t idx[5];
            double c[12], h[9];
            double scm[2] = {0, 0};
            key_to_idx(g, keys[j], idx);
            cell_intervals(g, level, idx, c);
            if (base == 3) centre_sincos(g, level, idx, scm);
            int32_t v = 0;
            for (int32_t i = 0; i < n_hits; i++) {
                hit_constants(w, wire_id[i], drift[i], h);
                v += base == 3 ? mid_vote_program(c, scm, h, NULL) : vote_pair(c, h, prec, NULL);
            }
            votes[j] = v;
        }
        fesetround(old);
    }
}

/* keys of all level-0 cells in linear order (d0 fastest, tanl slowest = key order) */
static void coarse_keys(const or_grid *g, uint64_t *keys) {
    int64_t n = 1;
    for (int a = 0; a < 5; a++) n *= g->bins[a];
    for (int64_t j = 0; j < n; j++) {
        int64_t r = j;
        int32_t idx[5];
        for (int a = 0; a < 5; a++) { idx[a] = (int32_t)(r % g->bins[a]); r /= g->bins[a]; }
        keys[j] = idx_to_key(g, idx);
    }
}

void or_coarse_keys(const or_grid *g, uint64_t *keys) { coarse_keys(g, keys); }

/* ------------------------------------------------------------------------------------ */
/* Top-K and bisection                                                                   */
/* ------------------------------------------------------------------------------------ */
typedef struct { uint64_t key; int32_t votes; } kv;

/* votes descending, then key ascending (deterministic tie-break) */
static int kv_cmp(const void *pa, const void *pb) {
    const kv *a = (const kv *)pa, *b = (const kv *)pb;
    if (a->votes != b->votes) return a->votes > b->votes ? -1 : 1;
    if (a->key != b->key) return a->key < b->key ? -1 : 1;
    return 0;
}

/* The K best cells by (votes desc, key asc); returns how many were written (min(K, n)). */
int64_t or_topk(const uint64_t *keys, const int32_t *votes, int64_t n, int32_t K,
                uint64_t *out_keys, int32_t *out_votes) {
    kv *a = (kv *)malloc(sizeof(kv) * (size_t)(n > 0 ? n : 1));
    for (int64_t j = 0; j < n; j++) { a[j].key = keys[j]; a[j].votes = votes[j]; }
    qsort(a, (size_t)n, sizeof(kv), kv_cmp);
    int64_t m = n < K ? n : K;
    for (int64_t j = 0; j < m; j++) { out_keys[j] = a[j].key; out_votes[j] = a[j].votes; }
    free(a);
    return m;
}

/* each cell -> its 32 children (index 2 idx_a + bit_a, bit_a = bit a of the child number) */
void or_children(const or_grid *g, const uint64_t *keys, int64_t n, uint64_t *children) {
    for (int64_t j = 0; j < n; j++) {
        int32_t idx[5], c[5];
        key_to_idx(g, keys[j], idx);
        for (int b = 0; b < 32; b++) {
            for (int a = 0; a < 5; a++) c[a] = 2 * idx[a] + ((b >> a) & 1);
            children[32 * j + b] = idx_to_key(g, c);
        }
    }
}

/* Final estimate (Section 3.3: values and errors from the centres and sizes of the
 * maximum-vote voxels): over the cells whose votes equal the maximum, in ascending key
 * order, value = mean of the cell centres (lo + hi) / 2 and error = (max hi - min lo) / 2
 * per axis, all in round-to-nearest. */
static void estimate(const or_grid *g, int level, const uint64_t *keys, const int32_t *votes,
                     int64_t n, double p[5], double werr[5], int32_t *best) {
    int32_t vmax = -1;
    for (int64_t j = 0; j < n; j++) if (votes[j] > vmax) vmax = votes[j];
    kv *a = (kv *)malloc(sizeof(kv) * (size_t)(n > 0 ? n : 1));
    int64_t m = 0;
    for (int64_t j = 0; j < n; j++)
        if (votes[j] == vmax) { a[m].key = keys[j]; a[m].votes = votes[j]; m++; }
    qsort(a, (size_t)m, sizeof(kv), kv_cmp);
    int sh = g->levels - level;
    for (int ax = 0; ax < 5; ax++) {
        double sum = 0, lo_min = INFINITY, hi_max = -INFINITY;
        for (int64_t j = 0; j < m; j++) {
            int32_t idx[5];
            key_to_idx(g, a[j].key, idx);
            double lo = g->lo_edge[ax][(int64_t)idx[ax] << sh];
            double hi = g->hi_edge[ax][(((int64_t)idx[ax] + 1) << sh) - 1];
            sum += (lo + hi) / 2;
            if (lo < lo_min) lo_min = lo;
            if (hi > hi_max) hi_max = hi;
        }
        p[ax] = sum / (double)m;
        werr[ax] = (hi_max - lo_min) / 2;
    }
    *best = vmax;
    free(a);
}

/* Whole coarse-to-fine search for one event (configuration of the grid: bins, levels,
 * top-K).  Level 0 is the full grid; at each level the K best cells survive and are
 * bisected along every axis; the last level's maximum-vote cells give the estimate.
 * prec[L] selects FP64 (0) or FP32 (1) intervals or the FP64 midpoint form (3) at level L.
 * Trace outputs (may be NULL): frontier keys / votes kept after level L, K per level,
 * and the last level's votes (K * 32). */
int or_solve_event(const or_grid *g, const or_wires *w, int32_t n_hits, const int32_t *wire_id,
                   const double *drift, const int32_t *prec, double p[5], double werr[5],
                   int32_t *best_votes, uint64_t *trace_keys, int32_t *trace_votes,
                   uint64_t *last_keys, int32_t *last_votes) {
    int64_t n0 = 1;
    for (int a = 0; a < 5; a++) n0 *= g->bins[a];
    int32_t K = g->topk;
    uint64_t *keys = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)n0);
    int32_t *votes = (int32_t *)malloc(sizeof(int32_t) * (size_t)n0);
    coarse_keys(g, keys);
    or_vote_cells(g, w, n_hits, wire_id, drift, 0, prec[0], keys, n0, votes);
    uint64_t *fk = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)K);
    int32_t *fv = (int32_t *)malloc(sizeof(int32_t) * (size_t)K);
    uint64_t *ck = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)K * 32);
    int32_t *cv = (int32_t *)malloc(sizeof(int32_t) * (size_t)K * 32);
    int64_t m = or_topk(keys, votes, n0, K, fk, fv);
    if (trace_keys) { memcpy(trace_keys, fk, sizeof(uint64_t) * (size_t)m); memcpy(trace_votes, fv, sizeof(int32_t) * (size_t)m); }
    for (int L = 1; L <= g->levels; L++) {
        or_children(g, fk, m, ck);
        or_vote_cells(g, w, n_hits, wire_id, drift, L, prec[L], ck, m * 32, cv);
        if (L == g->levels) {
            estimate(g, L, ck, cv, m * 32, p, werr, best_votes);
            if (last_keys) { memcpy(last_keys, ck, sizeof(uint64_t) * (size_t)m * 32); memcpy(last_votes, cv, sizeof(int32_t) * (size_t)m * 32); }
            break;
        }
        m = or_topk(ck, cv, m * 32, K, fk, fv);
        if (trace_keys) {
            memcpy(trace_keys + (size_t)L * K, fk, sizeof(uint64_t) * (size_t)m);
            memcpy(trace_votes + (size_t)L * K, fv, sizeof(int32_t) * (size_t)m);
        }
    }
    if (g->levels == 0) estimate(g, 0, keys, votes, n0, p, werr, best_votes);
    free(keys); free(votes); free(fk); free(fv); free(ck); free(cv);
    return 0;
}

/* ------------------------------------------------------------------------------------ */
/* Max-set schedule                                                                       */
/* ------------------------------------------------------------------------------------ */
static int kv_key_cmp(const void *pa, const void *pb) {
    uint64_t a = ((const kv *)pa)->key, b = ((const kv *)pb)->key;
    return a < b ? -1 : (a > b ? 1 : 0);
}

/* Estimate of Section 3.3 over the cells of `level` whose votes equal vmax (m of them):
 * per axis, with n_i of them at index i and centre c_i = (lo_i + hi_i) / 2, the value is
 * (sum over i ascending of n_i c_i) / m and the error (max hi - min lo) / 2, all in
 * round-to-nearest.  (The mean of the cells' centres, summed by index, so the result does
 * not depend on the order the cells come in.) */
static void estimate_groups(const or_grid *g, int level, const uint64_t *keys, const int32_t *votes,
                            int64_t n, int32_t vmax, double p[5], double werr[5], int64_t *m_out) {
    int sh = g->levels - level;
    int64_t m = 0;
    for (int64_t j = 0; j < n; j++) m += votes[j] == vmax;
    for (int ax = 0; ax < 5; ax++) {
        int64_t nb = (int64_t)g->bins[ax] << level;
        int64_t *cnt = (int64_t *)calloc((size_t)nb, sizeof(int64_t));
        for (int64_t j = 0; j < n; j++) {
            if (votes[j] != vmax) continue;
            int32_t idx[5];
            key_to_idx(g, keys[j], idx);
            cnt[idx[ax]]++;
        }
        double sum = 0, lo_min = INFINITY, hi_max = -INFINITY;
        for (int64_t i = 0; i < nb; i++) {
            if (!cnt[i]) continue;
            double lo = g->lo_edge[ax][i << sh];
            double hi = g->hi_edge[ax][((i + 1) << sh) - 1];
            sum += (double)cnt[i] * ((lo + hi) / 2);
            if (lo < lo_min) lo_min = lo;
            if (hi > hi_max) hi_max = hi;
        }
        p[ax] = m ? sum / (double)m : 0.0;
        werr[ax] = m ? (hi_max - lo_min) / 2 : 0.0;
        free(cnt);
    }
    *m_out = m;
}

/* Coarse-to-fine search that keeps whole vote groups (Section 3.3: the result is the set
 * of maximum-vote voxels).  At each level every cell is voted; with vmax the best count,
 * the kept set is {votes >= T} for the smallest T >= max(vmax - slack, min(vmax, 1)) with
 * at most max_keep cells.  If even the vmax group exceeds max_keep, or at the last level,
 * the search ends there and the estimate is taken over that level's vmax group.  Kept cells
 * are bisected along every axis.  prec[L]: as or_vote_cells (with or without
 * OR_OUTGOING).  Outputs: p, werr, *best_votes = vmax, *final_level, *n_final = the size of
 * the final vmax group; trace (may be NULL): per level L <= final level, trace_count[L]
 * cells kept (0 at the final level) and their keys / votes in ascending key order at
 * trace_keys / trace_votes + L * max_keep.  The final level's cells and votes are handed
 * back in *fin_keys / *fin_votes (*fin_n of them; the caller frees them). */
static void maxset_search(const or_grid *g, const or_wires *w, int32_t n_hits, const int32_t *wire_id,
                          const double *drift, const int32_t *prec, int32_t max_keep, int32_t slack,
                          double p[5], double werr[5], int32_t *best_votes, int32_t *final_level,
                          int64_t *n_final, int32_t *trace_count, uint64_t *trace_keys,
                          int32_t *trace_votes, uint64_t **fin_keys, int32_t **fin_votes, int64_t *fin_n) {
    int64_t n = 1;
    for (int a = 0; a < 5; a++) n *= g->bins[a];
    uint64_t *keys = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)n);
    int32_t *votes = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    coarse_keys(g, keys);
    or_vote_cells(g, w, n_hits, wire_id, drift, 0, prec[0], keys, n, votes);
    if (trace_count) for (int L = 0; L <= g->levels; L++) trace_count[L] = 0;
    for (int L = 0;; L++) {
        int32_t vmax = 0;
        for (int64_t j = 0; j < n; j++) if (votes[j] > vmax) vmax = votes[j];
        int64_t cnt[APO_OR_HIST];
        memset(cnt, 0, sizeof(cnt));
        for (int64_t j = 0; j < n; j++) {
            int32_t v = votes[j] < 0 ? 0 : (votes[j] >= APO_OR_HIST ? APO_OR_HIST - 1 : votes[j]);
            cnt[v]++;
        }
        if (L == g->levels || cnt[vmax] > max_keep) {
            estimate_groups(g, L, keys, votes, n, vmax, p, werr, n_final);
            *best_votes = vmax;
            *final_level = L;
            break;
        }
        int32_t lb = vmax - slack;
        int32_t floor1 = vmax < 1 ? vmax : 1;
        if (lb < floor1) lb = floor1;
        int32_t T = vmax;
        int64_t kept = cnt[vmax];
        while (T - 1 >= lb && kept + cnt[T - 1] <= max_keep) { T--; kept += cnt[T]; }
        kv *kk = (kv *)malloc(sizeof(kv) * (size_t)(kept > 0 ? kept : 1));
        int64_t m = 0;
        for (int64_t j = 0; j < n; j++)
            if (votes[j] >= T) { kk[m].key = keys[j]; kk[m].votes = votes[j]; m++; }
        qsort(kk, (size_t)m, sizeof(kv), kv_key_cmp);
        uint64_t *fk = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(m > 0 ? m : 1));
        for (int64_t q = 0; q < m; q++) fk[q] = kk[q].key;
        if (trace_count) {
            trace_count[L] = (int32_t)m;
            for (int64_t q = 0; q < m; q++) {
                trace_keys[(size_t)L * max_keep + q] = kk[q].key;
                trace_votes[(size_t)L * max_keep + q] = kk[q].votes;
            }
        }
        free(kk);
        free(keys);
        free(votes);
        n = m * 32;
        keys = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(n > 0 ? n : 1));
        votes = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
        or_children(g, fk, m, keys);
        free(fk);
        or_vote_cells(g, w, n_hits, wire_id, drift, L + 1, prec[L + 1], keys, n, votes);
    }
    *fin_keys = keys;
    *fin_votes = votes;
    *fin_n = n;
}

int or_solve_event_maxset(const or_grid *g, const or_wires *w, int32_t n_hits, const int32_t *wire_id,
                          const double *drift, const int32_t *prec, int32_t max_keep, int32_t slack,
                          double p[5], double werr[5], int32_t *best_votes, int32_t *final_level,
                          int64_t *n_final, int32_t *trace_count, uint64_t *trace_keys,
                          int32_t *trace_votes) {
    uint64_t *fk;
    int32_t *fv;
    int64_t fn;
    maxset_search(g, w, n_hits, wire_id, drift, prec, max_keep, slack, p, werr, best_votes, final_level,
                  n_final, trace_count, trace_keys, trace_votes, &fk, &fv, &fn);
    free(fk);
    free(fv);
    return 0;
}

/* The vote of one (cell, hit) pair with the drift widened to the interval [d_lo, d_hi]
 * (FP64): used to find the hits of a found track. */
static int vote_pair_drift_iv(const double c[12], const double h[9], double d_lo, double d_hi,
                              int outgoing) {
    iv_d C[6], H[9];
    for (int i = 0; i < 6; i++) C[i] = mk_d(c[2 * i], c[2 * i + 1]);
    for (int i = 0; i < 8; i++) H[i] = mk_d(h[i], h[i]);
    H[8] = mk_d(d_lo, d_hi);
    return vote_program_d(C[0], C[1], C[2], C[3], C[4], C[5], H[0], H[1], H[2], H[3], H[4],
                          H[5], H[6], H[7], H[8], outgoing, NULL);
}

/* Hit finding of Section 3.3 on a set of cells (the final maximum-vote cells of a found
 * track): hit i (with active[i] set, or every hit if active is NULL) is taken when it votes
 * (FP64) for at least one of the n cells (keys at `level`) with its drift widened to
 * [max(d - width, 0), d + width]; the widened end points are rounded outward.  taken[i] = 1
 * for taken hits, otherwise left unchanged.  Must run under FE_DOWNWARD. */
static void mask_hits(const or_grid *g, const or_wires *w, int32_t n_hits, const int32_t *wire_id,
                      const double *drift, const uint8_t *active, int32_t level,
                      const uint64_t *keys, int64_t n, double width, int outgoing, uint8_t *taken) {
    for (int64_t j = 0; j < n; j++) {
        int32_t idx[5];
        double c[12], h[9];
        key_to_idx(g, keys[j], idx);
        cell_intervals(g, level, idx, c);
        for (int32_t i = 0; i < n_hits; i++) {
            if ((active && !active[i]) || taken[i]) continue;
            hit_constants(w, wire_id[i], drift[i], h);
            volatile double lo = drift[i] - width;              /* rounded down */
            volatile double hi = -((-drift[i]) - width);        /* rounded up */
            double dlo = lo > 0 ? lo : 0.0;
            if (vote_pair_drift_iv(c, h, dlo, hi, outgoing)) taken[i] = 1;
        }
    }
}

void or_mask_hits(const or_grid *g, const or_wires *w, int32_t n_hits, const int32_t *wire_id,
                  const double *drift, const uint8_t *active, int32_t level, const uint64_t *keys,
                  int64_t n, double width, int outgoing, uint8_t *taken) {
    int old = fegetround();
    fesetround(FE_DOWNWARD);
    mask_hits(g, w, n_hits, wire_id, drift, active, level, keys, n, width, outgoing, taken);
    fesetround(old);
}

/* Multi-track extraction (the paper's hit finding of Section 3.3, applied to several
 * tracks): search the event's active hits; if the best final vote count is below
 * min_votes or no hit is active, stop; otherwise record the track and deactivate every
 * active hit that votes (FP64) for at least one of the final maximum-vote cells with its
 * drift widened to [max(d - 3 sigma, 0), d + 3 sigma]; repeat up to max_tracks times.
 * 3 sigma is 3.0 * mask_sigma in round-to-nearest; the widened end points are rounded
 * outward.  Outputs per track: p / werr (5 each), votes; *n_found; hit_track[i] = index
 * of the track that masked hit i, or -1. */
int or_solve_event_multi(const or_grid *g, const or_wires *w, int32_t n_hits, const int32_t *wire_id,
                         const double *drift, const int32_t *prec, int32_t max_tracks,
                         int32_t min_votes, double mask_sigma, double *p, double *werr,
                         int32_t *votes, int32_t *n_found, int32_t *hit_track) {
    const double width = 3.0 * mask_sigma;
    const int32_t K = g->topk;
    int32_t *wa = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n_hits > 0 ? n_hits : 1));
    double *da = (double *)malloc(sizeof(double) * (size_t)(n_hits > 0 ? n_hits : 1));
    int32_t *ia = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n_hits > 0 ? n_hits : 1));
    uint64_t *lk = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)K * 32);
    int32_t *lv = (int32_t *)malloc(sizeof(int32_t) * (size_t)K * 32);
    uint64_t *mk = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)K * 32);
    uint8_t *act = (uint8_t *)malloc((size_t)(n_hits > 0 ? n_hits : 1));
    uint8_t *tk = (uint8_t *)malloc((size_t)(n_hits > 0 ? n_hits : 1));
    for (int32_t i = 0; i < n_hits; i++) hit_track[i] = -1;
    *n_found = 0;
    for (int32_t t = 0; t < max_tracks; t++) {
        int32_t na = 0;
        for (int32_t i = 0; i < n_hits; i++)
            if (hit_track[i] < 0) { wa[na] = wire_id[i]; da[na] = drift[i]; ia[na] = i; na++; }
        if (na == 0) break;
        int32_t best = 0;
        or_solve_event(g, w, na, wa, da, prec, p + 5 * t, werr + 5 * t, &best, NULL, NULL, lk, lv);
        if (best < min_votes) break;
        votes[t] = best;
        *n_found = t + 1;
        /* the final maximum-vote cells, in the order of the last level's cells */
        int64_t nmax = 0;
        for (int64_t j = 0; j < (int64_t)K * 32; j++)
            if (lv[j] == best) mk[nmax++] = lk[j];
        for (int32_t i = 0; i < n_hits; i++) { act[i] = hit_track[i] < 0; tk[i] = 0; }
        int old = fegetround();
        fesetround(FE_DOWNWARD);
        mask_hits(g, w, n_hits, wire_id, drift, act, g->levels, mk, nmax, width,
                  (prec[g->levels] & OR_OUTGOING) != 0, tk);
        fesetround(old);
        for (int32_t i = 0; i < n_hits; i++) if (tk[i]) hit_track[i] = t;
    }
    free(wa); free(da); free(ia); free(lk); free(lv); free(mk); free(act); free(tk);
    return 0;
}

/* Vote of one hit for one cell (key at `level`) under precision code prec, as
 * or_vote_cells counts it.  Must run under FE_DOWNWARD. */
static int cell_hit_vote(const or_grid *g, const or_wires *w, int32_t level, int32_t prec, uint64_t key,
                         int32_t wire, double drift) {
    int32_t idx[5];
    double c[12], h[9];
    key_to_idx(g, key, idx);
    cell_intervals(g, level, idx, c);
    hit_constants(w, wire, drift, h);
    return vote_pair(c, h, prec, NULL);
}

/* Multi-track extraction with the max-set search (Section 3.3's hit finding applied to
 * several tracks, as or_solve_event_multi).  Round t searches the hits no earlier track
 * took; if none is left, or the final vmax is below min_votes, the extraction stops.
 * Otherwise the final vmax group can hold the cells of several tracks (tracks with equal
 * hit counts tie), so the round takes one of them: the seed is the group's lowest key, S
 * the searched hits that vote for it (vmax of them, at the final level's precision), and
 * the track's cells are the group's cells that every hit of S votes for (each has vmax
 * votes, so its voting hits are exactly S).  Track t is the estimate over those cells (p,
 * werr as or_solve_event_maxset, votes = vmax, final level, n_final = their number); it
 * takes the hits of S and every other hit still active that votes (FP64) for at least one
 * of its cells with the drift widened to [max(d - 3 sigma, 0), d + 3 sigma] (direction
 * condition as the final level's precision code).  Up to max_tracks rounds.
 * hit_track[i]: the track that took hit i, or -1. */
int or_solve_event_maxset_multi(const or_grid *g, const or_wires *w, int32_t n_hits, const int32_t *wire_id,
                                const double *drift, const int32_t *prec, int32_t max_keep, int32_t slack,
                                int32_t max_tracks, int32_t min_votes, double mask_sigma, double *p,
                                double *werr, int32_t *votes, int32_t *final_level, int64_t *n_final,
                                int32_t *n_found, int32_t *hit_track) {
    const double width = 3.0 * mask_sigma;
    size_t nb = (size_t)(n_hits > 0 ? n_hits : 1);
    int32_t *wa = (int32_t *)malloc(sizeof(int32_t) * nb);
    double *da = (double *)malloc(sizeof(double) * nb);
    int32_t *ia = (int32_t *)malloc(sizeof(int32_t) * nb);
    uint8_t *sv = (uint8_t *)malloc(nb);
    uint8_t *act = (uint8_t *)malloc(nb);
    uint8_t *tk = (uint8_t *)malloc(nb);
    for (int32_t i = 0; i < n_hits; i++) hit_track[i] = -1;
    *n_found = 0;
    for (int32_t t = 0; t < max_tracks; t++) {
        int32_t na = 0;
        for (int32_t i = 0; i < n_hits; i++)
            if (hit_track[i] < 0) { wa[na] = wire_id[i]; da[na] = drift[i]; ia[na] = i; na++; }
        if (na == 0) break;
        int32_t best = 0, fl = 0;
        int64_t nf = 0, fn = 0;
        uint64_t *fk;
        int32_t *fv;
        double pt[5], wt[5];
        maxset_search(g, w, na, wa, da, prec, max_keep, slack, pt, wt, &best, &fl, &nf, NULL, NULL, NULL,
                      &fk, &fv, &fn);
        if (best < min_votes) { free(fk); free(fv); break; }
        /* the final vmax group and its lowest key */
        int64_t m = 0;
        for (int64_t j = 0; j < fn; j++)
            if (fv[j] == best) fk[m++] = fk[j];
        uint64_t seed = fk[0];
        for (int64_t j = 1; j < m; j++) if (fk[j] < seed) seed = fk[j];
        int old = fegetround();
        fesetround(FE_DOWNWARD);
        for (int32_t q = 0; q < na; q++) sv[q] = (uint8_t)cell_hit_vote(g, w, fl, prec[fl], seed, wa[q], da[q]);
        /* the track's cells: the group's cells that every hit of S votes for (in place) */
        int64_t mc = 0;
        for (int64_t j = 0; j < m; j++) {
            int ok = 1;
            for (int32_t q = 0; q < na && ok; q++)
                if (sv[q] && !cell_hit_vote(g, w, fl, prec[fl], fk[j], wa[q], da[q])) ok = 0;
            if (ok) fk[mc++] = fk[j];
        }
        fesetround(old);
        for (int64_t j = 0; j < mc; j++) fv[j] = best;
        estimate_groups(g, fl, fk, fv, mc, best, pt, wt, &nf);
        for (int a = 0; a < 5; a++) { p[5 * t + a] = pt[a]; werr[5 * t + a] = wt[a]; }
        votes[t] = best;
        final_level[t] = fl;
        n_final[t] = nf;
        *n_found = t + 1;
        for (int32_t i = 0; i < n_hits; i++) { act[i] = hit_track[i] < 0; tk[i] = 0; }
        for (int32_t q = 0; q < na; q++) if (sv[q]) tk[ia[q]] = 1;
        old = fegetround();
        fesetround(FE_DOWNWARD);
        mask_hits(g, w, n_hits, wire_id, drift, act, fl, fk, mc, width, (prec[fl] & OR_OUTGOING) != 0, tk);
        fesetround(old);
        for (int32_t i = 0; i < n_hits; i++) if (tk[i]) hit_track[i] = t;
        free(fk);
        free(fv);
    }
    free(wa); free(da); free(ia); free(sv); free(act); free(tk);
    return 0;
}

int or_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void or_set_num_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* Directed operations of one full evaluation of the vote program, by phase (per cell,
 * per (cell, hit) without tan(lambda), tan(lambda)-dependent, both drift signs). */
void or_op_counts(const double cell[12], const double hit[9], int prec, unsigned long long out[4]) {
    int old = fegetround();
    fesetround(FE_DOWNWARD);
    for (int i = 0; i < 4; i++) { opcnt_d[i] = 0; opcnt_f[i] = 0; }
    vote_pair(cell, hit, prec, NULL);
    for (int i = 0; i < 4; i++) out[i] = prec == 0 ? opcnt_d[i] : opcnt_f[i];
    fesetround(old);
}

/* ------------------------------------------------------------------------------------ */
/* Exported for the pin tests: the transcendental enclosures on their own.               */
/* ------------------------------------------------------------------------------------ */
void or_atan_iv(double lo, double hi, int prec, double out[2]) {
    int old = fegetround();
    fesetround(FE_DOWNWARD);
    if (prec == 0) {
        iv_d r = atan_iv_d(mk_d(lo, hi));
        out[0] = r.lo; out[1] = r.hi;
    } else {
        iv_f r = atan_iv_f(mk_f(rd32(lo), ru32(hi)));
        out[0] = r.lo; out[1] = r.hi;
    }
    fesetround(old);
}

void or_sincos_iv(double lo, double hi, int prec, double out[4]) {
    int old = fegetround();
    fesetround(FE_DOWNWARD);
    if (prec == 0) {
        iv_d s, c;
        sincos_iv_d(mk_d(lo, hi), &s, &c);
        out[0] = s.lo; out[1] = s.hi; out[2] = c.lo; out[3] = c.hi;
    } else {
        iv_f s, c;
        sincos_iv_f(mk_f(rd32(lo), ru32(hi)), &s, &c);
        out[0] = s.lo; out[1] = s.hi; out[2] = c.lo; out[3] = c.hi;
    }
    fesetround(old);
}


/* ==================================================================================== */
/* The paper's own 4-D search (Sections 3.1-3.3, Table tabGridDef): voxels x_c x y_c x R  */
/* x z0 with two tan(lambda)-sign accumulators, the disk pre-filter, the midpoint form,  */
/* and three iterations with hit finding and a moving reference point.                  */
/* ==================================================================================== */

/* one iteration's grid for one event: axis a has n[a] voxels [lo + i w, lo + (i + 1) w] */
typedef struct { double lo[4], w[4]; int32_t n[4]; } or4_grid;

typedef struct {
    double p_gev, b_tesla, disk_radius, hit_factor;
    double glo[4];            /* lower corner of the global box of iterations 1 and 2 */
    double w[3][4];           /* voxel size per iteration */
    int32_t n[3][4];          /* voxels per axis per iteration */
    int32_t precision;        /* 0: FP64, 1: FP32 */
    int32_t n_iter;           /* 1 .. 3 */
    int32_t per_sign;         /* 1: iteration 3 searches each sign around its own estimate */
} or4_opts;

typedef struct {
    double value[4], err[4], ref[2];
    int32_t sign, vmax, n_max, n_sel;
} or4_iter;

/* voxel edges (round to nearest; the caller holds FE_TONEAREST) */
static void v4_edge(const or4_grid *g, int a, int i, double *lo, double *hi) {
    *lo = g->lo[a] + (double)i * g->w[a];
    *hi = g->lo[a] + (double)(i + 1) * g->w[a];
}

/* The vote of one hit for one voxel centre (m, the prefix at its z0, sign) and the
 * voxel's intervals X, Y, Rv, Z (either drift sign; a guard votes). */
static int v4_pair_d(const v4ctr_d *m, const v4pre_d *pre, int sign, const double h[9], iv_d X, iv_d Y,
                     iv_d Rv, iv_d Z) {
    double dax[2];
    int g = v4_dax_d(pre, sign > 0 ? m->aL : -m->aL, h, dax);
    fesetround(FE_DOWNWARD);
    int v = 0;
    for (int sg = 0; sg < 2 && !v; sg++)
        v = (g >> sg & 1) ? 1 : v4_test_d(X, Y, Rv, Z, mk_d(h[0], h[0]), mk_d(h[1], h[1]),
                                          mk_d(h[5], h[5]), mk_d(h[6], h[6]), dax[sg]);
    fesetround(FE_TONEAREST);
    return v;
}
static int v4_pair_f(const v4ctr_f *m, const v4pre_f *pre, int sign, const float hf[9], const double h[9],
                     iv_f X, iv_f Y, iv_f Rv, iv_f Z) {
    float dax[2];
    int g = v4_dax_f(pre, sign > 0 ? m->aL : -m->aL, hf, dax);
    fesetround(FE_DOWNWARD);
    iv_f x0 = mk_f(rd32(h[0]), ru32(h[0])), y0 = mk_f(rd32(h[1]), ru32(h[1]));
    iv_f spt = mk_f(rd32(h[5]), ru32(h[5])), cpt = mk_f(rd32(h[6]), ru32(h[6]));
    int v = 0;
    for (int sg = 0; sg < 2 && !v; sg++)
        v = (g >> sg & 1) ? 1 : v4_test_f(X, Y, Rv, Z, x0, y0, spt, cpt, dax[sg]);
    fesetround(FE_TONEAREST);
    return v;
}

/* Votes of every voxel of grid g for one event, both signs: votes[s * nvox + lin] with
 * lin = ix + nx (iy + ny (iR + nR iz)), s = 0 for tan(lambda) > 0.  active (may be NULL):
 * 1 for the hits that vote.  Voxels outside the disk (Eq. ApoVoteDisk) or without a real
 * tan(lambda) at their centre get 0. */
void or4_vote_grid(const or4_opts *o, const or4_grid *g, const double ref[2], const or_wires *w,
                   int32_t n_hits, const int32_t *wire_id, const double *drift,
                   const uint8_t *active, int32_t *votes) {
    const int nx = g->n[0], ny = g->n[1], nR = g->n[2], nz = g->n[3];
    const int64_t nvox = (int64_t)nx * ny * nR * nz;
    const int64_t ncol = (int64_t)nx * ny * nR;
    #pragma omp parallel
    {
        int old = fegetround();
        fesetround(FE_TONEAREST);
        double *hc = (double *)malloc(sizeof(double) * 9 * (size_t)(n_hits > 0 ? n_hits : 1));
        for (int32_t i = 0; i < n_hits; i++) hit_constants(w, wire_id[i], drift[i], hc + 9 * i);
        #pragma omp for schedule(dynamic, 64)
        for (int64_t col = 0; col < ncol; col++) {
            const int ix = (int)(col % nx), iy = (int)((col / nx) % ny), iR = (int)(col / ((int64_t)nx * ny));
            double xl, xh, yl, yh, rl, rh;
            v4_edge(g, 0, ix, &xl, &xh);
            v4_edge(g, 1, iy, &yl, &yh);
            v4_edge(g, 2, iR, &rl, &rh);
            const double xc = (xl + xh) * 0.5, yc = (yl + yh) * 0.5, Rc = (rl + rh) * 0.5;
            int32_t cnt[2][64];
            memset(cnt, 0, sizeof(cnt));
            fesetround(FE_DOWNWARD);
            int in_disk;
            iv_d Xd = mk_d(xl, xh), Yd = mk_d(yl, yh), Rd = mk_d(rl, rh);
            iv_f Xf = mk_f(rd32(xl), ru32(xh)), Yf = mk_f(rd32(yl), ru32(yh)), Rf = mk_f(rd32(rl), ru32(rh));
            if (o->precision == 0) in_disk = v4_disk_d(Xd, Yd, Rd, o->disk_radius);
            else in_disk = v4_disk_f(Xf, Yf, Rf, ru32(o->disk_radius));
            fesetround(FE_TONEAREST);
            if (in_disk) {
                if (o->precision == 0) {
                    v4ctr_d m = v4_centre_d(xc, yc, Rc, o->p_gev, o->b_tesla, ref[0], ref[1]);
                    if (m.valid)
                        for (int32_t i = 0; i < n_hits; i++) {
                            if (active && !active[i]) continue;
                            const double *h = hc + 9 * i;
                            for (int iz = 0; iz < nz; iz++) {
                                double zl, zh;
                                v4_edge(g, 3, iz, &zl, &zh);
                                const double zc = (zl + zh) * 0.5;
                                v4pre_d pre = v4_prefix_d(&m, zc, h);
                                iv_d Zd = mk_d(zl, zh);
                                for (int s = 0; s < 2; s++)
                                    cnt[s][iz] += pre.guard ? 1 : v4_pair_d(&m, &pre, s == 0 ? 1 : -1, h, Xd, Yd, Rd, Zd);
                            }
                        }
                } else {
                    v4ctr_f m = v4_centre_f((float)xc, (float)yc, (float)Rc, (float)o->p_gev,
                                            (float)o->b_tesla, (float)ref[0], (float)ref[1]);
                    if (m.valid)
                        for (int32_t i = 0; i < n_hits; i++) {
                            if (active && !active[i]) continue;
                            const double *h = hc + 9 * i;
                            float hf[9];
                            for (int k = 0; k < 9; k++) hf[k] = (float)h[k];
                            for (int iz = 0; iz < nz; iz++) {
                                double zl, zh;
                                v4_edge(g, 3, iz, &zl, &zh);
                                const float zc = (float)((zl + zh) * 0.5);
                                v4pre_f pre = v4_prefix_f(&m, zc, hf);
                                fesetround(FE_DOWNWARD);
                                iv_f Zf = mk_f(rd32(zl), ru32(zh));
                                fesetround(FE_TONEAREST);
                                for (int s = 0; s < 2; s++)
                                    cnt[s][iz] += pre.guard ? 1 : v4_pair_f(&m, &pre, s == 0 ? 1 : -1, hf, h, Xf, Yf, Rf, Zf);
                            }
                        }
                }
            }
            for (int s = 0; s < 2; s++)
                for (int iz = 0; iz < nz; iz++)
                    votes[(int64_t)s * nvox + col + ncol * iz] = cnt[s][iz];
        }
        free(hc);
        fesetround(old);
    }
}

/* Values and errors over the maximum-vote voxels of one sign's accumulator (s = 0 for
 * tan(lambda) > 0), Section 3.3: over its m maximum-vote voxels, value_a = lo_a + w_a (S_a / m
 * + 1/2) with S_a the sum of their indices on axis a (exact integers), error_a = w_a (i_max -
 * i_min + 1) / 2. */
static void v4_estimate_sign(const or4_grid *g, const int32_t *votes, int s, or4_iter *it) {
    const int64_t nvox = (int64_t)g->n[0] * g->n[1] * g->n[2] * g->n[3];
    int32_t vm = 0;
    for (int64_t j = 0; j < nvox; j++)
        if (votes[s * nvox + j] > vm) vm = votes[s * nvox + j];
    it->sign = s == 0 ? 1 : -1;
    it->vmax = vm;
    int64_t m = 0, S[4] = {0, 0, 0, 0};
    int32_t imin[4], imax[4];
    for (int a = 0; a < 4; a++) { imin[a] = g->n[a]; imax[a] = -1; }
    for (int64_t j = 0; j < nvox; j++) {
        if (votes[s * nvox + j] != vm) continue;
        int32_t idx[4];
        int64_t r = j;
        for (int a = 0; a < 4; a++) { idx[a] = (int32_t)(r % g->n[a]); r /= g->n[a]; }
        m++;
        for (int a = 0; a < 4; a++) {
            S[a] += idx[a];
            if (idx[a] < imin[a]) imin[a] = idx[a];
            if (idx[a] > imax[a]) imax[a] = idx[a];
        }
    }
    it->n_max = (int32_t)m;
    for (int a = 0; a < 4; a++) {
        double mu = (double)S[a] / (double)m;
        it->value[a] = g->lo[a] + g->w[a] * (mu + 0.5);
        it->err[a] = (g->w[a] * (double)(imax[a] + 1 - imin[a])) * 0.5;
    }
}

static int32_t v4_vmax_sign(const or4_grid *g, const int32_t *votes, int s) {
    const int64_t nvox = (int64_t)g->n[0] * g->n[1] * g->n[2] * g->n[3];
    int32_t vm = 0;
    for (int64_t j = 0; j < nvox; j++)
        if (votes[s * nvox + j] > vm) vm = votes[s * nvox + j];
    return vm;
}

/* Values and errors of one iteration: the sign whose accumulator has the larger maximum
 * (the paper's choice of the tan(lambda) sign; ties: tan(lambda) > 0), estimated as above. */
static void v4_estimate(const or4_grid *g, const int32_t *votes, or4_iter *it) {
    const int s = v4_vmax_sign(g, votes, 0) >= v4_vmax_sign(g, votes, 1) ? 0 : 1;
    v4_estimate_sign(g, votes, s, it);
}

/* exported for the pins: the disk pre-filter of one voxel (x_c, y_c, R lo / hi) */
int or4_disk(const double box[6], double radius, int32_t prec) {
    int old = fegetround();
    fesetround(FE_DOWNWARD);
    int r = prec == 0 ? v4_disk_d(mk_d(box[0], box[1]), mk_d(box[2], box[3]), mk_d(box[4], box[5]), radius)
                      : v4_disk_f(mk_f(rd32(box[0]), ru32(box[1])), mk_f(rd32(box[2]), ru32(box[3])),
                                  mk_f(rd32(box[4]), ru32(box[5])), ru32(radius));
    fesetround(old);
    return r;
}

/* exported for the pins */
void or4_estimate(const or4_grid *g, const int32_t *votes, or4_iter *it) {
    int old = fegetround();
    fesetround(FE_TONEAREST);
    v4_estimate(g, votes, it);
    fesetround(old);
}

/* Hit finding (Section 3.3): the box value +- factor * error, the chosen sign; a hit is
 * taken when the vote holds on that box (same form as the voting). */
static int v4_find_hits(const or4_opts *o, const or4_iter *it, const double ref[2], const or_wires *w,
                        int32_t n_hits, const int32_t *wire_id, const double *drift, uint8_t *sel) {
    double lo[4], hi[4], c[4];
    for (int a = 0; a < 4; a++) {
        double r = o->hit_factor * it->err[a];
        lo[a] = it->value[a] - r;
        hi[a] = it->value[a] + r;
        c[a] = (lo[a] + hi[a]) * 0.5;
    }
    int n = 0;
    for (int32_t i = 0; i < n_hits; i++) {
        double h[9];
        hit_constants(w, wire_id[i], drift[i], h);
        int v = 0;
        if (o->precision == 0) {
            v4ctr_d m = v4_centre_d(c[0], c[1], c[2], o->p_gev, o->b_tesla, ref[0], ref[1]);
            if (m.valid) {
                v4pre_d pre = v4_prefix_d(&m, c[3], h);
                v = pre.guard ? 1 : v4_pair_d(&m, &pre, it->sign, h, mk_d(lo[0], hi[0]),
                                              mk_d(lo[1], hi[1]), mk_d(lo[2], hi[2]), mk_d(lo[3], hi[3]));
            }
        } else {
            v4ctr_f m = v4_centre_f((float)c[0], (float)c[1], (float)c[2], (float)o->p_gev,
                                    (float)o->b_tesla, (float)ref[0], (float)ref[1]);
            if (m.valid) {
                float hf[9];
                for (int k = 0; k < 9; k++) hf[k] = (float)h[k];
                v4pre_f pre = v4_prefix_f(&m, (float)c[3], hf);
                fesetround(FE_DOWNWARD);
                iv_f X = mk_f(rd32(lo[0]), ru32(hi[0])), Y = mk_f(rd32(lo[1]), ru32(hi[1]));
                iv_f Rv = mk_f(rd32(lo[2]), ru32(hi[2])), Z = mk_f(rd32(lo[3]), ru32(hi[3]));
                fesetround(FE_TONEAREST);
                v = pre.guard ? 1 : v4_pair_f(&m, &pre, it->sign, hf, h, X, Y, Rv, Z);
            }
        }
        sel[i] = (uint8_t)v;
        n += v;
    }
    return n;
}

/* New reference point: the waist point of the selected hit nearest to the found circle,
 * | |(x0, y0) - (x_c, y_c)| - R | (first on ties); unchanged if no hit is selected. */
static void v4_new_ref(const or4_iter *it, const or_wires *w, int32_t n_hits, const int32_t *wire_id,
                       const uint8_t *sel, double ref[2]) {
    double best = INFINITY;
    int bi = -1;
    for (int32_t i = 0; i < n_hits; i++) {
        if (!sel[i]) continue;
        double dx = w->x0[wire_id[i]] - it->value[0], dy = w->y0[wire_id[i]] - it->value[1];
        double dist = fabs(sqrt(dx * dx + dy * dy) - it->value[2]);
        if (dist < best) { best = dist; bi = i; }
    }
    if (bi >= 0) { ref[0] = w->x0[wire_id[bi]]; ref[1] = w->y0[wire_id[bi]]; }
}

/* z0 of the found helix moved from reference point a to b: z0 + tan(lambda) R dpsi, dpsi
 * the phase of b minus that of a, both from the direction of the origin (as in the vote;
 * 0 if either is undefined). */
static double v4_move_z0(const or4_opts *o, const or4_iter *it, const double a[2], const double b[2]) {
    double xc = it->value[0], yc = it->value[1], R = it->value[2];
    double ox = -xc, oy = -yc, on = sqrt(ox * ox + oy * oy);
    int bad = !(on > 0);
    double ax = a[0] - xc, ay = a[1] - yc, bx = b[0] - xc, by = b[1] - yc;
    double pa = bad ? 0.0 : v4_phase_d(ox, oy, on, ax, ay, sqrt(ax * ax + ay * ay), &bad);
    double pb = bad ? 0.0 : v4_phase_d(ox, oy, on, bx, by, sqrt(bx * bx + by * by), &bad);
    double dpsi = bad ? 0.0 : pb - pa;
    double ratio = o->p_gev / ((0.3 * o->b_tesla) * R);
    double aL = ratio > 1 ? sqrt(ratio * ratio - 1.0) : 0.0;
    double L = it->sign > 0 ? aL : -aL;
    return it->value[3] + L * (R * dpsi);
}

/* The three iterations for one event (Section 3.3): iteration 1 on the global grid with the
 * reference point at the origin and every hit; iteration 2 on the global grid with finer
 * voxels, the reference point moved to the selected hit nearest to the found circle and
 * only the selected hits; iteration 3 on the box centred on iteration 2's values (z0 moved
 * to the new reference point) with the finest voxels.  Hit finding after each iteration
 * looks at every hit.  With o->per_sign, iteration 3 reads "the value determined by the
 * previous step" per accumulator: each tan(lambda) sign takes the estimate of its own
 * accumulator of iteration 2, its hit finding, reference point and centred box, and votes
 * on that box with its own selected hits; the sign with the larger maximum then gives the
 * result as before.  out: n_iter records; sel_out (may be NULL): the last selection. */
int or4_solve_event(const or4_opts *o, const or_wires *w, int32_t n_hits, const int32_t *wire_id,
                    const double *drift, or4_iter *out, uint8_t *sel_out) {
    int old = fegetround();
    fesetround(FE_TONEAREST);
    size_t nb = (size_t)(n_hits > 0 ? n_hits : 1);
    uint8_t *act = (uint8_t *)malloc(nb);
    uint8_t *sel = (uint8_t *)malloc(nb);
    for (int32_t i = 0; i < n_hits; i++) act[i] = 1;
    double ref[2] = {0.0, 0.0};
    or4_grid g;
    int32_t *prev_votes = NULL;   /* iteration 2's accumulators (per-sign iteration 3) */
    or4_grid prev_g;
    double prev_ref[2] = {0.0, 0.0};
    for (int k = 0; k < o->n_iter && k < 3; k++) {
        for (int a = 0; a < 4; a++) { g.w[a] = o->w[k][a]; g.n[a] = o->n[k][a]; }
        const int64_t nvox = (int64_t)g.n[0] * g.n[1] * g.n[2] * g.n[3];
        if (k == 2 && o->per_sign) {
            or4_grid gs[2];
            int32_t *vs[2];
            double rs[2][2];
            uint8_t *ss[2];
            for (int s = 0; s < 2; s++) {
                or4_iter es;
                v4_estimate_sign(&prev_g, prev_votes, s, &es);
                ss[s] = (uint8_t *)malloc(nb);
                v4_find_hits(o, &es, prev_ref, w, n_hits, wire_id, drift, ss[s]);
                fesetround(FE_TONEAREST);
                double ref_n[2] = {prev_ref[0], prev_ref[1]};
                v4_new_ref(&es, w, n_hits, wire_id, ss[s], ref_n);
                double c[4] = {es.value[0], es.value[1], es.value[2], v4_move_z0(o, &es, prev_ref, ref_n)};
                gs[s] = g;
                for (int a = 0; a < 4; a++) gs[s].lo[a] = c[a] - ((double)g.n[a] * g.w[a]) * 0.5;
                rs[s][0] = ref_n[0];
                rs[s][1] = ref_n[1];
                vs[s] = (int32_t *)malloc(sizeof(int32_t) * (size_t)(2 * nvox));
                or4_vote_grid(o, &gs[s], rs[s], w, n_hits, wire_id, drift, ss[s], vs[s]);
                fesetround(FE_TONEAREST);
            }
            const int sc = v4_vmax_sign(&gs[0], vs[0], 0) >= v4_vmax_sign(&gs[1], vs[1], 1) ? 0 : 1;
            v4_estimate_sign(&gs[sc], vs[sc], sc, &out[k]);
            ref[0] = rs[sc][0];
            ref[1] = rs[sc][1];
            for (int s = 0; s < 2; s++) { free(vs[s]); free(ss[s]); }
        } else {
            if (k < 2) {
                for (int a = 0; a < 4; a++) g.lo[a] = o->glo[a];
            } else {
                double ref_n[2] = {ref[0], ref[1]};
                v4_new_ref(&out[k - 1], w, n_hits, wire_id, sel, ref_n);
                double c[4] = {out[k - 1].value[0], out[k - 1].value[1], out[k - 1].value[2],
                               v4_move_z0(o, &out[k - 1], ref, ref_n)};
                ref[0] = ref_n[0]; ref[1] = ref_n[1];
                for (int a = 0; a < 4; a++) g.lo[a] = c[a] - ((double)g.n[a] * g.w[a]) * 0.5;
            }
            if (k == 1) v4_new_ref(&out[0], w, n_hits, wire_id, sel, ref);
            int32_t *votes = (int32_t *)malloc(sizeof(int32_t) * (size_t)(2 * nvox));
            or4_vote_grid(o, &g, ref, w, n_hits, wire_id, drift, act, votes);
            fesetround(FE_TONEAREST);
            v4_estimate(&g, votes, &out[k]);
            if (k == 1 && o->per_sign) {
                prev_votes = votes;
                prev_g = g;
                prev_ref[0] = ref[0];
                prev_ref[1] = ref[1];
            } else {
                free(votes);
            }
        }
        out[k].ref[0] = ref[0];
        out[k].ref[1] = ref[1];
        out[k].n_sel = v4_find_hits(o, &out[k], ref, w, n_hits, wire_id, drift, sel);
        fesetround(FE_TONEAREST);
        for (int32_t i = 0; i < n_hits; i++) act[i] = sel[i];
    }
    if (sel_out) memcpy(sel_out, sel, (size_t)n_hits);
    free(prev_votes);
    free(act);
    free(sel);
    fesetround(old);
    return 0;
}

/* One pair of the 4-D midpoint form (for the pins): box = (x_c, y_c, R, z0) lo/hi,
 * sign of tan(lambda), reference point, hit; out (may be NULL): d^Ax+, d^Ax-, guard flags,
 * |tan(lambda)| at the centre, psi. */
int or4_vote_pair(const double box[8], int32_t sign, const double ref[2], const double hit[9],
                  double p_gev, double b_tesla, int32_t prec, double out[5]) {
    int old = fegetround();
    fesetround(FE_TONEAREST);
    double c[4];
    for (int a = 0; a < 4; a++) c[a] = (box[2 * a] + box[2 * a + 1]) * 0.5;
    int v = 0;
    if (out) for (int i = 0; i < 5; i++) out[i] = 0;
    if (prec == 0) {
        v4ctr_d m = v4_centre_d(c[0], c[1], c[2], p_gev, b_tesla, ref[0], ref[1]);
        if (m.valid) {
            v4pre_d pre = v4_prefix_d(&m, c[3], hit);
            if (out) { out[3] = m.aL; out[4] = pre.psi; }
            if (pre.guard) { v = 1; if (out) out[2] = 3; }
            else {
                double dax[2];
                int gflag = v4_dax_d(&pre, sign > 0 ? m.aL : -m.aL, hit, dax);
                if (out) { out[0] = dax[0]; out[1] = dax[1]; out[2] = gflag; }
                v = v4_pair_d(&m, &pre, sign, hit, mk_d(box[0], box[1]), mk_d(box[2], box[3]),
                              mk_d(box[4], box[5]), mk_d(box[6], box[7]));
            }
        }
    } else {
        v4ctr_f m = v4_centre_f((float)c[0], (float)c[1], (float)c[2], (float)p_gev, (float)b_tesla,
                                (float)ref[0], (float)ref[1]);
        if (m.valid) {
            float hf[9];
            for (int k = 0; k < 9; k++) hf[k] = (float)hit[k];
            v4pre_f pre = v4_prefix_f(&m, (float)c[3], hf);
            if (out) { out[3] = m.aL; out[4] = pre.psi; }
            if (pre.guard) { v = 1; if (out) out[2] = 3; }
            else {
                float dax[2];
                int gflag = v4_dax_f(&pre, sign > 0 ? m.aL : -m.aL, hf, dax);
                if (out) { out[0] = dax[0]; out[1] = dax[1]; out[2] = gflag; }
                fesetround(FE_DOWNWARD);
                iv_f X = mk_f(rd32(box[0]), ru32(box[1])), Y = mk_f(rd32(box[2]), ru32(box[3]));
                iv_f Rv = mk_f(rd32(box[4]), ru32(box[5])), Z = mk_f(rd32(box[6]), ru32(box[7]));
                fesetround(FE_TONEAREST);
                v = v4_pair_f(&m, &pre, sign, hf, hit, X, Y, Rv, Z);
            }
        }
    }
    fesetround(old);
    return v;
}
