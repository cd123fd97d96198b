/* C ABI of the paper's own search on a 4-D voxel grid (arXiv:2401.04576, Sections 3.1-3.3,
 * Tables tabGridDef and HelixParametes), in libapo.so next to the 5-D path of apo.h.
 *
 * Voxels are x_c x y_c x R x z0 (metres): the helix's circle centre and radius, and its z
 * at the point of the circle nearest a reference point (x_ref, y_ref).  The momentum is
 * fixed, so tan(lambda) = +-sqrt((p / (0.3 B R))^2 - 1), one vote accumulator per sign
 * (Section 3.1).  A voxel is considered only if it passes the disk pre-filter of
 * Eq. ApoVoteDisk (the circle may pass within disk_radius of the origin); it gets one vote
 * per hit for which 0 lies in (x^Ax - x_c)^2 + (y^Ax - y_c)^2 - (R + d^Ax)^2 (Eq. ApoVote)
 * with x_c, y_c, R over the voxel and d^Ax (Eq. defdiAX_b) evaluated at the voxel centre:
 * the midpoint form the paper times.  The transverse reference plane is z = 0 (the wire
 * point is its waist point).  Each iteration takes, in the accumulator with the larger
 * maximum, the mean index and extent of the maximum-vote voxels as value and error
 * (Section 3.3), then finds the event's hits on the box value +- hit_factor * error.
 * Iteration 1 uses the global grid, the origin as reference point and every hit;
 * iteration 2 the global grid with smaller voxels, the reference point moved to the
 * selected hit nearest the found circle and only the selected hits; iteration 3 a box
 * centred on iteration 2's values (z0 moved to the new reference point).
 *
 * Every call returns an apo_status and never aborts; device work runs on the caller's
 * stream; the caller owns every buffer.  There is no CPU fallback.
 */
#ifndef APO4_H
#define APO4_H

#include <stddef.h>
#include <stdint.h>

#include "apo.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct apo4_chamber apo4_chamber;

/* Search settings.  Iteration k (0-based) uses n[k][a] voxels of size w[k][a] on axis a
 * (x_c, y_c, R, z0); iterations 0 and 1 start at glo, iteration 2 at its centre minus
 * n w / 2.  Limits: 1 <= n[k][a] <= 4096, n[k][3] <= 32, n[k][0] n[k][1] n[k][2] n[k][3]
 * <= 2^28, w > 0; precision APO_F64 or APO_F32 (point and interval parts of the vote);
 * 1 <= n_iter <= 3. */
typedef struct {
    double p_gev;          /* momentum [GeV/c] */
    double b_tesla;        /* field [T] */
    double disk_radius;    /* Eq. ApoVoteDisk: [-r, r] around the origin [m] */
    double hit_factor;     /* hit finding on value +- hit_factor * error */
    double glo[4];
    double w[3][4];
    int32_t n[3][4];
    int32_t precision;
    int32_t n_iter;
    int32_t per_sign;      /* 1 (default): with three iterations, iteration 3 searches each
                              tan(lambda) sign around its own accumulator's estimate of
                              iteration 2 (its own hit finding, reference point, z0 carry
                              and box), then keeps the sign with the larger maximum; 0: both
                              signs on the box of iteration 2's chosen sign */
} apo4_opts;

/* One iteration's result for one event.  value / err: x_c, y_c, R, z0 (z0 at ref); ref:
 * the reference point used; sign: of tan(lambda) (+1 / -1); vmax: the maximum vote count;
 * n_max: voxels at it; n_sel: hits found on the box after the iteration.  An event with a
 * malformed hit gets vmax = APO_EINVAL and no selected hit. */
typedef struct {
    double value[4];
    double err[4];
    double ref[2];
    int32_t sign;
    int32_t vmax;
    int32_t n_max;
    int32_t n_sel;
} apo4_iter;

/* Table tabGridDef in metres with z0 centred on the chamber middle, p = 0.105 GeV/c,
 * B = 1 T, disk radius 0.1 m, hit factor 5, FP64, three iterations, per_sign 1. */
void apo4_opts_default(apo4_opts *opts);

/* Uploads the wire table (as for apo_geometry_create). */
int apo4_chamber_create(const apo_wires *wires, apo4_chamber **out);
void apo4_chamber_destroy(apo4_chamber *chamber);

/* Device workspace apo4_solve_batch / apo4_vote need for n_events. */
int apo4_workspace_bytes(const apo4_chamber *chamber, int32_t n_events, const apo4_opts *opts,
                         size_t *bytes);

/* All iterations for a batch.  out: device, n_events x n_iter records (event-major).
 * selected (device, may be NULL): per hit of the batch (CSR order), 1 if the last
 * iteration's hit finding took it. */
int apo4_solve_batch(const apo4_chamber *chamber, const apo_hits *hits, const apo4_opts *opts,
                     apo4_iter *out, uint8_t *selected, void *workspace, size_t workspace_bytes,
                     void *stream);

/* Votes of one grid (n[iter], w[iter] of opts) for every event: lo (device, n_events x 4)
 * the lower corner per event, ref (device, n_events x 2) the reference point per event,
 * active (device, per hit, may be NULL = every hit) 1 for the hits that vote.
 * votes: device, n_events x 2 x nvox int32, index (event, sign, z0, R, y_c, x_c) with
 * sign 0 for tan(lambda) > 0; voxels outside the disk or without a real tan(lambda) at
 * their centre get 0. */
int apo4_vote(const apo4_chamber *chamber, const apo_hits *hits, const apo4_opts *opts,
              int32_t iter, const double *lo, const double *ref, const uint8_t *active,
              int32_t *votes, void *workspace, size_t workspace_bytes, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* APO4_H */
