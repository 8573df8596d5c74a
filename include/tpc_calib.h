/*
 * tpc_calib.h -- C ABI of the calibration chi2 of the refit and of its
 * adjoint (gradient with respect to the calibration parameters).
 *
 * Paper: section "Tracking" (continuous read-out: the drift time is turned
 * into z with the drift velocity; once the collision time is fixed by
 * matching, the final refit applies the calibration under the primary-track
 * assumption) and section "TPC Tracking" (online drift-velocity
 * calibration).  The paper gives no formulas for this part; the model below
 * is this library's reading.
 *
 * Calibration parameters theta (binary32, device, TPC_CALIB_N_THETA(ns)):
 *   theta[0] = v, drift velocity (cm/us); theta[1] = t0, time offset (us);
 *   theta[2 + ((s*8 + i)*8 + j)*2 + k] = spline coefficient of sector s,
 *   i along u = (x - x_first)/(x_last - x_first) (pad-row radius), j along
 *   w = |z|/z_max, k = 0: dy, k = 1: dz (cm), of an 8 x 8 uniform clamped
 *   cubic B-spline per sector.
 * A cluster (sector s, row, y, drift time t) of a track from a collision at
 * time t_c (side sgn = +1 for sectors 0-17, -1 for 18-35) is measured at
 *   zl = z_max - v (t - t_c - t0),  w = clamp(zl/z_max, 0, 1),
 *   m_y = y - dy(u, w),  m_z = sgn (zl - dz(u, w)).
 * The calibration chi2 of a track is the chi2 of one inward Kalman pass over
 * its clusters (outermost first) ending with a primary-vertex
 * pseudo-measurement (y = z = 0 at the origin, variance vertex_var; the last
 * step rotates the frame about the origin onto the innermost reference
 * position, then follows the helix to x = 0) and, for a track with a dip
 * angle from the matched inner track (tgl_ext), one more update of
 * tan(lambda) with variance tgl_var at the vertex, linearised
 * around a reference helix that does not depend on theta: the tracker's
 * output state (tpc_tracks.param etc.), its z moved from the tracker's frame
 * to absolute z by sgn v_nominal t_c, carried along the cluster planes.  Step
 * 0 sets the deviation from the reference to (m_y - y_ref, m_z - z_ref, 0, 0,
 * 0) with covariance diag(sigma_y^2, sigma_z^2, c0_snp, c0_tgl, c0_qpt) from
 * tpc_params.  A track is left out (used = 0) when its reference reaches
 * |sin(phi)| >= 0.9 at one of its clusters.  The gradient comes from a
 * reverse sweep: the forward pass stores the reference state every 16 steps
 * and the deviation after the last step; the backward pass recomputes each
 * 16-step segment's reference from its checkpoint and carries the smoothed
 * deviation back through the inverse step Jacobians, since the derivative of
 * the chi2 with respect to a measurement is twice its weighted smoothed
 * residual (the pass is a linear least-squares problem without process
 * noise).
 *
 * Arithmetic: binary32 (the state with compensated sums), gradient sums in
 * binary64.  All pointers in tpc_calib_tracks and the theta / chi2 / used /
 * dchi2 / grad arrays are device pointers owned by the caller; the
 * workspace is a caller-owned device buffer.  The forward and backward calls
 * only enqueue work on `stream` (no host synchronisation; capturable in a
 * CUDA graph); tpc_calib_status reads the error flag the kernels set.
 */
#ifndef TPC_CALIB_H
#define TPC_CALIB_H

#include <stddef.h>
#include <stdint.h>

#include "tpc_track.h"

#ifdef __cplusplus
extern "C" {
#endif

#define TPC_CALIB_NSPL 8
#define TPC_CALIB_N_THETA(n_sectors) (2 + (n_sectors) * TPC_CALIB_NSPL * TPC_CALIB_NSPL * 2)
#define TPC_CALIB_CKPT_STEPS 16           /* steps between stored states */

typedef struct {
    int32_t n_tracks;
    const int32_t *sector;        /* [T] sector of the reference state */
    const float *x;               /* [T] x of the reference state (cm) */
    const float *param;           /* [T][5] y, z (tracker frame), sin(phi), tan(lambda), q/pT */
    const int32_t *clus_offset;   /* [T+1], clus_offset[0] == 0, non-decreasing */
    const int32_t *clus_index;    /* cluster indices of each track, innermost first */
    const float *t_coll;          /* [T] collision time (us); NaN: the track is not used */
    int64_t n_clusters;           /* clusters in the arrays below (>= clus_offset[T]) */
    const uint8_t *cl_sector;     /* [n] */
    const uint8_t *cl_row;        /* [n] */
    const float *cl_y;            /* [n] local y (cm) */
    const float *cl_t;            /* [n] drift time (us) */
    const float *tgl_ext;         /* [T] dip angle tan(lambda) of the matched inner track, NaN = none;
                                     NULL: no track has one */
    float tgl_var;                /* its variance (> 0 when tgl_ext is given) */
} tpc_calib_tracks;

/* Device workspace (bytes) for n_tracks tracks holding at most n_clusters
 * clusters in total: a 256-byte header (error flag), one 48-byte reference
 * checkpoint per TPC_CALIB_CKPT_STEPS steps of each track, the deviation
 * after each track's last step (32 B) and the order in which both passes
 * visit the tracks (by decreasing cluster count; 4 B).  Errors:
 * TPC_ERR_ARG. */
int tpc_calib_workspace_size(const tpc_geometry *g, int32_t n_tracks, int64_t n_clusters, size_t *bytes);

/* Forward pass: chi2[r] (binary32) and used[r] (1: the track entered the
 * sum; 0: t_coll is NaN, fewer than 2 clusters, or a reference step left the
 * helix domain) for every track, and the checkpoints in `workspace`.
 * g must have drift times (g->continuous).  Errors: TPC_ERR_ARG,
 * TPC_ERR_CAPACITY (ws_bytes too small), TPC_ERR_CUDA.  Invalid data
 * (cluster index, sector or row out of range, decreasing offsets) mark the
 * track unused and set the flag tpc_calib_status reports. */
int tpc_calib_forward(const tpc_params *p, const tpc_geometry *g, float bz, float v_nominal, float vertex_var,
                      const tpc_calib_tracks *tr, const float *theta, float *chi2, uint8_t *used,
                      void *workspace, size_t ws_bytes, void *stream);

/* Backward pass: grad (binary64, TPC_CALIB_N_THETA(g->n_sectors), zeroed
 * by the call) = d/dtheta of sum_r dchi2[r] chi2_r over the tracks with
 * used[r] = 1, from the checkpoints of the last tpc_calib_forward on this
 * workspace with the same tracks and theta.  Errors as tpc_calib_forward. */
int tpc_calib_backward(const tpc_params *p, const tpc_geometry *g, float bz, float v_nominal, float vertex_var,
                       const tpc_calib_tracks *tr, const float *theta, const float *dchi2, const uint8_t *used,
                       const void *workspace, size_t ws_bytes, double *grad, void *stream);

/* Calibration track selection (the rule of this library's reading of the
 * online calibration, sections "Tracking" and "TPC Tracking": tracks from the
 * primary vertex whose collision time is known): t_sel[r] = t_coll[r] when
 * the track's refit succeeded (status[r] == 0) and |q/pT| <= qpt_max
 * (binary32, on param[r][4]); NaN otherwise, which tpc_calib_forward reads as
 * "not used".  Low-pT loopers (|q/pT| above TPC_CALIB_QPT_MAX, pT below
 * 0.2 GeV/c) are left out because their later legs do not point to the
 * vertex.  t_coll[r] may itself be NaN (no matched time).  Device arrays
 * owned by the caller: t_coll [n_tracks], status [n_tracks], param
 * [n_tracks][5] (as tpc_tracks), t_sel [n_tracks] (may alias t_coll).
 * Enqueues one kernel on `stream`.  Errors: TPC_ERR_ARG (n_tracks < 0, a
 * null array with n_tracks > 0, qpt_max not a number), TPC_ERR_CUDA. */
#define TPC_CALIB_QPT_MAX 5.0f
int tpc_calib_select(int32_t n_tracks, const float *t_coll, const int32_t *status, const float *param,
                     float qpt_max, float *t_sel, void *stream);

/* ------------------------------------------------------------------------
 * Closed-loop calibration (section "TPC Tracking": online drift-velocity
 * calibration; this library's reading): theta minimising
 *   F(theta) = sum over the selected tracks of chi2_r(theta)
 *              + sum over the spline coefficients of (c / prior_sigma)^2,
 * by L-BFGS (memory 10, backtracking line search with the sufficient
 * decrease condition) in the variables x = (theta - theta_start) / s with
 * s = (scale_v, scale_t0, prior_sigma, ...), chi2 and gradient from
 * tpc_calib_forward / tpc_calib_backward on the GPU, the L-BFGS algebra on
 * the host in binary64.  The Gaussian prior decides between the spline map
 * and (v, t0) where the tracks cannot: a common z offset or z scale of every
 * sector.  Track selection: the first round uses the tracks with t_coll set
 * whose chi2 / ndf (ndf = 2 n) at theta_start is below chi2ndf_first and the
 * dip angles whose chi2 contribution there is below anchor_cut_first; each
 * later round re-selects at the current theta with chi2ndf_cut and
 * anchor_cut and continues from it.  A round ends after max_iter iterations
 * or when an iteration lowers F by less than ftol F.
 * -------------------------------------------------------------------- */
typedef struct {
    float prior_sigma;            /* spline coefficients (cm), default 0.3 */
    float scale_v, scale_t0;      /* variable scales of v (cm/us) and t0 (us): 0.01, 0.1 */
    int32_t max_iter;             /* L-BFGS iterations per round (300) */
    int32_t rounds;               /* rounds after the first (2) */
    float chi2ndf_first, anchor_cut_first;   /* first selection (10, 100) */
    float chi2ndf_cut, anchor_cut;           /* later selections (2.5, 16) */
    double ftol;                  /* 1e-10 */
} tpc_calib_fit_opts;

typedef struct {
    double f_start, f_final;      /* F at theta_start (first selection) and at the result (last selection) */
    int32_t evaluations;          /* chi2 + gradient evaluations (forward + backward pairs) */
    int32_t rounds;               /* rounds run */
    int32_t tracks, anchors;      /* tracks and dip angles of the last selection */
} tpc_calib_fit_report;

int tpc_calib_fit_defaults(tpc_calib_fit_opts *opt);

/* Device workspace of tpc_calib_fit: the pass's workspace plus per-track
 * selections, chi2 buffers and the gradient.  Errors: TPC_ERR_ARG. */
int tpc_calib_fit_workspace_size(const tpc_geometry *g, int32_t n_tracks, int64_t n_clusters, size_t *bytes);

/* theta (device, binary32, TPC_CALIB_N_THETA(n_sectors)): the start on entry,
 * the result on return.  t_used / tgl_used (device [n_tracks], may be NULL):
 * the last selection, as t_coll / tgl_ext with NaN for the tracks and dip
 * angles left out.  rep (host) may be NULL.  Synchronises `stream` at every
 * evaluation.  Errors: as tpc_calib_forward; TPC_ERR_DATA when a pass flags
 * invalid track data. */
int tpc_calib_fit(const tpc_params *p, const tpc_geometry *g, float bz, float v_nominal, float vertex_var,
                  const tpc_calib_tracks *tr, const tpc_calib_fit_opts *opt, float *theta, void *workspace,
                  size_t ws_bytes, float *t_used, float *tgl_used, tpc_calib_fit_report *rep, void *stream);

/* Synchronises `stream` and writes the workspace's error flag to *err
 * (0: none; 1: invalid track data seen).  Errors: TPC_ERR_ARG, TPC_ERR_CUDA. */
int tpc_calib_status(const void *workspace, int32_t *err, void *stream);

#ifdef __cplusplus
}
#endif
#endif
