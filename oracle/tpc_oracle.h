/*
 * tpc_oracle.h -- CPU oracle of the TPC cellular-automaton + Kalman tracker.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  It shares no code,
 * header, table or constant generator with the CUDA tracker; both are written
 * independently from the same written specification of the method.
 *
 * Method: cellular-automaton seeding + Kalman-filter track following and
 * refit of the paper's section "TPC Tracking" (the combinatorial part is
 * confined to seeding, one hypothesis per track is followed, later steps are
 * linear), with continuous read-out handled as in section "Tracking" (time
 * scaled linearly to z with the average drift velocity, primary-track
 * assumption while seeding, later refit).
 *
 * Precision: every decision that produces an integer result (links, start
 * hits, tracklet hit lists, ownership, merges) is taken in IEEE binary32 with
 * an explicitly fixed operation order (fmaf where fused), exactly like the
 * GPU.  The final refit is IEEE binary64.
 */
#ifndef TPC_ORACLE_H
#define TPC_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    float dy_link, dz_link, s_max_link;   /* seeding windows (cm) and straightness cut (cm^2) */
    float sigma_y, sigma_z;               /* cluster errors (cm) */
    float c0_snp, c0_tgl, c0_qpt;         /* prior variances of sin(phi), tan(lambda), q/pT */
    float win_nsigma, win_min, win_max;   /* following window: clamp(n*sigma, min, max) (cm) */
    float chi2_cut;                       /* per-update chi2 cut while following (2 dof) */
    int32_t max_miss;                     /* stop after this many consecutive empty rows */
    int32_t min_hits;                     /* tracklet needs at least this many hits */
    int32_t min_owned;                    /* selector: owned hits needed */
    float edge_margin;                    /* stop following when |y| > x tan(10 deg) + margin */
    float merge_dz, merge_chi2;           /* merger candidate window (cm) and chi2 (5 dof) cut */
    int32_t refit_passes;                 /* Kalman refit passes, alternating direction */
    float refit_inflate;                  /* factor on the previous angular covariance at each pass start */
    int32_t packed_links;                 /* 1: the link pass sees y, z rounded to 1/256 cm (16-bit packed) */
    int32_t back_jump;                    /* TrackletConstructor phase C: rows per return jump (1: row by row) */
    float outlier_chi2;                   /* cluster rejection before the refit: dy^2/vy + dz^2/vz cut (0: off) */
} orc_params;

typedef struct {
    int32_t n_sectors;      /* 36 (18 per side) or 1 (one 20 degree wedge spanning both z signs) */
    int32_t n_rows;         /* pad rows */
    const float *row_x;     /* [n_rows] row plane x (cm) */
    float z_max;            /* drift length (cm) */
    int32_t continuous;     /* 1: cluster carries drift time (us), 0: z (cm) */
} orc_geom;

/* Everything the oracle computes; arrays are malloc'ed by the oracle. */
typedef struct {
    int32_t n;
    float *z;                 /* [n] z after time->z (cm) */
    int32_t *up_raw, *dn_raw; /* [n] best link pair per hit (cluster index or -1) */
    int32_t *up, *dn;         /* [n] mutual links after cleaning */
    uint8_t *is_start;        /* [n] chain start flag */
    /* tracklets: one per start hit, in ascending start cluster index */
    int32_t n_tracklets;
    int32_t *trk_start;       /* [nt] start cluster index */
    int32_t *trk_nhits;       /* [nt] */
    int32_t *trk_off;         /* [nt+1] offsets into trk_hits */
    int32_t *trk_hits;        /* cluster indices, ascending row */
    uint8_t *trk_kept;        /* [nt] selector verdict */
    float *trk_top;           /* [nt][21]: x, p[5], c[15] at the outermost fitted hit */
    float *trk_bot;           /* [nt][21]: x, p[5], c[15] at the innermost hit */
    /* segments = kept tracklets (ascending start index) */
    int32_t n_seg;
    int32_t *seg_trk;         /* [ns] tracklet index */
    int32_t *seg_next, *seg_prev;  /* [ns] merge links after the mutual-best rule, -1 none */
    /* merged + refitted tracks, ordered by the start index of their innermost segment */
    int32_t n_tracks;
    int32_t *tr_sector;       /* [T] sector of the innermost cluster (frame of the output state) */
    double *tr_x;             /* [T] */
    double *tr_p;             /* [T][5] y, z, sin(phi), tan(lambda), q/pT */
    double *tr_c;             /* [T][15] lower-triangular covariance */
    double *tr_chi2;          /* [T] */
    int32_t *tr_ndf;          /* [T] */
    int32_t *tr_status;       /* [T] 0 ok, 1 refit propagation failed */
    int32_t *tr_nclus;        /* [T] */
    int32_t *tr_off;          /* [T+1] */
    int32_t *tr_clus;         /* cluster indices inner -> outer */
    int32_t *assign;          /* [n] track index or -1 */
    uint8_t *rejected;        /* [n] 1: owned by a kept tracklet but rejected before the refit */
    int32_t n_rejected;
    float row_qup[256], row_qdn[256], row_w[256];
} orc_result;

void orc_params_default(orc_params *p);
int orc_track(const orc_params *P, const orc_geom *G, float bz, float v_drift, int32_t n,
              const uint8_t *sector, const uint8_t *row, const float *y, const float *zt,
              orc_result *out);
void orc_free(orc_result *r);

/* Track-based cluster attachment (tpc_oracle_attach.c).  Inputs: the clusters
 * (sector, row, y, z after time -> z) and the tracker's segments as
 * orc_track returns them (seg_trk/next/prev, the tracklet hit lists and
 * inner-end states, assign) and optionally (tr_leg, NULL: none) the looper
 * leg number of each track (orc_loopers).  Outputs per cluster: the adjacent
 * track (-1 none) and flags ORC_CL_*. */
#define ORC_CL_ATTACHED  1
#define ORC_CL_ADJACENT  2
#define ORC_CL_PROTECTED 4
#define ORC_CL_REMOVE    8
int orc_step_pos32(float *p, float x2, float kb);
int orc_attach(const orc_geom *G, float bz, int32_t n, const uint8_t *sector, const uint8_t *row,
               const float *y, const float *z, int32_t n_seg, const int32_t *seg_trk,
               const int32_t *seg_next, const int32_t *seg_prev, const int32_t *trk_off,
               const int32_t *trk_hits, const float *trk_bot, const int32_t *assign, float radius,
               float pt_min, const int32_t *tr_leg, int32_t *adjacent, uint8_t *flags);

/* Looper-leg identification (tpc_oracle_loopers.c).  Per track: sector and
 * time frame (frame may be NULL) of its innermost piece and that piece's
 * inner-end state (21 floats: x, y, z, sin(phi), tan(lambda), q/pT, cov);
 * outputs group (smallest track index of the legs of one particle, -1 alone)
 * and leg (0 = the earliest in drift, -1 alone). */
int orc_loopers(int32_t n_sectors, float z_max, float bz, float qpt_min, int32_t n_tracks, const int32_t *sector,
                const int32_t *frame, const float *state, int32_t *group, int32_t *leg);
float orc_atan2_own(float y, float x);

/* Cluster compression (tpc_oracle_compress.c): rANS coder of byte symbols,
 * the integer fields of the format (12 streams), their inverse, and the
 * coded size of one stream. */
int orc_rans_normalise(const uint32_t *hist, uint32_t *freq);
int orc_rans_encode(const uint8_t *sym, int32_t n, const uint32_t *freq, uint8_t *out, int32_t *nbytes);
int orc_rans_decode(const uint8_t *in, int32_t nbytes, const uint32_t *freq, int32_t n, uint8_t *sym);
int orc_compress_fields(int32_t n_sectors, int32_t n_rows, int32_t n, const uint8_t *sector, const uint8_t *row,
                        const float *y, const float *zt, int32_t ey, int32_t et, int32_t n_tracks,
                        const int32_t *clus_offset, const int32_t *clus_index, const int32_t *assign,
                        uint32_t **vals, int64_t *counts);
int orc_decompress_fields(int32_t n_sectors, int32_t n_rows, const uint32_t *const *vals, const int64_t *counts,
                          int32_t n_tracks, int32_t n, uint8_t *sector, uint8_t *row, int32_t *qy, int32_t *qt);
int64_t orc_symbolise(const uint32_t *v, int64_t n, uint8_t *sym, uint8_t *raw, int64_t *nraw);
int orc_desymbolise(const uint8_t *sym, int64_t n, const uint8_t *raw, int64_t nraw, uint32_t *v);
int orc_code_stream(const uint32_t *v, int64_t n, int32_t chunk, int64_t *bytes, int32_t *roundtrip_ok);
int64_t orc_pack_stream(const uint32_t *v, int64_t n, int32_t chunk, uint8_t *out);
int64_t orc_unpack_stream(const uint8_t *in, int64_t nbytes, uint32_t *v, int64_t vcap, int64_t *n_out);
void orc_free_ptr(void *p);

/* single Kalman steps, exposed for the pins */
int orc_prop32(float *st21, float x2, float kb);
int orc_rot32(float *st21, float cs, float sn, float kb);
int orc_update32(float *st21, float my, float mz, float vy, float vz, float chi2max, float *chi2);
int orc_prop64(double *st21, double x2, double kb);
int orc_rot64(double *st21, double cs, double sn, double kb);
/* the same FP64 steps on a bare state (x, p[5]) with their 5x5 Jacobians
 * (row = output parameter); on failure the state is left unchanged */
int orc_helix64(double *x, double *p, double x2, double kb, double F[5][5]);
int orc_rotate64(double *x, double *p, double cs, double sn, double kb, double J[5][5]);
int orc_update64(double *st21, double my, double mz, double vy, double vz, double *chi2);
/* FP64 multi-pass fit of a cluster list (inner -> outer); st21 in: initial
 * state in the outermost cluster's frame, out: state at the innermost cluster */
int orc_fit64(const orc_params *P, const orc_geom *G, double kb, int32_t n,
              const int32_t *sector, const double *x, const double *y, const double *z,
              int32_t n_passes, double *st21, double *chi2);
float orc_merge_chi2(const float *top21, const float *bot21, float cs, float sn, float kb);

/* ---- calibration chi2 of the refit and its gradient (tpc_oracle_calib.c) ----
 * theta = {v_drift (cm/us), t0 (us), c[n_sectors][8][8][2]}: per sector an
 * 8 x 8 clamped cubic B-spline of the cluster distortion (dy, dz) over
 * ((x - x_first)/(x_last - x_first), |z|/z_max).  Tracks: the tracker's
 * output (sector, x, 5 parameters in the tracker's z frame, cluster lists
 * inner -> outer); tcoll[r] = collision time (us), NaN = track not used.
 * chi2_out[r] / used[r] per track; grad (n_theta, may be NULL) = gradient of
 * sum_r weight[r] chi2_r (weight NULL = all 1).  tgl_ext (may be NULL; NaN
 * entries: none) is a dip angle tan(lambda) of the track measured outside
 * the TPC (the matched inner track), applied after the vertex step as one
 * more update with variance tgl_var.  Returns 0, or -1 for a geometry
 * without drift times. */
#define ORC_CALIB_NSPL 8
int orc_calib(const orc_params *P, const orc_geom *G, double bz, double v_nom, double vtx_var, int32_t n_tracks,
              const int32_t *tr_sector, const float *tr_x, const float *tr_p, const int32_t *tr_off,
              const int32_t *tr_clus, const uint8_t *sector, const uint8_t *row, const float *y, const float *t,
              const float *tcoll, const double *theta, const double *weight, double *chi2_out, uint8_t *used,
              double *grad, const float *tgl_ext, double tgl_var);
/* calibration track selection: t_sel[r] = t_coll[r] if status[r] == 0 and
 * |param[r][4]| <= qpt_max (binary32), else NaN */
void orc_calib_select(int32_t n, const float *t_coll, const int32_t *status, const float *param, float qpt_max,
                      float *t_sel);
/* the calibrated measurement of each cluster (for the pins) */
void orc_calib_measure(const orc_geom *G, const double *theta, int32_t n, const uint8_t *sector,
                       const uint8_t *row, const float *y, const float *t, const float *tc, double *my, double *mz);
/* one track's pass laid out for the pins: per step k = 0..n the Jacobian
 * F[k] (5x5, zero at k = 0), reference (y, z) h[k], measurement m[k] and its
 * variances v[k]; returns 0, or 1 when a reference step fails */
int orc_calib_explain(const orc_params *P, const orc_geom *G, double bz, double v_nom, double vtx_var,
                      const int32_t *tr_sector, const float *tr_x, const float *tr_p, const int32_t *tr_off,
                      const int32_t *tr_clus, const uint8_t *sector, const uint8_t *row, const float *y,
                      const float *t, const float *tcoll, const double *theta, int32_t r, double *F, double *h,
                      double *m, double *v, double *chi2);
/* all 8 B-spline basis values and derivatives at u (for the pins) */
void orc_bspline_all(double u, double *out, double *dout);

#ifdef __cplusplus
}
#endif
#endif
