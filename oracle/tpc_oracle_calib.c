/*
 * tpc_oracle_calib.c -- binary64 oracle of the calibration chi2 of the refit
 * and of its gradient with respect to the calibration parameters.
 *
 * TEST INFRASTRUCTURE ONLY, like tpc_oracle.c: only tests/, the smoke check
 * and the CPU baseline leg of the benchmark may load it.  It shares nothing
 * with the CUDA code.
 *
 * Paper: section "Tracking" (continuous read-out: time is turned into z with
 * the drift velocity; once matching has fixed the collision time, the final
 * refit applies the calibration under the primary-track assumption) and
 * section "TPC Tracking" (online drift-velocity calibration).
 *
 * Reading (the paper gives no formulas for this part):
 *   theta = {v, t0, c[s][i][j][k]}: drift velocity (cm/us), time offset (us)
 *   and, per sector s, an 8 x 8 uniform clamped cubic B-spline (i along
 *   u = (x - x_first)/(x_last - x_first), j along w = |z|/z_max) of the
 *   distortion (k = 0: dy, k = 1: dz along the drift direction).
 *   A cluster (sector s, row x, y, drift time t) of a track from a collision
 *   at time t_c is measured, on side sgn (+1 for sectors 0-17), at
 *       zl  = z_max - v (t - t_c - t0),   w = clamp(zl / z_max, 0, 1)
 *       m_y = y - dy(u, w),   m_z = sgn (zl - dz(u, w)).
 *   The calibration chi2 of a track is the chi2 of one inward Kalman pass over
 *   its clusters, outermost first, ending with a primary-vertex
 *   pseudo-measurement (y = z = 0 at the origin, variance vtx_var; the last
 *   step rotates the frame about the origin onto the innermost reference
 *   position and then follows the helix to x = 0, so that it stays well
 *   conditioned for tracks that bend far from the sector axis).  Tracks whose
 *   reference reaches |sin(phi)| >= 0.9 at a cluster are left out.  The pass is
 *   linearised around a reference helix that does not depend on theta: the
 *   tracker's output state, its z moved from the tracker's frame (nominal
 *   drift velocity v_nom, no t0, no collision time) to absolute z by
 *   sgn v_nom t_c, carried along the cluster planes.  Jacobians, covariances
 *   and gains are then fixed, the chi2 is a quadratic form in the
 *   measurements, and its gradient is the reverse sweep of the pass.
 *   Step 0 (outermost cluster) initialises the deviation from the reference
 *   with the measurement: (m_y - y_ref, m_z - z_ref, 0, 0, 0), covariance
 *   diag(sigma_y^2, sigma_z^2, c0_snp, c0_tgl, c0_qpt).  Steps 1 .. n-1 are
 *   the other clusters, inwards; step n is the vertex.
 */
#include "tpc_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define NSPL ORC_CALIB_NSPL

/* Uniform clamped cubic B-spline with NSPL coefficients on [0, 1]: the 4
 * basis functions that can be non-zero at u, their derivatives, and the index
 * of the first.  Cox-de Boor recursion on the knots
 * 0,0,0,0, 1/5, 2/5, 3/5, 4/5, 1,1,1,1; u is clamped to [0, 1]. */
static int bspline(double u, double *B, double *dB)
{
    enum { P = 3, NK = NSPL + P + 1 };
    double t[NK];
    const int nint = NSPL - P;
    for (int i = 0; i <= P; i++) t[i] = 0.0;
    for (int i = 1; i < nint; i++) t[P + i] = (double)i / nint;
    for (int i = 0; i <= P; i++) t[NSPL + i] = 1.0;
    if (u < 0) u = 0;
    if (u > 1) u = 1;
    int span = P;                       /* t[span] <= u < t[span+1], last span closed */
    while (span < NSPL - 1 && u >= t[span + 1]) span++;
    /* N[d][r]: degree-d basis function number span-d+r */
    double N[P + 1][P + 1];
    memset(N, 0, sizeof(N));
    N[0][0] = 1.0;
    for (int d = 1; d <= P; d++)
        for (int r = 0; r <= d; r++) {
            const int i = span - d + r;
            double v = 0.0;
            if (r >= 1) {                /* left term: N_{i,d-1} */
                const double den = t[i + d] - t[i];
                if (den > 0) v += (u - t[i]) / den * N[d - 1][r - 1];
            }
            if (r <= d - 1) {            /* right term: N_{i+1,d-1} */
                const double den = t[i + d + 1] - t[i + 1];
                if (den > 0) v += (t[i + d + 1] - u) / den * N[d - 1][r];
            }
            N[d][r] = v;
        }
    for (int r = 0; r <= P; r++) {
        const int i = span - P + r;
        double d = 0.0;
        if (r >= 1) {
            const double den = t[i + P] - t[i];
            if (den > 0) d += P / den * N[P - 1][r - 1];
        }
        if (r <= P - 1) {
            const double den = t[i + P + 1] - t[i + 1];
            if (den > 0) d -= P / den * N[P - 1][r];
        }
        B[r] = N[P][r];
        dB[r] = d;
    }
    return span - P;
}

void orc_bspline_all(double u, double *out, double *dout)
{
    double B[4], dB[4];
    for (int i = 0; i < NSPL; i++) out[i] = dout[i] = 0.0;
    const int i0 = bspline(u, B, dB);
    for (int a = 0; a < 4; a++) {
        out[i0 + a] = B[a];
        dout[i0 + a] = dB[a];
    }
}

static double side_of(int sector, int n_sectors) { return (n_sectors == 36 && sector >= 18) ? -1.0 : 1.0; }

static double sector_alpha(int s, int n_sectors)
{
    if (n_sectors == 1) return 10.0 * M_PI / 180.0;
    return ((s % 18) * 20.0 + 10.0) * M_PI / 180.0;
}

/* a calibrated measurement and what the gradient needs of it */
typedef struct {
    double my, mz;
    double dmy_dv, dmz_dv, dmy_dt0, dmz_dt0;
    double sgn;
    int sector, i0, j0;
    double Bu[4], Bw[4];
    /* error scale of m_z: s = (v / v_nom) (1 - d dz / d zl at the nominal
     * position), its derivatives: ds/dv = s / v, ds/dc[i0+a][j0n+b][1] =
     * -(v / v_nom) Bu[a] dBn[b] */
    double s;
    int j0n;
    double dBn[4];
} meas_t;

static void measure(const orc_geom *G, const double *theta, double v_nom, int sector, int row, double y, double t,
                    double tc, meas_t *m)
{
    const double v = theta[0], t0 = theta[1];
    const double x_first = G->row_x[0], x_last = G->row_x[G->n_rows - 1];
    const double zmax = G->z_max;
    const double tau = t - tc - t0;
    const double zl = zmax - v * tau;
    const double wraw = zl / zmax;
    const double dw_dzl = (wraw > 0.0 && wraw < 1.0) ? 1.0 / zmax : 0.0;   /* clamped outside */
    double dBu[4], dBw[4];
    m->i0 = bspline(((double)G->row_x[row] - x_first) / (x_last - x_first), m->Bu, dBu);
    m->j0 = bspline(wraw, m->Bw, dBw);
    const double *c = theta + 2 + (size_t)sector * NSPL * NSPL * 2;
    double dy = 0, dz = 0, dy_w = 0, dz_w = 0;
    for (int a = 0; a < 4; a++)
        for (int b = 0; b < 4; b++) {
            const double *cc = c + ((m->i0 + a) * NSPL + (m->j0 + b)) * 2;
            dy += m->Bu[a] * m->Bw[b] * cc[0];
            dz += m->Bu[a] * m->Bw[b] * cc[1];
            dy_w += m->Bu[a] * dBw[b] * cc[0];
            dz_w += m->Bu[a] * dBw[b] * cc[1];
        }
    const double sgn = side_of(sector, G->n_sectors);
    /* chain rule through zl: d zl / dv = -tau, d zl / dt0 = v */
    const double dzl[2] = {-tau, v};
    m->my = y - dy;
    m->mz = sgn * (zl - dz);
    m->dmy_dv = -dy_w * dw_dzl * dzl[0];
    m->dmz_dv = sgn * (1.0 - dz_w * dw_dzl) * dzl[0];
    m->dmy_dt0 = -dy_w * dw_dzl * dzl[1];
    m->dmz_dt0 = sgn * (1.0 - dz_w * dw_dzl) * dzl[1];
    m->sgn = sgn;
    m->sector = sector;
    /* the drift-time error carried into m_z: the slope of the map is taken at
     * the nominal position (v_nom, no t0), so that s is linear in the map */
    const double wn = (zmax - v_nom * (t - tc)) / zmax;
    const double dwn = (wn > 0.0 && wn < 1.0) ? 1.0 / zmax : 0.0;
    double Bn[4], dBn[4];
    m->j0n = bspline(wn, Bn, dBn);
    double dzn = 0.0;
    for (int a = 0; a < 4; a++)
        for (int b = 0; b < 4; b++) dzn += m->Bu[a] * dBn[b] * c[((m->i0 + a) * NSPL + (m->j0n + b)) * 2 + 1];
    m->s = (v / v_nom) * (1.0 - dzn * dwn);
    for (int b = 0; b < 4; b++) m->dBn[b] = dBn[b] * dwn;
}

void orc_calib_measure(const orc_geom *G, const double *theta, int32_t n, const uint8_t *sector,
                       const uint8_t *row, const float *y, const float *t, const float *tc, double *my, double *mz)
{
    for (int32_t i = 0; i < n; i++) {
        meas_t m;
        measure(G, theta, theta[0], sector[i], row[i], y[i], t[i], tc[i], &m);
        my[i] = m.my;
        mz[i] = m.mz;
    }
}

static void mat_mul(double A[5][5], double B[5][5], double C[5][5])
{
    double T[5][5];
    for (int i = 0; i < 5; i++)
        for (int j = 0; j < 5; j++) {
            double s = 0;
            for (int k = 0; k < 5; k++) s += A[i][k] * B[k][j];
            T[i][j] = s;
        }
    memcpy(C, T, sizeof(T));
}

/* the calibration pass leaves out tracks whose reference runs at more than
 * asin(0.9) = 64 degrees to the pad-row normal at any of their clusters
 * (nearly tangent to the rows, where the helix step is ill conditioned) */
#define SNP_CALIB 0.9

/* reference step to the plane x2 of sector s2: rotation when the sector
 * changes, then the helix; F = (helix Jacobian)(rotation Jacobian) */
static int ref_step(const orc_geom *G, double kb, int *sec, double *x, double *q, int s2, double x2, double F[5][5])
{
    double J[5][5], H[5][5];
    for (int i = 0; i < 5; i++)
        for (int j = 0; j < 5; j++) J[i][j] = i == j;
    if (s2 != *sec) {
        double da = sector_alpha(s2, G->n_sectors) - sector_alpha(*sec, G->n_sectors);
        while (da > M_PI) da -= 2 * M_PI;
        while (da <= -M_PI) da += 2 * M_PI;
        if (!orc_rotate64(x, q, cos(da), sin(da), kb, J)) return 0;
        *sec = s2;
    }
    if (!orc_helix64(x, q, x2, kb, H)) return 0;
    if (!(fabs(q[2]) < SNP_CALIB)) return 0;
    mat_mul(H, J, F);
    return 1;
}

/* reference step to the primary vertex: rotate the frame about the origin
 * onto the reference position (new x along it, y = 0), then the helix to
 * x = 0; the track crosses x = 0 at a small angle to the new axis, where the
 * step is well conditioned.  F = (helix Jacobian)(rotation Jacobian). */
static int vertex_step(double kb, double *x, double *q, double F[5][5])
{
    double J[5][5], H[5][5];
    const double r = hypot(*x, q[0]);
    if (!(r > 0.0)) return 0;
    if (!orc_rotate64(x, q, *x / r, q[0] / r, kb, J)) return 0;
    if (!orc_helix64(x, q, 0.0, kb, H)) return 0;
    mat_mul(H, J, F);
    return 1;
}

/* the dip-angle update after the vertex step */
typedef struct {
    int on;
    double K[5], W, r;
} anchor_t;

/* per-step record of the inward pass of one track */
typedef struct {
    double F[5][5];     /* Jacobian from the previous step's state */
    double K[5][2];     /* gain */
    double W[2][2];     /* inverse innovation covariance */
    double r[2];        /* innovation */
    double hy, hz;      /* reference (y, z) */
    double my, mz, vy, vz;
    meas_t m;           /* cluster measurement (steps < n) */
} step_t;

/* Runs the inward pass of track r; fills steps[0 .. n] (n = clusters), returns
 * 1 and the chi2, or 0 when a reference step fails. */
static int track_pass(const orc_params *P, const orc_geom *G, double kb, double v_nom, double vtx_var,
                      const int32_t *tr_sector, const float *tr_x, const float *tr_p, const int32_t *tr_off,
                      const int32_t *tr_clus, const uint8_t *sector, const uint8_t *row, const float *y,
                      const float *t, const float *tcoll, const double *theta, int r, step_t *S, double *chi2o,
                      double tgl_m, double tgl_var, anchor_t *A)
{
    const int off = tr_off[r], n = tr_off[r + 1] - tr_off[r];
    const double tc = tcoll[r];
    int sec = tr_sector[r];
    double x = tr_x[r], q[5];
    for (int k = 0; k < 5; k++) q[k] = tr_p[5 * r + k];
    if (!(fabs(q[2]) < SNP_CALIB)) return 0;
    q[1] += side_of(sec, G->n_sectors) * v_nom * tc;      /* tracker frame -> absolute z */
    double F[5][5];
    /* out to the outermost cluster along the cluster list */
    for (int i = 1; i < n; i++) {
        const int c = tr_clus[off + i];
        if (!ref_step(G, kb, &sec, &x, q, sector[c], G->row_x[row[c]], F)) return 0;
    }
    const double vy = (double)P->sigma_y * P->sigma_y, vz = (double)P->sigma_z * P->sigma_z;
    double dp[5], C[5][5];
    double chi2 = 0.0;
    for (int k = 0; k <= n; k++) {
        step_t *st = &S[k];
        if (k < n) {
            const int c = tr_clus[off + n - 1 - k];
            if (k > 0 && !ref_step(G, kb, &sec, &x, q, sector[c], G->row_x[row[c]], st->F)) return 0;
            measure(G, theta, v_nom, sector[c], row[c], y[c], t[c], tc, &st->m);
            st->my = st->m.my;
            st->mz = st->m.mz;
            st->vy = vy;
            st->vz = vz * st->m.s * st->m.s;
        } else {
            if (!vertex_step(kb, &x, q, st->F)) return 0;
            st->my = 0.0;
            st->mz = 0.0;
            st->vy = vtx_var;
            st->vz = vtx_var;
        }
        st->hy = q[0];
        st->hz = q[1];
        if (k == 0) {
            for (int i = 0; i < 5; i++)
                for (int j = 0; j < 5; j++) st->F[i][j] = 0.0;
            memset(C, 0, sizeof(C));
            C[0][0] = vy;
            C[1][1] = st->vz;
            C[2][2] = P->c0_snp;
            C[3][3] = P->c0_tgl;
            C[4][4] = P->c0_qpt;
            dp[0] = st->my - st->hy;
            dp[1] = st->mz - st->hz;
            dp[2] = dp[3] = dp[4] = 0.0;
            continue;
        }
        /* prediction */
        double pm[5], Cm[5][5], T[5][5];
        for (int i = 0; i < 5; i++) {
            double s = 0;
            for (int j = 0; j < 5; j++) s += st->F[i][j] * dp[j];
            pm[i] = s;
        }
        mat_mul(st->F, C, T);
        for (int i = 0; i < 5; i++)
            for (int j = 0; j < 5; j++) {
                double s = 0;
                for (int l = 0; l < 5; l++) s += T[i][l] * st->F[j][l];
                Cm[i][j] = s;
            }
        /* update with the measurement (H selects y, z) */
        st->r[0] = st->my - (st->hy + pm[0]);
        st->r[1] = st->mz - (st->hz + pm[1]);
        const double s00 = Cm[0][0] + st->vy, s01 = Cm[0][1], s11 = Cm[1][1] + st->vz;
        const double det = s00 * s11 - s01 * s01;
        if (!(det > 0)) return 0;
        st->W[0][0] = s11 / det;
        st->W[0][1] = st->W[1][0] = -s01 / det;
        st->W[1][1] = s00 / det;
        chi2 += st->r[0] * (st->W[0][0] * st->r[0] + st->W[0][1] * st->r[1]) +
                st->r[1] * (st->W[1][0] * st->r[0] + st->W[1][1] * st->r[1]);
        for (int i = 0; i < 5; i++) {
            st->K[i][0] = Cm[i][0] * st->W[0][0] + Cm[i][1] * st->W[1][0];
            st->K[i][1] = Cm[i][0] * st->W[0][1] + Cm[i][1] * st->W[1][1];
        }
        for (int i = 0; i < 5; i++) dp[i] = pm[i] + st->K[i][0] * st->r[0] + st->K[i][1] * st->r[1];
        for (int i = 0; i < 5; i++)
            for (int j = 0; j < 5; j++) C[i][j] = Cm[i][j] - (st->K[i][0] * Cm[0][j] + st->K[i][1] * Cm[1][j]);
    }
    /* the dip-angle pseudo-measurement of the matched inner track (when
     * given): one more update at the vertex, H selecting tan(lambda) */
    A->on = 0;
    if (tgl_m == tgl_m) {
        A->on = 1;
        A->r = tgl_m - (q[3] + dp[3]);
        const double sv = C[3][3] + tgl_var;
        if (!(sv > 0)) return 0;
        A->W = 1.0 / sv;
        chi2 += A->r * A->W * A->r;
        for (int i = 0; i < 5; i++) A->K[i] = C[i][3] * A->W;
    }
    *chi2o = chi2;
    return 1;
}

int orc_calib(const orc_params *P, const orc_geom *G, double bz, double v_nom, double vtx_var, int32_t n_tracks,
              const int32_t *tr_sector, const float *tr_x, const float *tr_p, const int32_t *tr_off,
              const int32_t *tr_clus, const uint8_t *sector, const uint8_t *row, const float *y, const float *t,
              const float *tcoll, const double *theta, const double *weight, double *chi2_out, uint8_t *used,
              double *grad, const float *tgl_ext, double tgl_var)
{
    if (!G->continuous || G->n_rows < 2) return -1;
    /* the field constant as the tracker forms it (binary32 product) */
    const double kb = (double)(-2.99792458e-3f * (float)bz);
    const int n_theta = 2 + G->n_sectors * NSPL * NSPL * 2;
    if (grad) memset(grad, 0, sizeof(double) * (size_t)n_theta);
    int nmax = 0;
    for (int r = 0; r < n_tracks; r++) {
        const int n = tr_off[r + 1] - tr_off[r];
        if (n > nmax) nmax = n;
    }
    step_t *S = (step_t *)malloc(sizeof(step_t) * (size_t)(nmax + 1));
    if (!S) return -2;
    for (int r = 0; r < n_tracks; r++) {
        chi2_out[r] = 0.0;
        used[r] = 0;
        const int n = tr_off[r + 1] - tr_off[r];
        if (n < 2 || !(tcoll[r] == tcoll[r])) continue;
        double chi2;
        anchor_t A;
        const double tgl_m = tgl_ext ? (double)tgl_ext[r] : NAN;
        if (!track_pass(P, G, kb, v_nom, vtx_var, tr_sector, tr_x, tr_p, tr_off, tr_clus, sector, row, y, t, tcoll,
                        theta, r, S, &chi2, tgl_m, tgl_var, &A))
            continue;
        chi2_out[r] = chi2;
        used[r] = 1;
        const double wr = weight ? weight[r] : 1.0;
        if (!grad || wr == 0.0) continue;
        /* reverse sweep: lam = d chi2 / d(deviation after step k);
         * a = d chi2 / d(measurement of step k) */
        double lam[5] = {0, 0, 0, 0, 0};
        if (A.on) lam[3] = -2.0 * A.W * A.r;     /* through the dip-angle update (its gain meets lam = 0) */
        for (int k = n; k >= 0; k--) {
            const step_t *st = &S[k];
            double a[2];
            if (k == 0) {
                a[0] = lam[0];
                a[1] = lam[1];
            } else {
                for (int e = 0; e < 2; e++) {
                    double s = 2.0 * (st->W[e][0] * st->r[0] + st->W[e][1] * st->r[1]);
                    for (int i = 0; i < 5; i++) s += st->K[i][e] * lam[i];
                    a[e] = s;
                }
                double mu[5] = {lam[0] - a[0], lam[1] - a[1], lam[2], lam[3], lam[4]};
                for (int j = 0; j < 5; j++) {
                    double s = 0;
                    for (int i = 0; i < 5; i++) s += st->F[i][j] * mu[i];
                    lam[j] = s;
                }
            }
            if (k == n) continue;          /* the vertex does not depend on theta */
            const meas_t *m = &st->m;
            /* through the variance of m_z: d chi2 / d vz = -(r*_z / vz)^2 with
             * the smoothed residual r*_z = vz a_z / 2, d vz / ds = 2 vz / s */
            const double q = -0.5 * a[1] * a[1] * st->vz / m->s;
            grad[0] += wr * q * m->s / theta[0];
            {
                double *gz = grad + 2 + (size_t)m->sector * NSPL * NSPL * 2;
                const double f = -theta[0] / v_nom;
                for (int i = 0; i < 4; i++)
                    for (int j = 0; j < 4; j++)
                        gz[((m->i0 + i) * NSPL + (m->j0n + j)) * 2 + 1] += wr * q * f * m->Bu[i] * m->dBn[j];
            }
            grad[0] += wr * (a[0] * m->dmy_dv + a[1] * m->dmz_dv);
            grad[1] += wr * (a[0] * m->dmy_dt0 + a[1] * m->dmz_dt0);
            double *g = grad + 2 + (size_t)m->sector * NSPL * NSPL * 2;
            for (int i = 0; i < 4; i++)
                for (int j = 0; j < 4; j++) {
                    const double b = m->Bu[i] * m->Bw[j];
                    double *gc = g + ((m->i0 + i) * NSPL + (m->j0 + j)) * 2;
                    gc[0] -= wr * a[0] * b;                 /* m_y = y - dy */
                    gc[1] -= wr * a[1] * m->sgn * b;        /* m_z = sgn (zl - dz) */
                }
        }
    }
    free(S);
    return 0;
}

int orc_calib_explain(const orc_params *P, const orc_geom *G, double bz, double v_nom, double vtx_var,
                      const int32_t *tr_sector, const float *tr_x, const float *tr_p, const int32_t *tr_off,
                      const int32_t *tr_clus, const uint8_t *sector, const uint8_t *row, const float *y,
                      const float *t, const float *tcoll, const double *theta, int32_t r, double *F, double *h,
                      double *m, double *v, double *chi2)
{
    const double kb = (double)(-2.99792458e-3f * (float)bz);
    const int n = tr_off[r + 1] - tr_off[r];
    step_t *S = (step_t *)malloc(sizeof(step_t) * (size_t)(n + 1));
    if (!S) return -2;
    anchor_t A;
    const int ok = track_pass(P, G, kb, v_nom, vtx_var, tr_sector, tr_x, tr_p, tr_off, tr_clus, sector, row, y, t,
                              tcoll, theta, r, S, chi2, NAN, 1.0, &A);
    if (ok)
        for (int k = 0; k <= n; k++) {
            memcpy(F + 25 * k, S[k].F, sizeof(double) * 25);
            h[2 * k] = S[k].hy;
            h[2 * k + 1] = S[k].hz;
            m[2 * k] = S[k].my;
            m[2 * k + 1] = S[k].mz;
            v[2 * k] = S[k].vy;
            v[2 * k + 1] = S[k].vz;
        }
    free(S);
    return ok ? 0 : 1;
}

/* Calibration track selection (the reading: tracks from the primary vertex
 * whose collision time is known): a track is used when its refit succeeded
 * and |q/pT| <= qpt_max, decided in binary32 on the binary32 parameter the
 * calibration pass consumes; t_sel = t_coll for a used track, NaN otherwise
 * (low-pT loopers: their later legs do not point to the vertex). */
void orc_calib_select(int32_t n, const float *t_coll, const int32_t *status, const float *param, float qpt_max,
                      float *t_sel)
{
    for (int32_t r = 0; r < n; r++) {
        float q = param[5 * (int64_t)r + 4];
        int keep = status[r] == 0 && fabsf(q) <= qpt_max;
        t_sel[r] = keep ? t_coll[r] : NAN;
    }
}
