/*
 * tpc_oracle.c -- plain, slow CPU oracle of the TPC tracker.
 *
 * TEST INFRASTRUCTURE ONLY: loaded by tests/, the smoke check and the CPU
 * baseline leg of the benchmark, never by the product path.  Shares no code
 * with the CUDA tracker.
 *
 * The paper (section "TPC Tracking") fixes the structure: cellular-automaton
 * seeding is the only combinatorial step, one track hypothesis is followed
 * with a Kalman filter, every later step is linear in the number of hits;
 * section "Tracking" fixes the continuous read-out handling (time scaled to z
 * with the average drift velocity during seeding, primary-track assumption,
 * later refit).  The per-step numbers (windows, cuts, priors, tie-breaks) are
 * readings of a silent paper; this file follows them step by step, in the
 * order seeding -> following -> selection -> merging -> refit.
 *
 * Pins (tests/test_oracle_*.py): propagation and rotation against exact
 * helix crossings (forward and backward), Jacobians against finite
 * differences, the update against the information form, the B = 0 fit
 * against closed-form least squares, exact recovery of noise-free helices,
 * the refit passes' fixed point against a batch least-squares helix fit and
 * their contraction against 1/(1 + refit_inflate), pulls and chi2/ndf, the
 * NeighboursFinder against an exhaustive search with exact binary32
 * emulation, hand-built link cases, the merger's chi2 against noise-free
 * split helices (zero), a closed form (d^T C^-1 d) and the chi2
 * distribution with five degrees of freedom, hand-built straight-line
 * tracklet cases with hand-derived tracklets and tracks (the selector's
 * tie-break in both input orders, following across an empty row, the state
 * against numpy's least-squares line), efficiency / clone / fake rates
 * against generator truth.  The paper prints no worked example of the
 * tracklet constructor, selector or merger: on real events their exact
 * decisions are pinned only by those hand-built cases, the statistical bars
 * and the structural invariants.
 *
 * Build: gcc -O2 -std=c11 -ffp-contract=off -fno-fast-math (see build.py);
 * x86-64 evaluates float in binary32 (FLT_EVAL_METHOD 0), so every float
 * expression below is one correctly rounded binary32 operation and fmaf() is
 * the correctly rounded fused multiply-add.
 */
#include "tpc_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ---------------------------------------------------------------- constants */
#define SNP_MAX   0.999f
#define U_MAX     0.1f
/* arcsine series asin(u)/u = 1 + u^2/6 + 3u^4/40 + 5u^6/112 + ... and its derivative */
#define AS1 0.16666666666666666667f
#define AS2 0.075f
#define AS3 0.044642857142857142857f
#define AD1 0.33333333333333333333f
#define AD2 0.3f
#define AD3 0.26785714285714285714f
#define TAN10 0.17632698070846497347f
#define SIN20 0.34202014332566873304f
#define COS20 0.93969262078590838405f
#define KB_C  (-2.99792458e-3f)    /* d sin(phi)/dx = KB_C * Bz[T] * q/pT[1/GeV] (cm^-1) */

#define NST 21   /* x, p[5], c[15] */
#define MIN_KEEP 5  /* cluster rejection leaves a tracklet at least this many owned hits */

static inline size_t nz(int n) { return n > 0 ? (size_t)n : 1; }
static inline int ci(int i, int j) { return i >= j ? i * (i + 1) / 2 + j : j * (j + 1) / 2 + i; }

void orc_params_default(orc_params *p)
{
    p->dy_link = 3.0f; p->dz_link = 3.0f; p->s_max_link = 0.5f;
    p->sigma_y = 0.1f; p->sigma_z = 0.15f;
    p->c0_snp = 0.25f; p->c0_tgl = 0.25f; p->c0_qpt = 100.0f;
    p->win_nsigma = 3.0f; p->win_min = 0.5f; p->win_max = 3.0f;
    p->chi2_cut = 10.0f;
    p->max_miss = 8; p->min_hits = 10; p->min_owned = 10;
    p->edge_margin = 1.0f;
    p->merge_dz = 10.0f; p->merge_chi2 = 50.0f;
    p->refit_passes = 3;
    p->refit_inflate = 100.0f;
    p->packed_links = 0;
    p->back_jump = 32;
    p->outlier_chi2 = 25.0f;
}

/* ===================================================================== *
 *  Kalman mathematics, binary32 decision path.                          *
 *  State at plane x: (y, z, sin(phi), tan(lambda), q/pT), covariance    *
 *  lower-triangular packed.  Helix in uniform Bz, no material.          *
 * ===================================================================== */

/* covariance C' = F C F^T for F = I + (a e0e2 + b e0e4 + c e1e2 + d e1e3 + e e1e4 + f e2e4) */
static void cov_transport32(float *c, float a, float b, float cc, float d, float e, float f)
{
    float C[5][5], D[5][5];
    for (int i = 0; i < 5; i++)
        for (int j = 0; j < 5; j++) C[i][j] = c[ci(i, j)];
    for (int j = 0; j < 5; j++) {
        D[0][j] = fmaf(b, C[4][j], fmaf(a, C[2][j], C[0][j]));
        D[1][j] = fmaf(e, C[4][j], fmaf(d, C[3][j], fmaf(cc, C[2][j], C[1][j])));
        D[2][j] = fmaf(f, C[4][j], C[2][j]);
        D[3][j] = C[3][j];
        D[4][j] = C[4][j];
    }
    for (int i = 0; i < 5; i++) {
        for (int j = 0; j <= i; j++) {
            float v;
            switch (j) {
            case 0: v = fmaf(b, D[i][4], fmaf(a, D[i][2], D[i][0])); break;
            case 1: v = fmaf(e, D[i][4], fmaf(d, D[i][3], fmaf(cc, D[i][2], D[i][1]))); break;
            case 2: v = fmaf(f, D[i][4], D[i][2]); break;
            case 3: v = D[i][3]; break;
            default: v = D[i][4]; break;
            }
            c[ci(i, j)] = v;
        }
    }
}

/* Propagate to plane x2 along the helix.  sin(phi) is linear in x
 * (s2 = s1 + k dx), dy = dx (s1+s2)/(c1+c2) exactly, the transverse arc is
 * chord * asin(u)/u with u = k chord / 2 (series to u^6, |u| <= 0.1); chord
 * and arc carry the sign of dx. */
int orc_prop32(float *st, float x2, float kb)
{
    float *p = st + 1, *c = st + 6;
    float dx = x2 - st[0];
    if (dx == 0.0f) return 1;
    float k = kb * p[4];
    float s1 = p[2];
    float s2 = fmaf(k, dx, s1);
    if (!(fabsf(s1) < SNP_MAX) || !(fabsf(s2) < SNP_MAX)) return 0;
    float c1 = sqrtf((1.0f - s1) * (1.0f + s1));
    float c2 = sqrtf((1.0f - s2) * (1.0f + s2));
    float ss = s1 + s2, cc = c1 + c2;
    float tt = ss / cc;
    float dy = dx * tt;
    float dl0 = sqrtf(fmaf(dx, dx, dy * dy));
    float dl = dx < 0.0f ? -dl0 : dl0;
    float u = (0.5f * k) * dl;
    if (!(fabsf(u) <= U_MAX)) return 0;
    float u2 = u * u;
    float A = fmaf(u2, fmaf(u2, fmaf(u2, AS3, AS2), AS1), 1.0f);
    float dS = dl * A;
    float dz = dS * p[3];
    /* Jacobian: d(dy)/d(s1), d(dy)/dk, d(dS)/d(s1), d(dS)/dk */
    float r1 = s1 / c1, r2 = s2 / c2;
    float cc2 = cc * cc;
    float dt_ds = fmaf(ss, r1 + r2, 2.0f * cc) / cc2;
    float dt_dk = (dx * fmaf(ss, r2, cc)) / cc2;
    float dy_ds = dx * dt_ds;
    float dy_dk = dx * dt_dk;
    float g = dy / dl;
    float B = 1.0f / sqrtf((1.0f - u) * (1.0f + u));
    float dS_ds = B * (g * dy_ds);
    float Ap = u * fmaf(u2, fmaf(u2, AD3, AD2), AD1);
    float h2 = ((0.5f * dl) * dl) * Ap;
    float dS_dk = fmaf(B, g * dy_dk, h2);
    float ja = dy_ds;
    float jb = dy_dk * kb;
    float jc = p[3] * dS_ds;
    float jd = dS;
    float je = (p[3] * dS_dk) * kb;
    float jf = dx * kb;
    cov_transport32(c, ja, jb, jc, jd, je, jf);
    st[0] = x2;
    p[0] = p[0] + dy;
    p[1] = p[1] + dz;
    p[2] = s2;
    return 1;
}

/* Rotate the local frame by +angle (cs = cos, sn = sin): the state is then at
 * x' = x cs + y sn in the new frame.  First-order Jacobian at fixed x'. */
int orc_rot32(float *st, float cs, float sn, float kb)
{
    float *p = st + 1, *c = st + 6;
    float x = st[0], y = p[0], sp = p[2];
    float cf = sqrtf((1.0f - sp) * (1.0f + sp));
    float spn = fmaf(sp, cs, -(cf * sn));
    float cfn = fmaf(cf, cs, sp * sn);
    if (!(fabsf(spn) < SNP_MAX) || !(cfn > 0.0f)) return 0;
    float xn = fmaf(x, cs, y * sn);
    float yn = fmaf(-x, sn, y * cs);
    float k = kb * p[4];
    float J00 = cf / cfn;
    float J10 = -(sn * p[3]) / cfn;
    float J20 = -(k * sn);
    float J22 = cfn / cf;
    float C[5][5], D[5][5];
    for (int i = 0; i < 5; i++)
        for (int j = 0; j < 5; j++) C[i][j] = c[ci(i, j)];
    for (int j = 0; j < 5; j++) {
        D[0][j] = J00 * C[0][j];
        D[1][j] = fmaf(J10, C[0][j], C[1][j]);
        D[2][j] = fmaf(J22, C[2][j], J20 * C[0][j]);
        D[3][j] = C[3][j];
        D[4][j] = C[4][j];
    }
    for (int i = 0; i < 5; i++) {
        for (int j = 0; j <= i; j++) {
            float v;
            switch (j) {
            case 0: v = J00 * D[i][0]; break;
            case 1: v = fmaf(J10, D[i][0], D[i][1]); break;
            case 2: v = fmaf(J22, D[i][2], J20 * D[i][0]); break;
            case 3: v = D[i][3]; break;
            default: v = D[i][4]; break;
            }
            c[ci(i, j)] = v;
        }
    }
    st[0] = xn;
    p[0] = yn;
    p[2] = spn;
    return 1;
}

/* Kalman update with the measurement (my, mz), V = diag(vy, vz), H = [I2 0];
 * rejected (state untouched) when the predicted chi2 exceeds chi2max. */
int orc_update32(float *st, float my, float mz, float vy, float vz, float chi2max, float *chi2o)
{
    float *p = st + 1, *c = st + 6;
    float r0 = my - p[0], r1 = mz - p[1];
    float s00 = c[0] + vy, s01 = c[1], s11 = c[2] + vz;
    float det = fmaf(s00, s11, -(s01 * s01));
    if (!(det > 0.0f)) return 0;
    float idet = 1.0f / det;
    float i00 = s11 * idet, i01 = -(s01 * idet), i11 = s00 * idet;
    float a0 = fmaf(i00, r0, i01 * r1);
    float a1 = fmaf(i01, r0, i11 * r1);
    float chi2 = fmaf(r0, a0, r1 * a1);
    if (chi2o) *chi2o = chi2;
    if (!(chi2 <= chi2max)) return 0;
    float K0[5], K1[5], row0[5], row1[5];
    for (int i = 0; i < 5; i++) {
        float c0 = c[ci(i, 0)], c1 = c[ci(i, 1)];
        K0[i] = fmaf(c0, i00, c1 * i01);
        K1[i] = fmaf(c0, i01, c1 * i11);
        row0[i] = c0;
        row1[i] = c1;
    }
    for (int i = 0; i < 5; i++) p[i] = p[i] + fmaf(K0[i], r0, K1[i] * r1);
    for (int i = 0; i < 5; i++)
        for (int j = 0; j <= i; j++)
            c[ci(i, j)] = c[ci(i, j)] - fmaf(K0[i], row0[j], K1[i] * row1[j]);
    return 1;
}

/* chi2 of two states of one track (outer end of A, inner end of B in the
 * neighbouring sector): A is rotated into B's frame, propagated to B's x,
 * chi2 = d^T (C_A + C_B)^-1 d over all five parameters (Cholesky). */
float orc_merge_chi2(const float *top, const float *bot, float cs, float sn, float kb)
{
    float t[NST];
    memcpy(t, top, sizeof(t));
    if (!orc_rot32(t, cs, sn, kb)) return INFINITY;
    if (!orc_prop32(t, bot[0], kb)) return INFINITY;
    float d[5], S[15], L[15], v[5];
    for (int i = 0; i < 5; i++) d[i] = t[1 + i] - bot[1 + i];
    for (int i = 0; i < 15; i++) S[i] = t[6 + i] + bot[6 + i];
    for (int i = 0; i < 5; i++) {
        for (int j = 0; j <= i; j++) {
            float s = S[ci(i, j)];
            for (int k = 0; k < j; k++) s = fmaf(-L[ci(i, k)], L[ci(j, k)], s);
            if (i == j) {
                if (!(s > 0.0f)) return INFINITY;
                L[ci(i, i)] = sqrtf(s);
            } else {
                L[ci(i, j)] = s / L[ci(j, j)];
            }
        }
    }
    float chi2 = 0.0f;
    for (int i = 0; i < 5; i++) {
        float s = d[i];
        for (int k = 0; k < i; k++) s = fmaf(-L[ci(i, k)], v[k], s);
        v[i] = s / L[ci(i, i)];
        chi2 = fmaf(v[i], v[i], chi2);
    }
    return chi2;
}

/* ===================================================================== *
 *  Kalman mathematics, binary64 refit (exact arcsine).                  *
 * ===================================================================== */
static void asin_ratio(double u, double *A, double *Ap)
{
    /* A = asin(u)/u and dA/du; series for small |u| to avoid cancellation */
    double u2 = u * u;
    if (fabs(u) < 0.05) {
        *A = 1 + u2 * (1.0 / 6 + u2 * (3.0 / 40 + u2 * (5.0 / 112 + u2 * (35.0 / 1152 + u2 * 63.0 / 2816))));
        *Ap = u * (1.0 / 3 + u2 * (3.0 / 10 + u2 * (15.0 / 56 + u2 * (35.0 / 144 + u2 * 315.0 / 1408))));
    } else {
        double as = asin(u);
        *A = as / u;
        *Ap = (u / sqrt(1 - u2) - as) / u2;
    }
}

static void sandwich64(double *c, double F[5][5])
{
    double C[5][5], T[5][5];
    for (int i = 0; i < 5; i++)
        for (int j = 0; j < 5; j++) C[i][j] = c[ci(i, j)];
    for (int i = 0; i < 5; i++)
        for (int j = 0; j < 5; j++) {
            double s = 0;
            for (int k = 0; k < 5; k++) s += F[i][k] * C[k][j];
            T[i][j] = s;
        }
    for (int i = 0; i < 5; i++)
        for (int j = 0; j <= i; j++) {
            double s = 0;
            for (int k = 0; k < 5; k++) s += T[i][k] * F[j][k];
            c[ci(i, j)] = s;
        }
}

int orc_helix64(double *x, double *p, double x2, double kb, double F[5][5])
{
    for (int i = 0; i < 5; i++)
        for (int j = 0; j < 5; j++) F[i][j] = i == j;
    double dx = x2 - *x;
    if (dx == 0.0) return 1;
    double k = kb * p[4];
    double s1 = p[2], s2 = s1 + k * dx;
    if (!(fabs(s1) < 0.999) || !(fabs(s2) < 0.999)) return 0;
    double c1 = sqrt((1 - s1) * (1 + s1)), c2 = sqrt((1 - s2) * (1 + s2));
    double ss = s1 + s2, cc = c1 + c2;
    double dy = dx * ss / cc;
    double dl = copysign(sqrt(dx * dx + dy * dy), dx);
    double u = 0.5 * k * dl;
    if (!(fabs(u) < 1.0)) return 0;
    double A, Ap;
    asin_ratio(u, &A, &Ap);
    double dS = dl * A;
    double dz = dS * p[3];
    double r1 = s1 / c1, r2 = s2 / c2;
    double dy_ds = dx * (2 * cc + ss * (r1 + r2)) / (cc * cc);
    double dy_dk = dx * dx * (cc + ss * r2) / (cc * cc);
    double g = dy / dl;
    double B = 1 / sqrt((1 - u) * (1 + u));
    double dS_ds = B * g * dy_ds;
    double dS_dk = B * g * dy_dk + 0.5 * dl * dl * Ap;
    F[0][2] = dy_ds; F[0][4] = dy_dk * kb;
    F[1][2] = p[3] * dS_ds; F[1][3] = dS; F[1][4] = p[3] * dS_dk * kb;
    F[2][4] = dx * kb;
    *x = x2;
    p[0] += dy;
    p[1] += dz;
    p[2] = s2;
    return 1;
}

int orc_prop64(double *st, double x2, double kb)
{
    double F[5][5];
    if (x2 == st[0]) return 1;
    if (!orc_helix64(&st[0], st + 1, x2, kb, F)) return 0;
    sandwich64(st + 6, F);
    return 1;
}

int orc_rotate64(double *x, double *p, double cs, double sn, double kb, double J[5][5])
{
    for (int i = 0; i < 5; i++)
        for (int j = 0; j < 5; j++) J[i][j] = i == j;
    double y = p[0], sp = p[2];
    double cf = sqrt((1 - sp) * (1 + sp));
    double spn = sp * cs - cf * sn;
    double cfn = cf * cs + sp * sn;
    if (!(fabs(spn) < 0.999) || !(cfn > 0)) return 0;
    double k = kb * p[4];
    J[0][0] = cf / cfn;
    J[1][0] = -sn * p[3] / cfn;
    J[2][0] = -k * sn;
    J[2][2] = cfn / cf;
    double x0 = *x;
    *x = x0 * cs + y * sn;
    p[0] = -x0 * sn + y * cs;
    p[2] = spn;
    return 1;
}

int orc_rot64(double *st, double cs, double sn, double kb)
{
    double J[5][5];
    if (!orc_rotate64(&st[0], st + 1, cs, sn, kb, J)) return 0;
    sandwich64(st + 6, J);
    return 1;
}

int orc_update64(double *st, double my, double mz, double vy, double vz, double *chi2o)
{
    double *p = st + 1, *c = st + 6;
    double r0 = my - p[0], r1 = mz - p[1];
    double s00 = c[0] + vy, s01 = c[1], s11 = c[2] + vz;
    double det = s00 * s11 - s01 * s01;
    if (!(det > 0)) return 0;
    double i00 = s11 / det, i01 = -s01 / det, i11 = s00 / det;
    double chi2 = r0 * (i00 * r0 + i01 * r1) + r1 * (i01 * r0 + i11 * r1);
    if (chi2o) *chi2o = chi2;
    double K0[5], K1[5], row0[5], row1[5];
    for (int i = 0; i < 5; i++) {
        double c0 = c[ci(i, 0)], c1 = c[ci(i, 1)];
        K0[i] = c0 * i00 + c1 * i01;
        K1[i] = c0 * i01 + c1 * i11;
        row0[i] = c0;
        row1[i] = c1;
    }
    for (int i = 0; i < 5; i++) p[i] += K0[i] * r0 + K1[i] * r1;
    for (int i = 0; i < 5; i++)
        for (int j = 0; j <= i; j++) c[ci(i, j)] -= K0[i] * row0[j] + K1[i] * row1[j];
    return 1;
}

static double sector_alpha64(int s, int n_sectors)
{
    if (n_sectors == 1) return 10.0 * M_PI / 180.0;
    return ((s % 18) * 20.0 + 10.0) * M_PI / 180.0;
}

/* Multi-pass refit ("multiple fit iterations", section "TPC Tracking"):
 * pass 1 runs from the outermost cluster inwards, the next pass outwards,
 * and so on.  Each pass restarts from the previous fit's state: y, z from
 * the first measurement (variance sigma^2, no correlations), sin(phi),
 * tan(lambda), q/pT with the previous covariance block times refit_inflate
 * (pass 1 starts from the tracklet's outer-end fit).  A fixed point of the
 * passes is the least-squares fit; keeping the previous angular covariance,
 * instead of a wide diagonal prior, keeps the filter well conditioned where
 * a looper runs nearly parallel to the pad rows.  Clusters in another sector
 * are reached by rotating the frame. */
int orc_fit64(const orc_params *P, const orc_geom *G, double kb, int32_t n,
              const int32_t *sector, const double *x, const double *y, const double *z,
              int32_t n_passes, double *st, double *chi2o)
{
    double vy = (double)P->sigma_y * P->sigma_y, vz = (double)P->sigma_z * P->sigma_z;
    int sec = sector[n - 1];
    double chi2 = 0;
    for (int pass = 0; pass < n_passes; pass++) {
        int inward = (pass % 2) == 0;
        chi2 = 0;
        for (int q = 0; q < n; q++) {
            int i = inward ? n - 1 - q : q;
            if (sector[i] != sec) {
                double da = sector_alpha64(sector[i], G->n_sectors) - sector_alpha64(sec, G->n_sectors);
                while (da > M_PI) da -= 2 * M_PI;
                while (da <= -M_PI) da += 2 * M_PI;
                if (!orc_rot64(st, cos(da), sin(da), kb)) { *chi2o = chi2; return 0; }
                sec = sector[i];
            }
            if (!orc_prop64(st, x[i], kb)) { *chi2o = chi2; return 0; }
            if (q == 0) {
                /* restart: position from the first measurement, its
                 * correlations dropped; angles and curvature keep the
                 * previous fit's covariance inflated by refit_inflate */
                double *c = st + 6;
                st[1] = y[i];
                st[2] = z[i];
                c[0] = vy; c[1] = 0; c[2] = vz;
                for (int a = 2; a < 5; a++) {
                    c[a * (a + 1) / 2 + 0] = 0;
                    c[a * (a + 1) / 2 + 1] = 0;
                    for (int b = 2; b <= a; b++) c[a * (a + 1) / 2 + b] *= (double)P->refit_inflate;
                }
            } else {
                double c2;
                if (!orc_update64(st, y[i], z[i], vy, vz, &c2)) { *chi2o = chi2; return 0; }
                chi2 += c2;
            }
        }
    }
    *chi2o = chi2;
    return 1;
}

/* ===================================================================== *
 *  The tracker.                                                         *
 * ===================================================================== */
typedef struct {
    int n, n_rows, n_planes;
    const float *y, *z;
    int32_t *ord;        /* cluster indices sorted by (plane, z, index) */
    int32_t *pstart;     /* [n_planes + 1] */
    float *zs;           /* z in sorted order */
} grid_t;

static const float *g_sort_z;
static const int32_t *g_sort_pl;
static int cmp_cluster(const void *a, const void *b)
{
    int32_t i = *(const int32_t *)a, j = *(const int32_t *)b;
    if (g_sort_pl[i] != g_sort_pl[j]) return g_sort_pl[i] < g_sort_pl[j] ? -1 : 1;
    if (g_sort_z[i] != g_sort_z[j]) return g_sort_z[i] < g_sort_z[j] ? -1 : 1;
    return (i > j) - (i < j);
}

/* first position in plane pl with z >= zlo (plain binary search) */
static int plane_lower(const grid_t *g, int pl, double zlo)
{
    int lo = g->pstart[pl], hi = g->pstart[pl + 1];
    while (lo < hi) {
        int mid = (lo + hi) / 2;
        if ((double)g->zs[mid] < zlo) lo = mid + 1; else hi = mid;
    }
    return lo;
}

/* Nearest cluster of plane pl inside |dy| <= wy, |dz| <= wz of (yp, zp):
 * minimum dy^2 + dz^2 (binary32, fused), ties to the smaller cluster index.
 * The z scan range is a superset of the window; the window test decides. */
static int find_nearest(const grid_t *g, int pl, float yp, float zp, float wy, float wz)
{
    int best = -1;
    float bd = 0.0f;
    int end = g->pstart[pl + 1];
    for (int q = plane_lower(g, pl, (double)zp - 2.0 * wz - 1.0); q < end; q++) {
        if ((double)g->zs[q] > (double)zp + 2.0 * wz + 1.0) break;
        int c = g->ord[q];
        float dy = g->y[c] - yp;
        float dz = g->z[c] - zp;
        if (!(fabsf(dy) <= wy) || !(fabsf(dz) <= wz)) continue;
        float d2 = fmaf(dy, dy, dz * dz);
        if (best < 0 || d2 < bd || (d2 == bd && c < best)) { best = c; bd = d2; }
    }
    return best;
}

typedef struct { int n, cap; int32_t *v; } ivec;
static void iv_push(ivec *a, int32_t x)
{
    if (a->n == a->cap) {
        a->cap = a->cap ? 2 * a->cap : 64;
        a->v = (int32_t *)realloc(a->v, (size_t)a->cap * sizeof(int32_t));
    }
    a->v[a->n++] = x;
}

/* merge partner sector of s: dir +1 / -1 the next / previous wedge of the
 * same side, dir 0 the same wedge on the other side of the central membrane */
static int neighbour_sector(int s, int dir, int n_sectors)
{
    if (n_sectors != 36) return -1;
    int side = s / 18, w = s % 18;
    if (dir == 0) return (1 - side) * 18 + w;
    return side * 18 + (w + (dir > 0 ? 1 : 17)) % 18;
}

static uint64_t tracklet_weight(int nhits, int start)
{
    return ((uint64_t)(uint32_t)nhits << 32) | (uint64_t)(0xFFFFFFFFu - (uint32_t)start);
}

int orc_track(const orc_params *P, const orc_geom *G, float bz, float v_drift, int32_t n,
              const uint8_t *sector, const uint8_t *row, const float *y, const float *zt,
              orc_result *R)
{
    memset(R, 0, sizeof(*R));
    R->n = n;
    const int NR = G->n_rows;
    const float *X = G->row_x;
    const float vy = P->sigma_y * P->sigma_y, vz = P->sigma_z * P->sigma_z;
    const float kb = KB_C * bz;
    if (NR < 3 || NR > 256 || n < 0) return -1;
    for (int i = 0; i < n; i++)
        if (sector[i] >= G->n_sectors || row[i] >= NR) return -2;

    /* per-row binary32 tables: q_up = X[r+1]/X[r], q_dn = X[r-1]/X[r],
     * w = (X[r]-X[r-1]) / (X[r+1]-X[r-1]) */
    for (int r = 1; r + 1 < NR; r++) {
        R->row_qup[r] = X[r + 1] / X[r];
        R->row_qdn[r] = X[r - 1] / X[r];
        R->row_w[r] = (X[r] - X[r - 1]) / (X[r + 1] - X[r - 1]);
    }

    /* ---- a1: time -> z, linear in the average drift velocity (section
     * "Tracking", first bullet): z = s (Zmax - v t), s = +1 on the A side. */
    R->z = (float *)malloc(sizeof(float) * nz(n));
    for (int i = 0; i < n; i++) {
        if (G->continuous) {
            float zl = G->z_max - v_drift * zt[i];
            R->z[i] = (G->n_sectors == 36 && sector[i] >= 18) ? -zl : zl;
        } else {
            R->z[i] = zt[i];
        }
    }

    /* ---- a2: per-row grid: clusters of each (sector, row) plane sorted by z */
    grid_t g;
    g.n = n; g.n_rows = NR; g.n_planes = G->n_sectors * NR;
    g.y = y; g.z = R->z;
    int32_t *pl = (int32_t *)malloc(sizeof(int32_t) * nz(n));
    for (int i = 0; i < n; i++) pl[i] = sector[i] * NR + row[i];
    g.ord = (int32_t *)malloc(sizeof(int32_t) * nz(n));
    for (int i = 0; i < n; i++) g.ord[i] = i;
    g_sort_z = R->z; g_sort_pl = pl;
    qsort(g.ord, (size_t)n, sizeof(int32_t), cmp_cluster);
    g.pstart = (int32_t *)calloc((size_t)g.n_planes + 1, sizeof(int32_t));
    for (int i = 0; i < n; i++) g.pstart[pl[i] + 1]++;
    for (int p = 0; p < g.n_planes; p++) g.pstart[p + 1] += g.pstart[p];
    g.zs = (float *)malloc(sizeof(float) * nz(n));
    for (int q = 0; q < n; q++) g.zs[q] = R->z[g.ord[q]];

    /* ---- a3: NeighboursFinder.  For each hit on rows 1..NR-2: candidates on
     * the rows above/below inside |y_c - y q| <= DY (primary assumption in the
     * bending plane: y scales with x), |z_c - z| <= DZ; the pair (up, down)
     * whose chord passes closest to the hit, score < S_MAX, ties to the
     * smaller (up, down) cluster indices. */
    R->up_raw = (int32_t *)malloc(sizeof(int32_t) * nz(n));
    R->dn_raw = (int32_t *)malloc(sizeof(int32_t) * nz(n));
    /* Packed-coordinate variant (configuration of the batched workload): the
     * link pass sees every coordinate rounded to the nearest multiple of
     * 2^-8 cm (ties to even), i.e. the value a 16-bit packed field of a
     * fixed-point coordinate with that step decodes to. */
    const float *ly = y, *lzc = R->z;
    float *qy = NULL, *qz = NULL;
    if (P->packed_links) {
        qy = (float *)malloc(sizeof(float) * nz(n));
        qz = (float *)malloc(sizeof(float) * nz(n));
        for (int i = 0; i < n; i++) {
            qy[i] = rintf(y[i] * 256.0f) * 0.00390625f;
            qz[i] = rintf(R->z[i] * 256.0f) * 0.00390625f;
        }
        ly = qy;
        lzc = qz;
    }
    ivec U = {0, 0, NULL}, D = {0, 0, NULL};
    for (int h = 0; h < n; h++) {
        R->up_raw[h] = -1; R->dn_raw[h] = -1;
        int r = row[h];
        if (r < 1 || r > NR - 2) continue;
        int s = sector[h];
        float yh = ly[h], zh = lzc[h];
        float yu_pred = yh * R->row_qup[r];
        float yd_pred = yh * R->row_qdn[r];
        U.n = 0; D.n = 0;
        for (int side = 0; side < 2; side++) {
            int plq = s * NR + (side == 0 ? r + 1 : r - 1);
            float ypred = side == 0 ? yu_pred : yd_pred;
            int end = g.pstart[plq + 1];
            for (int q = plane_lower(&g, plq, (double)zh - 2.0 * P->dz_link - 1.0); q < end; q++) {
                if ((double)g.zs[q] > (double)zh + 2.0 * P->dz_link + 1.0) break;
                int c = g.ord[q];
                if (fabsf(ly[c] - ypred) <= P->dy_link && fabsf(lzc[c] - zh) <= P->dz_link)
                    iv_push(side == 0 ? &U : &D, c);
            }
        }
        float w = R->row_w[r];
        int bu = -1, bd = -1;
        float bs = 0.0f;
        for (int a = 0; a < U.n; a++) {
            int u = U.v[a];
            for (int b = 0; b < D.n; b++) {
                int d = D.v[b];
                float ey = fmaf(ly[u] - ly[d], w, ly[d]) - yh;
                float ez = fmaf(lzc[u] - lzc[d], w, lzc[d]) - zh;
                float sc = fmaf(ey, ey, ez * ez);
                if (!(sc < P->s_max_link)) continue;
                if (bu < 0 || sc < bs || (sc == bs && (u < bu || (u == bu && d < bd)))) {
                    bu = u; bd = d; bs = sc;
                }
            }
        }
        R->up_raw[h] = bu;
        R->dn_raw[h] = bd;
    }
    free(U.v); free(D.v);
    free(qy); free(qz);

    /* ---- a4: NeighboursCleaner: keep only mutual links */
    R->up = (int32_t *)malloc(sizeof(int32_t) * nz(n));
    R->dn = (int32_t *)malloc(sizeof(int32_t) * nz(n));
    for (int h = 0; h < n; h++) {
        int u = R->up_raw[h], d = R->dn_raw[h];
        R->up[h] = (u >= 0 && R->dn_raw[u] == h) ? u : -1;
        R->dn[h] = (d >= 0 && R->up_raw[d] == h) ? d : -1;
    }

    /* ---- a5: StartHitsFinder: an up link, no down link, chain of >= 3 hits */
    R->is_start = (uint8_t *)malloc(nz(n));
    int nt = 0;
    for (int h = 0; h < n; h++) {
        int u = R->up[h];
        R->is_start[h] = (u >= 0 && R->dn[h] < 0 && R->up[u] >= 0) ? 1 : 0;
        nt += R->is_start[h];
    }

    /* ---- a6: TrackletConstructor (binary32, one hypothesis per start) */
    R->n_tracklets = nt;
    R->trk_start = (int32_t *)malloc(sizeof(int32_t) * nz(nt));
    R->trk_nhits = (int32_t *)malloc(sizeof(int32_t) * nz(nt));
    R->trk_off = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nt + 1));
    R->trk_top = (float *)malloc(sizeof(float) * NST * nz(nt));
    R->trk_bot = (float *)malloc(sizeof(float) * NST * nz(nt));
    ivec hits = {0, 0, NULL};
    int32_t *up_list = (int32_t *)malloc(sizeof(int32_t) * (size_t)NR);
    int32_t *dn_list = (int32_t *)malloc(sizeof(int32_t) * (size_t)NR);
    R->trk_off[0] = 0;
    int t = 0;
    for (int h1 = 0; h1 < n; h1++) {
        if (!R->is_start[h1]) continue;
        int s = sector[h1], r1 = row[h1];
        int h2 = R->up[h1];
        float st[NST], top[NST], bot[NST];
        /* initial state at the start hit: y, z measured, slopes from the first link */
        float x1 = X[r1], x2 = X[r1 + 1];
        float dx12 = x2 - x1;
        float dy12 = y[h2] - y[h1], dz12 = R->z[h2] - R->z[h1];
        float ty = dy12 / dx12;
        float sp = ty / sqrtf(fmaf(ty, ty, 1.0f));
        float dl12 = sqrtf(fmaf(dx12, dx12, dy12 * dy12));
        float tl = dz12 / dl12;
        memset(st, 0, sizeof(st));
        st[0] = x1; st[1] = y[h1]; st[2] = R->z[h1]; st[3] = sp; st[4] = tl; st[5] = 0.0f;
        st[6 + 0] = vy; st[6 + 2] = vz; st[6 + 5] = P->c0_snp; st[6 + 9] = P->c0_tgl; st[6 + 14] = P->c0_qpt;
        int nu = 0, nd = 0;
        up_list[nu++] = h1;
        memcpy(top, st, sizeof(st));
        int rc = r1;         /* row of the current state */
        int ok = 1;
        /* phase A: fit along the up links */
        for (int hc = h1; R->up[hc] >= 0;) {
            int hn = R->up[hc];
            int rn = row[hn];
            if (!orc_prop32(st, X[rn], kb)) { ok = 0; break; }
            rc = rn;
            orc_update32(st, y[hn], R->z[hn], vy, vz, INFINITY, NULL);
            up_list[nu++] = hn;
            memcpy(top, st, sizeof(st));
            hc = hn;
        }
        /* phase B: follow row by row beyond the chain end */
        if (ok) {
            int miss = 0;
            for (int r = rc + 1; r < NR; r++) {
                if (!orc_prop32(st, X[r], kb)) break;
                rc = r;
                if (fabsf(st[1]) > fmaf(st[0], TAN10, P->edge_margin)) break;
                float wy = fminf(fmaxf(P->win_nsigma * sqrtf(st[6 + 0] + vy), P->win_min), P->win_max);
                float wz = fminf(fmaxf(P->win_nsigma * sqrtf(st[6 + 2] + vz), P->win_min), P->win_max);
                int c = find_nearest(&g, s * NR + r, st[1], st[2], wy, wz);
                if (c >= 0 && orc_update32(st, y[c], R->z[c], vy, vz, P->chi2_cut, NULL)) {
                    up_list[nu++] = c;
                    memcpy(top, st, sizeof(st));
                    miss = 0;
                } else if (++miss >= P->max_miss) {
                    break;
                }
            }
        }
        /* phase C: back to the start row in jumps of at most back_jump rows
         * (a refused jump -- |u| or |sin(phi)| out of range -- is retried
         * with half as many rows; a refused single-row step ends the
         * tracklet), then follow row by row below the start */
        memcpy(bot, top, sizeof(st));
        if (rc == r1) memcpy(bot, st, sizeof(st));
        int back_ok = 1;
        for (int jump = P->back_jump > 0 ? P->back_jump : 1; rc > r1;) {
            int tgt = rc - jump > r1 ? rc - jump : r1;
            if (orc_prop32(st, X[tgt], kb)) {
                rc = tgt;
                if (rc == r1) memcpy(bot, st, sizeof(st));
            } else if (jump > 1) {
                jump >>= 1;
            } else {
                back_ok = 0;
                break;
            }
        }
        if (back_ok) {
            int miss = 0;
            for (int r = r1 - 1; r >= 0; r--) {
                if (!orc_prop32(st, X[r], kb)) break;
                if (fabsf(st[1]) > fmaf(st[0], TAN10, P->edge_margin)) break;
                float wy = fminf(fmaxf(P->win_nsigma * sqrtf(st[6 + 0] + vy), P->win_min), P->win_max);
                float wz = fminf(fmaxf(P->win_nsigma * sqrtf(st[6 + 2] + vz), P->win_min), P->win_max);
                int c = find_nearest(&g, s * NR + r, st[1], st[2], wy, wz);
                if (c >= 0 && orc_update32(st, y[c], R->z[c], vy, vz, P->chi2_cut, NULL)) {
                    dn_list[nd++] = c;
                    memcpy(bot, st, sizeof(st));
                    miss = 0;
                } else if (++miss >= P->max_miss) {
                    break;
                }
            }
        }
        R->trk_start[t] = h1;
        R->trk_nhits[t] = nu + nd;
        for (int q = nd - 1; q >= 0; q--) iv_push(&hits, dn_list[q]);
        for (int q = 0; q < nu; q++) iv_push(&hits, up_list[q]);
        R->trk_off[t + 1] = hits.n;
        memcpy(R->trk_top + (size_t)t * NST, top, sizeof(top));
        memcpy(R->trk_bot + (size_t)t * NST, bot, sizeof(bot));
        t++;
    }
    free(up_list); free(dn_list);
    R->trk_hits = hits.v ? hits.v : (int32_t *)malloc(sizeof(int32_t));

    /* ---- a7: TrackletSelector: each hit goes to the tracklet with the most
     * hits (ties: smaller start index); a tracklet survives with >= min_owned
     * owned hits and at least half of its own hits. */
    uint64_t *hitw = (uint64_t *)calloc(nz(n), sizeof(uint64_t));
    for (int q = 0; q < nt; q++) {
        if (R->trk_nhits[q] < P->min_hits) continue;
        uint64_t w = tracklet_weight(R->trk_nhits[q], R->trk_start[q]);
        for (int k = R->trk_off[q]; k < R->trk_off[q + 1]; k++) {
            int c = R->trk_hits[k];
            if (w > hitw[c]) hitw[c] = w;
        }
    }
    R->trk_kept = (uint8_t *)calloc(nz(nt), 1);
    int ns = 0;
    for (int q = 0; q < nt; q++) {
        if (R->trk_nhits[q] < P->min_hits) continue;
        uint64_t w = tracklet_weight(R->trk_nhits[q], R->trk_start[q]);
        int own = 0;
        for (int k = R->trk_off[q]; k < R->trk_off[q + 1]; k++) own += hitw[R->trk_hits[k]] == w;
        if (own >= P->min_owned && 2 * own >= R->trk_nhits[q]) { R->trk_kept[q] = 1; ns++; }
    }

    /* ---- cluster rejection before the refit (section "TPC Tracking": the
     * track fit rejects clusters).  Reading: each kept tracklet's inner-end
     * state -- binary32, after all of its hits -- is carried row by row with
     * the decision-path propagation up through the rows of its hits; an
     * owned hit whose residual to it passes dy^2/vy + dz^2/vz > outlier_chi2
     * is rejected: it leaves the track's cluster list, the refit and the
     * assignment.  A refused step ends the check of that tracklet.  A
     * tracklet that would keep fewer than MIN_KEEP owned hits rejects none. */
    R->rejected = (uint8_t *)calloc(nz(n), 1);
    R->n_rejected = 0;
    if (P->outlier_chi2 > 0.0f) {
        const float ivy = 1.0f / vy, ivz = 1.0f / vz;
        int32_t *cand = (int32_t *)malloc(sizeof(int32_t) * (size_t)NR);
        for (int q = 0; q < nt; q++) {
            if (!R->trk_kept[q]) continue;
            uint64_t w = tracklet_weight(R->trk_nhits[q], R->trk_start[q]);
            int own = 0, nc = 0;
            for (int k = R->trk_off[q]; k < R->trk_off[q + 1]; k++) own += hitw[R->trk_hits[k]] == w;
            float st[NST];
            memcpy(st, R->trk_bot + (size_t)q * NST, sizeof(st));
            for (int k = R->trk_off[q]; k < R->trk_off[q + 1]; k++) {
                int c = R->trk_hits[k];
                if (!orc_prop32(st, X[row[c]], kb)) break;
                float dy = y[c] - st[1];
                float dz = R->z[c] - st[2];
                float q2 = fmaf(dy * dy, ivy, (dz * dz) * ivz);
                if (hitw[c] == w && q2 > P->outlier_chi2) cand[nc++] = c;
            }
            if (own - nc < MIN_KEEP) continue;
            for (int k = 0; k < nc; k++) R->rejected[cand[k]] = 1;
            R->n_rejected += nc;
        }
        free(cand);
    }

    /* ---- a8: cross-sector merger: adjacent sectors of one side and, where
     * the clusters carry z, the mirror sector across the central membrane.
     * The two sides share the wedge's local frame (no rotation); with drift
     * times the two halves of a crossing track are displaced in z by twice
     * the drift over the unknown collision time, so that pair is not tried. */
    R->n_seg = ns;
    R->seg_trk = (int32_t *)malloc(sizeof(int32_t) * nz(ns));
    R->seg_next = (int32_t *)malloc(sizeof(int32_t) * nz(ns));
    R->seg_prev = (int32_t *)malloc(sizeof(int32_t) * nz(ns));
    for (int q = 0, k = 0; q < nt; q++)
        if (R->trk_kept[q]) R->seg_trk[k++] = q;
    int32_t *best_next = (int32_t *)malloc(sizeof(int32_t) * nz(ns));
    int32_t *best_prev = (int32_t *)malloc(sizeof(int32_t) * nz(ns));
    int NS = G->n_sectors;
    int32_t *sstart = (int32_t *)calloc((size_t)NS + 1, sizeof(int32_t));
    int32_t *sidx = (int32_t *)malloc(sizeof(int32_t) * nz(ns));
    for (int a = 0; a < ns; a++) sstart[sector[R->trk_start[R->seg_trk[a]]] + 1]++;
    for (int q = 0; q < NS; q++) sstart[q + 1] += sstart[q];
    {
        int32_t *fill = (int32_t *)malloc(sizeof(int32_t) * (size_t)NS);
        for (int q = 0; q < NS; q++) fill[q] = sstart[q];
        for (int a = 0; a < ns; a++) sidx[fill[sector[R->trk_start[R->seg_trk[a]]]]++] = a;
        free(fill);
    }
    for (int a = 0; a < ns; a++) { best_next[a] = -1; best_prev[a] = -1; }
    /* A's outer end -> B's inner end; best B for each A and best A for each B
     * (minimum chi2, ties to the smaller start index) */
    float *bchi_n = (float *)malloc(sizeof(float) * nz(ns));
    float *bchi_p = (float *)malloc(sizeof(float) * nz(ns));
    for (int a = 0; a < ns; a++) {
        int ta = R->seg_trk[a];
        int sa = sector[R->trk_start[ta]];
        const float *top = R->trk_top + (size_t)ta * NST;
        for (int dir = 1; dir >= -1; dir--) {
            if (dir == 0 && G->continuous) continue;
            int sb = neighbour_sector(sa, dir, NS);
            if (sb < 0) continue;
            float cs = dir == 0 ? 1.0f : COS20;
            float sn = dir > 0 ? SIN20 : (dir < 0 ? -SIN20 : 0.0f);
            for (int q = sstart[sb]; q < sstart[sb + 1]; q++) {
                int b = sidx[q];
                int tb = R->seg_trk[b];
                const float *bot = R->trk_bot + (size_t)tb * NST;
                /* across the membrane B must continue A outward (one frame:
                 * B's inner end not inside A's outer end); the pair taken
                 * the other way round fits as well at small dip angles and
                 * would close a two-segment cycle */
                if (dir == 0 && !(bot[0] >= top[0])) continue;
                if (!(fabsf(bot[2] - top[2]) <= P->merge_dz)) continue;
                /* screen: tan(lambda) and q/pT (and their variances) are not
                 * changed by the rotation or the propagation, and each pull
                 * alone bounds the 5-parameter chi2 from below (d_i^2 / S_ii
                 * <= d^T S^-1 d for the SPD sum S): a candidate with either
                 * pull above twice the cut is not evaluated */
                float dtl = top[4] - bot[4], dqp = top[5] - bot[5];
                float lim = 2.0f * P->merge_chi2;
                if (dtl * dtl > lim * (top[6 + 9] + bot[6 + 9]) || dqp * dqp > lim * (top[6 + 14] + bot[6 + 14]))
                    continue;
                float c2 = orc_merge_chi2(top, bot, cs, sn, kb);
                if (!(c2 < P->merge_chi2)) continue;
                int ida = R->trk_start[ta], idb = R->trk_start[tb];
                if (best_next[a] < 0 || c2 < bchi_n[a] ||
                    (c2 == bchi_n[a] && idb < R->trk_start[R->seg_trk[best_next[a]]])) {
                    best_next[a] = b; bchi_n[a] = c2;
                }
                if (best_prev[b] < 0 || c2 < bchi_p[b] ||
                    (c2 == bchi_p[b] && ida < R->trk_start[R->seg_trk[best_prev[b]]])) {
                    best_prev[b] = a; bchi_p[b] = c2;
                }
            }
        }
    }
    for (int a = 0; a < ns; a++) { R->seg_next[a] = -1; R->seg_prev[a] = -1; }
    for (int a = 0; a < ns; a++) {
        int b = best_next[a];
        if (b >= 0 && best_prev[b] == a) { R->seg_next[a] = b; R->seg_prev[b] = a; }
    }
    /* a segment whose inward walk does not end within 36 steps (a closed
     * cycle) is not merged, nor are the links that point to it */
    uint8_t *bad = (uint8_t *)calloc(nz(ns), 1);
    for (int a = 0; a < ns; a++) {
        int c = a, steps = 0;
        while (R->seg_prev[c] >= 0 && steps <= 36) { c = R->seg_prev[c]; steps++; }
        if (R->seg_prev[c] >= 0) bad[a] = 1;
    }
    int32_t *nx2 = (int32_t *)malloc(sizeof(int32_t) * nz(ns));
    int32_t *pv2 = (int32_t *)malloc(sizeof(int32_t) * nz(ns));
    for (int a = 0; a < ns; a++) {
        nx2[a] = R->seg_next[a]; pv2[a] = R->seg_prev[a];
        if (bad[a]) { nx2[a] = -1; pv2[a] = -1; continue; }
        if (nx2[a] >= 0 && bad[nx2[a]]) nx2[a] = -1;
        if (pv2[a] >= 0 && bad[pv2[a]]) pv2[a] = -1;
    }
    memcpy(R->seg_next, nx2, sizeof(int32_t) * nz(ns));
    memcpy(R->seg_prev, pv2, sizeof(int32_t) * nz(ns));
    free(nx2); free(pv2);
    free(bad); free(best_next); free(best_prev); free(bchi_n); free(bchi_p); free(sstart); free(sidx);

    /* ---- merged tracks: chains from their innermost segment (no prev), in
     * ascending start index of that segment; clusters inner -> outer */
    int T = 0;
    for (int a = 0; a < ns; a++) T += R->seg_prev[a] < 0;
    R->n_tracks = T;
    R->tr_sector = (int32_t *)malloc(sizeof(int32_t) * nz(T));
    R->tr_x = (double *)malloc(sizeof(double) * nz(T));
    R->tr_p = (double *)malloc(sizeof(double) * 5 * nz(T));
    R->tr_c = (double *)malloc(sizeof(double) * 15 * nz(T));
    R->tr_chi2 = (double *)malloc(sizeof(double) * nz(T));
    R->tr_ndf = (int32_t *)malloc(sizeof(int32_t) * nz(T));
    R->tr_status = (int32_t *)malloc(sizeof(int32_t) * nz(T));
    R->tr_nclus = (int32_t *)malloc(sizeof(int32_t) * nz(T));
    R->tr_off = (int32_t *)malloc(sizeof(int32_t) * (size_t)(T + 1));
    ivec cl = {0, 0, NULL};
    R->assign = (int32_t *)malloc(sizeof(int32_t) * nz(n));
    for (int i = 0; i < n; i++) R->assign[i] = -1;
    R->tr_off[0] = 0;
    int tr = 0;
    int cap = 64;
    int32_t *csec = (int32_t *)malloc(sizeof(int32_t) * (size_t)cap);
    double *cx = (double *)malloc(sizeof(double) * (size_t)cap);
    double *cy = (double *)malloc(sizeof(double) * (size_t)cap);
    double *cz = (double *)malloc(sizeof(double) * (size_t)cap);
    for (int a = 0; a < ns; a++) {
        if (R->seg_prev[a] >= 0) continue;
        int first = cl.n;
        int tail = a;
        for (int b = a; b >= 0; b = R->seg_next[b]) {
            int tq = R->seg_trk[b];
            uint64_t w = tracklet_weight(R->trk_nhits[tq], R->trk_start[tq]);
            for (int k = R->trk_off[tq]; k < R->trk_off[tq + 1]; k++) {
                int c = R->trk_hits[k];
                if (hitw[c] == w && !R->rejected[c]) iv_push(&cl, c);
            }
            tail = b;
        }
        int nc = cl.n - first;
        if (nc > cap) {
            cap = nc;
            csec = (int32_t *)realloc(csec, sizeof(int32_t) * (size_t)cap);
            cx = (double *)realloc(cx, sizeof(double) * (size_t)cap);
            cy = (double *)realloc(cy, sizeof(double) * (size_t)cap);
            cz = (double *)realloc(cz, sizeof(double) * (size_t)cap);
        }
        for (int k = 0; k < nc; k++) {
            int c = cl.v[first + k];
            csec[k] = sector[c];
            cx[k] = (double)X[row[c]];
            cy[k] = (double)y[c];
            cz[k] = (double)R->z[c];
            R->assign[c] = tr;
        }
        /* ---- a9: refit, starting from the outer end state of the outermost segment */
        double st[NST];
        const float *top = R->trk_top + (size_t)R->seg_trk[tail] * NST;
        for (int k = 0; k < NST; k++) st[k] = (double)top[k];
        double chi2 = 0;
        int okf = orc_fit64(P, G, (double)kb, nc, csec, cx, cy, cz, P->refit_passes, st, &chi2);
        R->tr_sector[tr] = csec[0];
        R->tr_x[tr] = st[0];
        for (int k = 0; k < 5; k++) R->tr_p[5 * tr + k] = st[1 + k];
        for (int k = 0; k < 15; k++) R->tr_c[15 * tr + k] = st[6 + k];
        R->tr_chi2[tr] = chi2;
        R->tr_ndf[tr] = 2 * nc - 5;
        R->tr_status[tr] = okf ? 0 : 1;
        R->tr_nclus[tr] = nc;
        R->tr_off[tr + 1] = cl.n;
        tr++;
    }
    free(csec); free(cx); free(cy); free(cz);
    R->tr_clus = cl.v ? cl.v : (int32_t *)malloc(sizeof(int32_t));
    free(hitw);
    free(pl); free(g.ord); free(g.pstart); free(g.zs);
    return 0;
}

void orc_free(orc_result *R)
{
    free(R->z); free(R->up_raw); free(R->dn_raw); free(R->up); free(R->dn); free(R->is_start);
    free(R->trk_start); free(R->trk_nhits); free(R->trk_off); free(R->trk_hits); free(R->trk_kept);
    free(R->trk_top); free(R->trk_bot);
    free(R->seg_trk); free(R->seg_next); free(R->seg_prev);
    free(R->tr_sector); free(R->tr_x); free(R->tr_p); free(R->tr_c); free(R->tr_chi2); free(R->tr_ndf);
    free(R->tr_status); free(R->tr_nclus); free(R->tr_off); free(R->tr_clus); free(R->assign); free(R->rejected);
    memset(R, 0, sizeof(*R));
}
