/*
 * helix.c -- exact crossings of helices from the origin with the pad-row
 * planes (input generation only; no tracker arithmetic).
 *
 * A track turns with sense h (+1 counter-clockwise) on a circle of radius R
 * through the origin, starting in direction phi0; after transverse path s
 * its direction is phi0 + h s / R.  The plane x_local = X of a wedge with
 * centre azimuth alpha is crossed where
 *     sin(phi - alpha) = sin(phi0 - alpha) + h X / R,
 * at the local position y = h R (cos(phi0 - alpha) - cos(phi - alpha)) and
 * z = s tan(lambda).  Crossings outside the wedge (|y| > X tan(half opening))
 * or beyond the track's end s_max are dropped; loopers repeat every turn.
 * Output order: by track, row, wedge, branch, turn (deterministic).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>

static int64_t one_track(double R, double h, double phi0, double tgl, double smax, int looper, int nw,
                         const double *alpha, int nr, const double *X, double tan_half, int max_turns, int32_t trk,
                         int32_t *o_trk, int32_t *o_wedge, int32_t *o_row, double *o_y, double *o_z, double *o_snp,
                         double *o_s)
{
    const double two_pi = 2.0 * M_PI, dw = two_pi / 18.0;
    const int nturn = looper ? max_turns : 1;
    int64_t k = 0;
    for (int r = 0; r < nr; r++) {
        const double xr = X[r];
        int wl[18], nwl = 0;
        if (nw == 1 || looper) {
            for (int a = 0; a < nw; a++) wl[nwl++] = a;
        } else {
            double q = xr / (2 * R);
            if (q > 1) q = 1;
            double ang = fmod(phi0 + h * asin(q), two_pi);
            if (ang < 0) ang += two_pi;
            int w0 = ((int)floor(ang / dw)) % 18;
            wl[nwl++] = (w0 + 17) % 18;
            wl[nwl++] = w0;
            wl[nwl++] = (w0 + 1) % 18;
        }
        for (int q = 0; q < nwl; q++) {
            const int a = wl[q];
            const double al = alpha[a];
            const double w = sin(phi0 - al) + h * xr / R;
            if (fabs(w) > 1.0) continue;
            const double asw = asin(w);
            for (int br = 0; br < 2; br++) {
                const double psi = br == 0 ? asw : M_PI - asw;
                const double yl = h * R * (cos(phi0 - al) - cos(psi));
                if (fabs(yl) > xr * tan_half) continue;
                double dphi = fmod(h * (al + psi - phi0), two_pi);
                if (dphi < 0) dphi += two_pi;
                for (int t = 0; t < nturn; t++) {
                    const double s = R * (dphi + two_pi * t);
                    if (s > smax) break;
                    if (o_trk) {
                        o_trk[k] = trk;
                        o_wedge[k] = a;
                        o_row[k] = r;
                        o_y[k] = yl;
                        o_z[k] = s * tgl;
                        o_snp[k] = sin(psi);
                        o_s[k] = s;
                    }
                    k++;
                }
            }
        }
    }
    return k;
}

/* Two calls: with null outputs it returns the total count and fills
 * counts[ntrk]; then with outputs sized by that total it fills them. */
int64_t helix_crossings(int64_t ntrk, const double *R, const double *h, const double *phi0, const double *tgl,
                        const double *smax, const uint8_t *looper, int nw, const double *alpha, int nr,
                        const double *X, double tan_half, int max_turns, int64_t *counts, int32_t *o_trk,
                        int32_t *o_wedge, int32_t *o_row, double *o_y, double *o_z, double *o_snp, double *o_s)
{
    if (!o_trk) {
        int64_t tot = 0;
#pragma omp parallel for schedule(dynamic, 256) reduction(+ : tot)
        for (int64_t i = 0; i < ntrk; i++) {
            counts[i] = one_track(R[i], h[i], phi0[i], tgl[i], smax[i], looper[i], nw, alpha, nr, X, tan_half,
                                  max_turns, (int32_t)i, 0, 0, 0, 0, 0, 0, 0);
            tot += counts[i];
        }
        return tot;
    }
    int64_t *off = (int64_t *)malloc(sizeof(int64_t) * (size_t)(ntrk + 1));
    off[0] = 0;
    for (int64_t i = 0; i < ntrk; i++) off[i + 1] = off[i] + counts[i];
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t i = 0; i < ntrk; i++) {
        const int64_t o = off[i];
        one_track(R[i], h[i], phi0[i], tgl[i], smax[i], looper[i], nw, alpha, nr, X, tan_half, max_turns, (int32_t)i,
                  o_trk + o, o_wedge + o, o_row + o, o_y + o, o_z + o, o_snp + o, o_s + o);
    }
    int64_t tot = off[ntrk];
    free(off);
    return tot;
}
