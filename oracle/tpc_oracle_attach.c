/*
 * tpc_oracle_attach.c -- plain CPU oracle of the track-based cluster
 * attachment and rejection (paper, section "TPC Data Compression", the
 * cluster rejection step and the figure of attachment categories).
 *
 * TEST INFRASTRUCTURE ONLY: loaded by tests/ and the benchmark's CPU
 * baseline leg, never by the product path.  Shares no code with the CUDA
 * tracker.
 *
 * What the paper fixes: the tracker forms a tube of 1.5 cm around each track;
 * a cluster attached to no track is marked adjacent to the track of highest
 * transverse momentum whose tube contains it; clusters in the tube of a good
 * track (one used for physics) are protected; attached or adjacent clusters
 * that are not protected are removed.  Tracks below 50 MeV/c are not used for
 * physics.  Readings of what it leaves open (each also listed with the
 * design notes):
 *   - the tube follows a track's fitted trajectory: for every sector piece
 *     (segment) of the track, its inner-end state of the TrackletConstructor
 *     (the binary32 Kalman state at its innermost hit, after all of its hits)
 *     is propagated row by row, up to the piece's highest hit row and down to
 *     its lowest, stopping at the first refused step (|sin phi| or the arc
 *     series out of range);
 *   - a cluster lies in the tube when, on a traced row of the piece's sector,
 *     dy^2 + dz^2 < R^2 with (dy, dz) its offset from the traced point
 *     (binary32, fused multiply-add for dy*dy + dz*dz);
 *   - a track's pT, for the adjacency order and the 50 MeV/c cut, is that of
 *     the inner-end state of its innermost piece: |q/pT| of that state, a
 *     track being good when |q/pT| <= 1 / pt_min (binary32); among the tracks
 *     whose tube holds a cluster the one with the smallest |q/pT| wins, ties
 *     to the smaller track index;
 *   - the clusters attached to a good track are protected (they are used for
 *     physics) as well as the clusters in its tube.
 *   - a secondary leg of a looper (tr_leg >= 1: a later leg of a particle
 *     below 200 MeV/c, tpc_oracle_loopers.c) is not a good track: its
 *     clusters are removed unless a good track protects them (the paper's
 *     category of secondary legs of low-pT loopers).
 * The remaining categories of the paper (high-inclination segments left out
 * of the fit, noise and broken pads) need cluster shapes and pad data that the
 * inputs do not carry.
 *
 * Pins (tests/test_oracle_attach.py): the traced points against the closed-
 * form helix in binary64, the tube membership and the adjacency against a
 * brute-force search with that closed form (away from the tube boundary), the
 * flag invariants, and the special cases R = 0, pt_min = 0 and pt_min = inf.
 *
 * Build: as tpc_oracle.c (-ffp-contract=off: every float expression is one
 * correctly rounded binary32 operation).
 */
#include "tpc_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define A_SNP_MAX 0.999f
#define A_U_MAX   0.1f
#define A_AS1 0.16666666666666666667f
#define A_AS2 0.075f
#define A_AS3 0.044642857142857142857f
#define A_KB_C (-2.99792458e-3f)
#define A_NST 21

/* One helix step of the position (x, y, z, sin phi; tan lambda and q/pT are
 * constant) to the plane x2: sin(phi) is linear in x with slope k = kb q/pT;
 * dy = dx (s1 + s2) / (c1 + c2) is exact for the circle; the arc length is the
 * signed chord times asin(u)/u, u = k chord / 2, by its series to u^6 (valid
 * for |u| <= 0.1); dz = tan(lambda) times the arc.  Returns 0 (state left
 * as it was) when |sin phi| would reach 0.999 or |u| > 0.1. */
int orc_step_pos32(float *p, float x2, float kb)
{
    /* p: x, y, z, sin(phi), tan(lambda), q/pT */
    float dx = x2 - p[0];
    if (dx == 0.0f) return 1;
    float k = kb * p[5];
    float s1 = p[3];
    float s2 = fmaf(k, dx, s1);
    if (!(fabsf(s1) < A_SNP_MAX) || !(fabsf(s2) < A_SNP_MAX)) return 0;
    float c1 = sqrtf((1.0f - s1) * (1.0f + s1));
    float c2 = sqrtf((1.0f - s2) * (1.0f + s2));
    float dy = dx * ((s1 + s2) / (c1 + c2));
    float chord = sqrtf(fmaf(dx, dx, dy * dy));
    if (dx < 0.0f) chord = -chord;
    float u = (0.5f * k) * chord;
    if (!(fabsf(u) <= A_U_MAX)) return 0;
    float u2 = u * u;
    float arc = chord * fmaf(u2, fmaf(u2, fmaf(u2, A_AS3, A_AS2), A_AS1), 1.0f);
    p[0] = x2;
    p[1] = p[1] + dy;
    p[2] = p[2] + arc * p[4];
    p[3] = s2;
    return 1;
}

/* ------------------------------------------------------------ plane index */
typedef struct {
    int32_t *ord;     /* cluster indices sorted by (plane, z, index) */
    int32_t *pstart;  /* [planes + 1] */
    float *zs;        /* z in that order */
} plane_index;

static const int32_t *s_pl;
static const float *s_z;
static int cmp_pz(const void *a, const void *b)
{
    int32_t i = *(const int32_t *)a, j = *(const int32_t *)b;
    if (s_pl[i] != s_pl[j]) return s_pl[i] < s_pl[j] ? -1 : 1;
    if (s_z[i] != s_z[j]) return s_z[i] < s_z[j] ? -1 : 1;
    return (i > j) - (i < j);
}

static int first_at_or_above(const plane_index *X, int pl, double zlo)
{
    int lo = X->pstart[pl], hi = X->pstart[pl + 1];
    while (lo < hi) {
        int mid = (lo + hi) / 2;
        if ((double)X->zs[mid] < zlo) lo = mid + 1; else hi = mid;
    }
    return lo;
}

/* the clusters of plane pl in the tube disc around (yp, zp) */
typedef struct {
    const plane_index *X;
    const float *y, *z;
    const int32_t *assign;
    uint64_t *key;       /* [n] best adjacency key so far (0: none) */
    uint8_t *prot;       /* [n] in the tube of a good track */
    float R, R2;
} tube_ctx;

static void visit(const tube_ctx *T, int pl, float yp, float zp, uint64_t key, int good)
{
    const plane_index *X = T->X;
    int end = X->pstart[pl + 1];
    for (int q = first_at_or_above(X, pl, (double)zp - (double)T->R - 1.0); q < end; q++) {
        if ((double)X->zs[q] > (double)zp + (double)T->R + 1.0) break;
        int c = X->ord[q];
        float dy = T->y[c] - yp;
        float dz = T->z[c] - zp;
        if (!(fabsf(dy) <= T->R) || !(fabsf(dz) <= T->R)) continue;
        float d2 = fmaf(dy, dy, dz * dz);
        if (!(d2 < T->R2)) continue;
        if (good) T->prot[c] = 1;
        if (T->assign[c] < 0 && key > T->key[c]) T->key[c] = key;
    }
}

static uint32_t fbits(float f)
{
    uint32_t u;
    memcpy(&u, &f, 4);
    return u;
}

int orc_attach(const orc_geom *G, float bz, int32_t n, const uint8_t *sector, const uint8_t *row,
               const float *y, const float *z, int32_t n_seg, const int32_t *seg_trk,
               const int32_t *seg_next, const int32_t *seg_prev, const int32_t *trk_off,
               const int32_t *trk_hits, const float *trk_bot, const int32_t *assign, float radius,
               float pt_min, const int32_t *tr_leg, int32_t *adjacent, uint8_t *flags)
{
    const int NR = G->n_rows, NP = G->n_sectors * G->n_rows;
    const float *Xr = G->row_x;
    const float kb = A_KB_C * bz;
    const float qmax = pt_min > 0.0f ? 1.0f / pt_min : INFINITY;
    if (n < 0 || n_seg < 0 || !(radius >= 0.0f)) return -1;

    /* tracks: chains of segments from their innermost one, numbered in
     * ascending index of that segment (the tracker's track order) */
    int32_t *seg_track = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n_seg > 0 ? n_seg : 1));
    int32_t *seg_head = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n_seg > 0 ? n_seg : 1));
    for (int a = 0; a < n_seg; a++) seg_track[a] = -1;
    int n_tracks = 0;
    for (int a = 0; a < n_seg; a++) {
        if (seg_prev[a] >= 0) continue;
        for (int b = a; b >= 0; b = seg_next[b]) { seg_track[b] = n_tracks; seg_head[b] = a; }
        n_tracks++;
    }
    /* pT of each track: |q/pT| of its innermost piece's inner-end state */
    float *tr_aq = (float *)malloc(sizeof(float) * (size_t)(n_tracks > 0 ? n_tracks : 1));
    uint8_t *tr_good = (uint8_t *)malloc((size_t)(n_tracks > 0 ? n_tracks : 1));
    for (int a = 0; a < n_seg; a++)
        if (seg_prev[a] < 0) tr_aq[seg_track[a]] = fabsf(trk_bot[(size_t)seg_trk[a] * A_NST + 5]);
    for (int t = 0; t < n_tracks; t++) tr_good[t] = tr_aq[t] <= qmax && !(tr_leg && tr_leg[t] >= 1);

    /* clusters of each (sector, row) plane sorted by z */
    plane_index X;
    int32_t *pl = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    for (int i = 0; i < n; i++) pl[i] = sector[i] * NR + row[i];
    X.ord = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    for (int i = 0; i < n; i++) X.ord[i] = i;
    s_pl = pl; s_z = z;
    qsort(X.ord, (size_t)n, sizeof(int32_t), cmp_pz);
    X.pstart = (int32_t *)calloc((size_t)NP + 1, sizeof(int32_t));
    for (int i = 0; i < n; i++) X.pstart[pl[i] + 1]++;
    for (int p = 0; p < NP; p++) X.pstart[p + 1] += X.pstart[p];
    X.zs = (float *)malloc(sizeof(float) * (size_t)(n > 0 ? n : 1));
    for (int q = 0; q < n; q++) X.zs[q] = z[X.ord[q]];

    tube_ctx T;
    T.X = &X; T.y = y; T.z = z; T.assign = assign; T.R = radius; T.R2 = radius * radius;
    T.key = (uint64_t *)calloc((size_t)(n > 0 ? n : 1), sizeof(uint64_t));
    T.prot = (uint8_t *)calloc((size_t)(n > 0 ? n : 1), 1);

    /* the tube of every piece */
    for (int a = 0; a < n_seg; a++) {
        int tr = seg_track[a];
        if (tr < 0) continue;
        int t = seg_trk[a];
        const int32_t *hits = trk_hits + trk_off[t];
        int nh = trk_off[t + 1] - trk_off[t];
        if (nh <= 0) continue;
        int s = sector[hits[0]];
        int r_lo = row[hits[0]], r_hi = row[hits[nh - 1]];   /* hits ascend in row */
        float aq = tr_aq[tr];
        int good = tr_good[tr];
        uint64_t key = ((uint64_t)(0xFFFFFFFFu - fbits(aq)) << 32) | (uint64_t)(0xFFFFFFFFu - (uint32_t)tr);
        const float *b = trk_bot + (size_t)t * A_NST;
        /* the row of the inner-end state */
        int r_b = -1;
        for (int r = 0; r < NR; r++)
            if (Xr[r] == b[0]) { r_b = r; break; }
        if (r_b < 0) continue;
        if (r_b >= r_lo && r_b <= r_hi) visit(&T, s * NR + r_b, b[1], b[2], key, good);
        float p[6];
        memcpy(p, b, sizeof(p));
        for (int r = r_b + 1; r <= r_hi; r++) {
            if (!orc_step_pos32(p, Xr[r], kb)) break;
            if (r >= r_lo) visit(&T, s * NR + r, p[1], p[2], key, good);
        }
        memcpy(p, b, sizeof(p));
        for (int r = r_b - 1; r >= r_lo; r--) {
            if (!orc_step_pos32(p, Xr[r], kb)) break;
            if (r <= r_hi) visit(&T, s * NR + r, p[1], p[2], key, good);
        }
    }

    /* categories */
    for (int c = 0; c < n; c++) {
        int att = assign[c] >= 0;
        int adj = !att && T.key[c] != 0;
        int prot = T.prot[c] || (att && tr_good[assign[c]]);
        int rem = (att || adj) && !prot;
        flags[c] = (uint8_t)(att | (adj << 1) | (prot << 2) | (rem << 3));
        adjacent[c] = adj ? (int32_t)(0xFFFFFFFFu - (uint32_t)(T.key[c] & 0xFFFFFFFFu)) : -1;
    }
    free(T.key); free(T.prot);
    free(X.ord); free(X.pstart); free(X.zs); free(pl);
    free(tr_aq); free(tr_good); free(seg_track); free(seg_head);
    return 0;
}
