/*
 * tpc_oracle_loopers.c -- oracle of the looper-leg identification.
 *
 * TEST INFRASTRUCTURE ONLY, like tpc_oracle.c: only tests/, the smoke check
 * and the CPU baseline leg of the benchmark may load it.  It shares nothing
 * with the CUDA code.
 *
 * Paper: a low-momentum particle spirals in the magnetic field and leaves
 * several legs in the TPC (section "Introduction"); the cluster rejection of
 * section "TPC Data Compression" removes the secondary legs of loopers below
 * 200 MeV/c.  In continuous read-out every leg of a particle carries the
 * same drift offset of its collision, so in the tracker's coordinates (z
 * from the average drift velocity) the legs lie on one helix.
 *
 * Reading (binary32, fixed operation order; the paper gives no numbers):
 *   - a track is a looper candidate when |q/pT| >= qpt_min of the inner-end
 *     state of its innermost piece (a TrackletConstructor state, identical
 *     on every implementation of the decision path);
 *   - its circle: curvature k = kb q/pT, local centre (x - sinphi/k,
 *     y + cosphi/k), rotated to the global frame with the sector's angle;
 *     radius 1/|k|; its point P = the state's position, rotated likewise;
 *     a = |tan(lambda)| / |k|, the z advance per radian of turning;
 *   - the radius is known to s_R = R sqrt(C_qq) / |q/pT| (the state's own
 *     q/pT variance); a leg with s_R > 5 cm is too short to be grouped;
 *   - candidates i < j of one time frame are legs of one particle when,
 *     with s = sqrt(s_Ri^2 + s_Rj^2),
 *       |R_i - R_j| < 2 s + 1 cm, |C_i - C_j|^2 < (2 s + 2 cm)^2,
 *       | |tl_i| - |tl_j| | < 0.05, |z_j - z_i| <= z_max,
 *     and, with the turning angle dpsi = atan2(cross, dot) of P_i - C_i
 *     and P_j - C_i (counter-clockwise positive), a = (a_i + a_j)/2 and
 *     the sense sigma of the z advance (below):
 *       w = sigma (z_j - z_i) - a dpsi,  m = clamp(rint(w / (2 pi a)), -10, 10),
 *       |w - 2 pi a m| < 3 cm + |tl| (|dpsi| + 2 pi |m|) 2 s;
 *   - the sense: along the motion z advances by tan(lambda) R per radian
 *     the particle turns, and the turning sense is the sign of the
 *     curvature, so z advances by sigma a per radian of counter-clockwise
 *     turning with sigma = sign(k tan(lambda)); the tracker fits an inward
 *     leg in the direction of increasing x, which flips both k and
 *     tan(lambda), so sigma is the same on every leg of a particle.  Two
 *     candidates need the same sigma when both |tan(lambda)| >= 0.02; below
 *     that (z nearly constant along the helix) either sense is tried;
 *     (legs of one helix differ in z by the advance over the turning angle
 *     between them, plus whole turns; a looper makes at most 10 turns, its
 *     legs lie on one side of the drift volume);
 *   - groups are the connected components of that relation; group = the
 *     smallest track index of the component, -1 for a track alone; legs
 *     are numbered in ascending s z (s = +1 on the A side, -1 on the C
 *     side: the earliest leg of the drift is leg 0, the primary), ties by
 *     track index; leg = -1 outside a group.
 *   - atan2 is this file's own: two half-angle reductions
 *     atan(x) = 2 atan(x / (1 + sqrt(1 + x^2))) bring |x| <= 1 below
 *     tan(pi/16), where the Maclaurin series of atan to x^15 is exact in
 *     binary32 (next term < 1e-13).
 */
#include "tpc_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define LOOP_DR 1.0f        /* radius tolerance beyond 2 s (cm) */
#define LOOP_DC 2.0f        /* centre tolerance beyond 2 s (cm) */
#define LOOP_NSIG 2.0f
#define LOOP_SRMAX 5.0f     /* legs with a radius uncertainty above this are not grouped (cm) */
#define LOOP_DTGL 0.05f
#define LOOP_DZ 3.0f
#define LOOP_TLSENSE 0.02f  /* both |tan(lambda)| above this: the z-advance senses must agree */
#define LOOP_TURNS 10.0f
#define PI_F 3.14159265358979323846f
#define TWO_PI_F 6.28318530717958647692f
#define HALF_PI_F 1.57079632679489661923f

/* cos and sin of the sector angles (s mod 18) * 20 + 10 degrees */
static const float SEC_COS[18] = {
    0.98480775301220805936f, 0.86602540378443864676f, 0.64278760968653932632f, 0.34202014332566873304f,
    0.0f, -0.34202014332566873304f, -0.64278760968653932632f, -0.86602540378443864676f,
    -0.98480775301220805936f, -0.98480775301220805936f, -0.86602540378443864676f, -0.64278760968653932632f,
    -0.34202014332566873304f, 0.0f, 0.34202014332566873304f, 0.64278760968653932632f,
    0.86602540378443864676f, 0.98480775301220805936f};
static const float SEC_SIN[18] = {
    0.17364817766693034885f, 0.5f, 0.76604444311897803520f, 0.93969262078590838405f,
    1.0f, 0.93969262078590838405f, 0.76604444311897803520f, 0.5f,
    0.17364817766693034885f, -0.17364817766693034885f, -0.5f, -0.76604444311897803520f,
    -0.93969262078590838405f, -1.0f, -0.93969262078590838405f, -0.76604444311897803520f,
    -0.5f, -0.17364817766693034885f};

/* atan(x) for |x| <= 1 */
static float atan_unit(float x)
{
    float x1 = x / (1.0f + sqrtf(fmaf(x, x, 1.0f)));
    float x2 = x1 / (1.0f + sqrtf(fmaf(x1, x1, 1.0f)));
    float t2 = x2 * x2;
    float p = fmaf(t2, -0.066666666666666666667f, 0.076923076923076923077f);
    p = fmaf(t2, p, -0.090909090909090909091f);
    p = fmaf(t2, p, 0.11111111111111111111f);
    p = fmaf(t2, p, -0.14285714285714285714f);
    p = fmaf(t2, p, 0.2f);
    p = fmaf(t2, p, -0.33333333333333333333f);
    float a = fmaf(x2 * t2, p, x2);
    return 4.0f * a;
}

static float atan2_own(float y, float x)
{
    if (x == 0.0f && y == 0.0f) return 0.0f;
    if (fabsf(y) <= fabsf(x)) {
        float a = atan_unit(y / x);
        if (x < 0.0f) a = y >= 0.0f ? a + PI_F : a - PI_F;
        return a;
    }
    float a = atan_unit(x / y);
    return (y > 0.0f ? HALF_PI_F : -HALF_PI_F) - a;
}

float orc_atan2_own(float y, float x) { return atan2_own(y, x); }

typedef struct {
    int idx;
    float R, sr, cx, cy, px, py, z, tl, a, sz;
    int frame, sense;
} cand_t;

static int find_root(int32_t *par, int i)
{
    while (par[i] != i) {
        par[i] = par[par[i]];
        i = par[i];
    }
    return i;
}

static int cmp_sz(const void *A, const void *B)
{
    const cand_t *a = (const cand_t *)A, *b = (const cand_t *)B;
    if (a->sz != b->sz) return a->sz < b->sz ? -1 : 1;
    return (a->idx > b->idx) - (a->idx < b->idx);
}

int orc_loopers(int32_t n_sectors, float z_max, float bz, float qpt_min, int32_t n_tracks, const int32_t *sector,
                const int32_t *frame, const float *state, int32_t *group, int32_t *leg)
{
    if (n_tracks < 0 || !(qpt_min > 0.0f)) return -1;
    const float kb = -2.99792458e-3f * bz;
    cand_t *c = (cand_t *)malloc(sizeof(cand_t) * (size_t)(n_tracks > 0 ? n_tracks : 1));
    int nc = 0;
    for (int t = 0; t < n_tracks; t++) {
        group[t] = -1;
        leg[t] = -1;
        const float *s = state + 21 * (size_t)t;    /* x, y, z, sinphi, tanlambda, q/pT, cov */
        float q = s[5];
        if (!(fabsf(q) >= qpt_min)) continue;
        float k = kb * q;
        float sp = s[3];
        float cp = sqrtf((1.0f - sp) * (1.0f + sp));
        float ik = 1.0f / k;
        float lx = s[0] - sp * ik, ly = fmaf(cp, ik, s[1]);
        int w = n_sectors == 1 ? 0 : sector[t] % 18;
        float cs = n_sectors == 1 ? SEC_COS[0] : SEC_COS[w], sn = n_sectors == 1 ? SEC_SIN[0] : SEC_SIN[w];
        cand_t *e = &c[nc++];
        e->idx = t;
        e->frame = frame ? frame[t] : 0;
        e->R = fabsf(ik);
        e->sr = e->R * (sqrtf(s[6 + 14]) / fabsf(q));
        if (!(e->sr <= LOOP_SRMAX)) {
            nc--;
            continue;
        }
        e->cx = fmaf(lx, cs, -(ly * sn));
        e->cy = fmaf(lx, sn, ly * cs);
        e->px = fmaf(s[0], cs, -(s[1] * sn));
        e->py = fmaf(s[0], sn, s[1] * cs);
        e->z = s[2];
        e->tl = fabsf(s[4]);
        e->sense = k * s[4] >= 0.0f ? 1 : -1;
        e->a = e->tl * e->R;
        float side = (n_sectors == 36 && sector[t] >= 18) ? -1.0f : 1.0f;
        e->sz = side * s[2];
    }
    int32_t *par = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nc > 0 ? nc : 1));
    for (int i = 0; i < nc; i++) par[i] = i;
    for (int i = 0; i < nc; i++) {
        for (int j = i + 1; j < nc; j++) {
            const cand_t *A = &c[i], *B = &c[j];
            if (A->frame != B->frame) continue;
            float sg2 = sqrtf(fmaf(A->sr, A->sr, B->sr * B->sr));
            float tsg = LOOP_NSIG * sg2;
            if (!(fabsf(A->R - B->R) < tsg + LOOP_DR)) continue;
            float dx = B->cx - A->cx, dy = B->cy - A->cy;
            float dc = tsg + LOOP_DC;
            if (!(fmaf(dx, dx, dy * dy) < dc * dc)) continue;
            if (!(fabsf(A->tl - B->tl) < LOOP_DTGL)) continue;
            if (!(fabsf(B->z - A->z) <= z_max)) continue;
            float ux = A->px - A->cx, uy = A->py - A->cy;
            float vx = B->px - A->cx, vy = B->py - A->cy;
            float cr = fmaf(ux, vy, -(uy * vx));
            float dt = fmaf(ux, vx, uy * vy);
            float dpsi = atan2_own(cr, dt);
            float a = 0.5f * (A->a + B->a);
            float tl = 0.5f * (A->tl + B->tl);
            float tpa = TWO_PI_F * a;
            int steep = A->tl >= LOOP_TLSENSE && B->tl >= LOOP_TLSENSE;
            if (steep && A->sense != B->sense) continue;
            int ok = 0;
            for (int sg = 0; sg < 2 && !ok; sg++) {
                int sense = sg == 0 ? A->sense : -A->sense;
                if (steep && sg == 1) break;
                float dz = B->z - A->z;
                float w = (sense > 0 ? dz : -dz) - a * dpsi;
                float m = tpa > 0.0f ? rintf(w / tpa) : 0.0f;
                m = fminf(fmaxf(m, -LOOP_TURNS), LOOP_TURNS);
                float res = fmaf(-tpa, m, w);
                float turn = fmaf(TWO_PI_F, fabsf(m), fabsf(dpsi));
                float tol = fmaf(tl * turn, tsg, LOOP_DZ);
                ok = fabsf(res) < tol;
            }
            if (!ok) continue;
            int ra = find_root(par, i), rb = find_root(par, j);
            if (ra != rb) par[ra > rb ? ra : rb] = ra < rb ? ra : rb;
        }
    }
    /* groups: the smallest track index of each component with two or more members */
    int32_t *cnt = (int32_t *)calloc((size_t)(nc > 0 ? nc : 1), sizeof(int32_t));
    int32_t *gmin = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nc > 0 ? nc : 1));
    for (int i = 0; i < nc; i++) gmin[i] = -1;
    for (int i = 0; i < nc; i++) {
        int r = find_root(par, i);
        cnt[r]++;
        if (gmin[r] < 0 || c[i].idx < gmin[r]) gmin[r] = c[i].idx;
    }
    /* legs: members of a group in ascending (s z, index) */
    cand_t *tmp = (cand_t *)malloc(sizeof(cand_t) * (size_t)(nc > 0 ? nc : 1));
    for (int i = 0; i < nc; i++) {
        int r = find_root(par, i);
        if (cnt[r] < 2) continue;
        group[c[i].idx] = gmin[r];
    }
    for (int i = 0; i < nc; i++) {
        int r = find_root(par, i);
        if (cnt[r] < 2 || gmin[r] != c[i].idx) continue;     /* once per group, at its smallest member */
        int m = 0;
        for (int j = 0; j < nc; j++)
            if (find_root(par, j) == r) tmp[m++] = c[j];
        qsort(tmp, (size_t)m, sizeof(cand_t), cmp_sz);
        for (int q = 0; q < m; q++) leg[tmp[q].idx] = q;
    }
    free(tmp); free(cnt); free(gmin); free(par); free(c);
    return 0;
}
