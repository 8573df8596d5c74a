// tpc_dev.cuh -- device-side building blocks of the B300 TPC tracker.
//
// Binary32 Kalman mathematics of the decision path (tracklet following and
// merging, paper section "TPC Tracking"): helix propagation between pad-row
// planes in a uniform Bz, rotation into a neighbouring sector frame, Kalman
// update with a chi2 gate, and the 5-parameter matching chi2.  Every
// expression is one IEEE binary32 operation in a fixed order; fused
// multiply-adds are written explicitly (__fmaf_rn) and the translation units
// that include this header are compiled with -fmad=false, so the results are
// bit-identical to any other IEEE implementation of the same operation order.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace tpc {

constexpr int NST = 21;                // x, p[5], c[15]
constexpr int ROWTAB = 6;              // per-row table: X, q_up, q_dn, w, y-bin origin, 1/y-bin width
constexpr float SNP_MAX = 0.999f;
constexpr float U_MAX = 0.1f;
// asin(u)/u = 1 + u^2/6 + 3u^4/40 + 5u^6/112 + ..., and d/du of it
constexpr float AS1 = 0.16666666666666666667f;
constexpr float AS2 = 0.075f;
constexpr float AS3 = 0.044642857142857142857f;
constexpr float AD1 = 0.33333333333333333333f;
constexpr float AD2 = 0.3f;
constexpr float AD3 = 0.26785714285714285714f;
constexpr float TAN10 = 0.17632698070846497347f;   // tan(10 deg): sector half-opening
constexpr float SIN20 = 0.34202014332566873304f;   // sector opening 20 deg
constexpr float COS20 = 0.93969262078590838405f;
constexpr float KB_C = -2.99792458e-3f;            // d sin(phi)/dx = KB_C * Bz[T] * q/pT

// packed lower-triangular index of (i, j), i >= j
#define CI(i, j) ((i) * ((i) + 1) / 2 + (j))

__device__ __forceinline__ int cidx(int i, int j) { return i >= j ? CI(i, j) : CI(j, i); }

// F C F^T for F = I + a e0e2 + b e0e4 + c e1e2 + d e1e3 + e e1e4 + f e2e4
__device__ __forceinline__ void cov_transport(float* c, float a, float b, float cc, float d, float e, float f)
{
    float C[5][5], D[5][5];
#pragma unroll
    for (int i = 0; i < 5; i++)
#pragma unroll
        for (int j = 0; j < 5; j++) C[i][j] = c[cidx(i, j)];
#pragma unroll
    for (int j = 0; j < 5; j++) {
        D[0][j] = __fmaf_rn(b, C[4][j], __fmaf_rn(a, C[2][j], C[0][j]));
        D[1][j] = __fmaf_rn(e, C[4][j], __fmaf_rn(d, C[3][j], __fmaf_rn(cc, C[2][j], C[1][j])));
        D[2][j] = __fmaf_rn(f, C[4][j], C[2][j]);
        D[3][j] = C[3][j];
        D[4][j] = C[4][j];
    }
#pragma unroll
    for (int i = 0; i < 5; i++) {
        c[CI(i, 0)] = __fmaf_rn(b, D[i][4], __fmaf_rn(a, D[i][2], D[i][0]));
        if (i >= 1) c[CI(i, 1)] = __fmaf_rn(e, D[i][4], __fmaf_rn(d, D[i][3], __fmaf_rn(cc, D[i][2], D[i][1])));
        if (i >= 2) c[CI(i, 2)] = __fmaf_rn(f, D[i][4], D[i][2]);
        if (i >= 3) c[CI(i, 3)] = D[i][3];
        if (i >= 4) c[CI(i, 4)] = D[i][4];
    }
}

// Propagation to the plane x2 (returns false and leaves the state unchanged
// when |sin phi| would reach SNP_MAX or the arc series leaves |u| <= U_MAX).
// sin(phi) is linear in x; dy = dx (s1 + s2) / (c1 + c2); the transverse arc
// is the signed chord times asin(u)/u with u = k chord / 2.
__device__ __forceinline__ bool prop32(float* st, float x2, float kb)
{
    float* p = st + 1;
    float* c = st + 6;
    const float dx = x2 - st[0];
    if (dx == 0.0f) return true;
    const float k = kb * p[4];
    const float s1 = p[2];
    const float s2 = __fmaf_rn(k, dx, s1);
    if (!(fabsf(s1) < SNP_MAX) || !(fabsf(s2) < SNP_MAX)) return false;
    const float c1 = __fsqrt_rn((1.0f - s1) * (1.0f + s1));
    const float c2 = __fsqrt_rn((1.0f - s2) * (1.0f + s2));
    const float ss = s1 + s2, cc = c1 + c2;
    const float tt = __fdiv_rn(ss, cc);
    const float dy = dx * tt;
    const float dl0 = __fsqrt_rn(__fmaf_rn(dx, dx, dy * dy));
    const float dl = dx < 0.0f ? -dl0 : dl0;
    const float u = (0.5f * k) * dl;
    if (!(fabsf(u) <= U_MAX)) return false;
    const float u2 = u * u;
    const float A = __fmaf_rn(u2, __fmaf_rn(u2, __fmaf_rn(u2, AS3, AS2), AS1), 1.0f);
    const float dS = dl * A;
    const float dz = dS * p[3];
    const float r1 = __fdiv_rn(s1, c1), r2 = __fdiv_rn(s2, c2);
    const float cc2 = cc * cc;
    const float dt_ds = __fdiv_rn(__fmaf_rn(ss, r1 + r2, 2.0f * cc), cc2);
    const float dt_dk = __fdiv_rn(dx * __fmaf_rn(ss, r2, cc), cc2);
    const float dy_ds = dx * dt_ds;
    const float dy_dk = dx * dt_dk;
    const float g = __fdiv_rn(dy, dl);
    const float B = __fdiv_rn(1.0f, __fsqrt_rn((1.0f - u) * (1.0f + u)));
    const float dS_ds = B * (g * dy_ds);
    const float Ap = u * __fmaf_rn(u2, __fmaf_rn(u2, AD3, AD2), AD1);
    const float h2 = ((0.5f * dl) * dl) * Ap;
    const float dS_dk = __fmaf_rn(B, g * dy_dk, h2);
    const float ja = dy_ds;
    const float jb = dy_dk * kb;
    const float jc = p[3] * dS_ds;
    const float jd = dS;
    const float je = (p[3] * dS_dk) * kb;
    const float jf = dx * kb;
    cov_transport(c, ja, jb, jc, jd, je, jf);
    st[0] = x2;
    p[0] = p[0] + dy;
    p[1] = p[1] + dz;
    p[2] = s2;
    return true;
}

// The parameter half of prop32: the same operations in the same order for x,
// y, z and sin(phi) and the same refusals, without the Jacobian and the
// covariance (for passes that only need the track's position).
__device__ __forceinline__ bool prop32_pos(float* st, float x2, float kb)
{
    float* p = st + 1;
    const float dx = x2 - st[0];
    if (dx == 0.0f) return true;
    const float k = kb * p[4];
    const float s1 = p[2];
    const float s2 = __fmaf_rn(k, dx, s1);
    if (!(fabsf(s1) < SNP_MAX) || !(fabsf(s2) < SNP_MAX)) return false;
    const float c1 = __fsqrt_rn((1.0f - s1) * (1.0f + s1));
    const float c2 = __fsqrt_rn((1.0f - s2) * (1.0f + s2));
    const float ss = s1 + s2, cc = c1 + c2;
    const float tt = __fdiv_rn(ss, cc);
    const float dy = dx * tt;
    const float dl0 = __fsqrt_rn(__fmaf_rn(dx, dx, dy * dy));
    const float dl = dx < 0.0f ? -dl0 : dl0;
    const float u = (0.5f * k) * dl;
    if (!(fabsf(u) <= U_MAX)) return false;
    const float u2 = u * u;
    const float A = __fmaf_rn(u2, __fmaf_rn(u2, __fmaf_rn(u2, AS3, AS2), AS1), 1.0f);
    const float dS = dl * A;
    const float dz = dS * p[3];
    st[0] = x2;
    p[0] = p[0] + dy;
    p[1] = p[1] + dz;
    p[2] = s2;
    return true;
}

// Rotation of the local frame by +angle (cs = cos, sn = sin); the state is
// then at x' = x cs + y sn.  First-order Jacobian at fixed x'.
__device__ __forceinline__ bool rot32(float* st, float cs, float sn, float kb)
{
    float* p = st + 1;
    float* c = st + 6;
    const float x = st[0], y = p[0], sp = p[2];
    const float cf = __fsqrt_rn((1.0f - sp) * (1.0f + sp));
    const float spn = __fmaf_rn(sp, cs, -(cf * sn));
    const float cfn = __fmaf_rn(cf, cs, sp * sn);
    if (!(fabsf(spn) < SNP_MAX) || !(cfn > 0.0f)) return false;
    const float xn = __fmaf_rn(x, cs, y * sn);
    const float yn = __fmaf_rn(-x, sn, y * cs);
    const float k = kb * p[4];
    const float J00 = __fdiv_rn(cf, cfn);
    const float J10 = __fdiv_rn(-(sn * p[3]), cfn);
    const float J20 = -(k * sn);
    const float J22 = __fdiv_rn(cfn, cf);
    float C[5][5], D[5][5];
#pragma unroll
    for (int i = 0; i < 5; i++)
#pragma unroll
        for (int j = 0; j < 5; j++) C[i][j] = c[cidx(i, j)];
#pragma unroll
    for (int j = 0; j < 5; j++) {
        D[0][j] = J00 * C[0][j];
        D[1][j] = __fmaf_rn(J10, C[0][j], C[1][j]);
        D[2][j] = __fmaf_rn(J22, C[2][j], J20 * C[0][j]);
        D[3][j] = C[3][j];
        D[4][j] = C[4][j];
    }
#pragma unroll
    for (int i = 0; i < 5; i++) {
        c[CI(i, 0)] = J00 * D[i][0];
        if (i >= 1) c[CI(i, 1)] = __fmaf_rn(J10, D[i][0], D[i][1]);
        if (i >= 2) c[CI(i, 2)] = __fmaf_rn(J22, D[i][2], J20 * D[i][0]);
        if (i >= 3) c[CI(i, 3)] = D[i][3];
        if (i >= 4) c[CI(i, 4)] = D[i][4];
    }
    st[0] = xn;
    p[0] = yn;
    p[2] = spn;
    return true;
}

// Kalman update with (my, mz), V = diag(vy, vz), H = [I2 0].  Rejected
// (state untouched, false) when the predicted chi2 exceeds chi2max.
__device__ __forceinline__ bool update32(float* st, float my, float mz, float vy, float vz, float chi2max)
{
    float* p = st + 1;
    float* c = st + 6;
    const float r0 = my - p[0], r1 = mz - p[1];
    const float s00 = c[0] + vy, s01 = c[1], s11 = c[2] + vz;
    const float det = __fmaf_rn(s00, s11, -(s01 * s01));
    if (!(det > 0.0f)) return false;
    const float idet = __fdiv_rn(1.0f, det);
    const float i00 = s11 * idet, i01 = -(s01 * idet), i11 = s00 * idet;
    const float a0 = __fmaf_rn(i00, r0, i01 * r1);
    const float a1 = __fmaf_rn(i01, r0, i11 * r1);
    const float chi2 = __fmaf_rn(r0, a0, r1 * a1);
    if (!(chi2 <= chi2max)) return false;
    float K0[5], K1[5], row0[5], row1[5];
#pragma unroll
    for (int i = 0; i < 5; i++) {
        const float c0 = c[cidx(i, 0)], c1 = c[cidx(i, 1)];
        K0[i] = __fmaf_rn(c0, i00, c1 * i01);
        K1[i] = __fmaf_rn(c0, i01, c1 * i11);
        row0[i] = c0;
        row1[i] = c1;
    }
#pragma unroll
    for (int i = 0; i < 5; i++) p[i] = p[i] + __fmaf_rn(K0[i], r0, K1[i] * r1);
#pragma unroll
    for (int i = 0; i < 5; i++)
#pragma unroll
        for (int j = 0; j <= i; j++) c[CI(i, j)] = c[CI(i, j)] - __fmaf_rn(K0[i], row0[j], K1[i] * row1[j]);
    return true;
}

// chi2 between the outer-end state of piece A and the inner-end state of
// piece B in the neighbouring sector (A rotated into B's frame, propagated to
// B's x); Cholesky of C_A + C_B; +inf when the transport fails.
__device__ __forceinline__ float merge_chi2(const float* top, const float* bot, float cs, float sn, float kb)
{
    float t[NST];
#pragma unroll
    for (int i = 0; i < NST; i++) t[i] = top[i];
    if (!rot32(t, cs, sn, kb)) return __int_as_float(0x7f800000);
    if (!prop32(t, bot[0], kb)) return __int_as_float(0x7f800000);
    float d[5], S[15], L[15], v[5];
#pragma unroll
    for (int i = 0; i < 5; i++) d[i] = t[1 + i] - bot[1 + i];
#pragma unroll
    for (int i = 0; i < 15; i++) S[i] = t[6 + i] + bot[6 + i];
#pragma unroll
    for (int i = 0; i < 5; i++) {
#pragma unroll
        for (int j = 0; j <= i; j++) {
            float s = S[CI(i, j)];
#pragma unroll
            for (int k = 0; k < j; k++) s = __fmaf_rn(-L[CI(i, k)], L[CI(j, k)], s);
            if (i == j) {
                if (!(s > 0.0f)) return __int_as_float(0x7f800000);
                L[CI(i, i)] = __fsqrt_rn(s);
            } else {
                L[CI(i, j)] = __fdiv_rn(s, L[CI(j, j)]);
            }
        }
    }
    float chi2 = 0.0f;
#pragma unroll
    for (int i = 0; i < 5; i++) {
        float s = d[i];
#pragma unroll
        for (int k = 0; k < i; k++) s = __fmaf_rn(-L[CI(i, k)], v[k], s);
        v[i] = __fdiv_rn(s, L[CI(i, i)]);
        chi2 = __fmaf_rn(v[i], v[i], chi2);
    }
    return chi2;
}

// ---------------------------------------------------------------------------
// shared layout of the per-call device state
// ---------------------------------------------------------------------------
// The counters that a stage bumps with many atomics (the tracklet queues, the
// merger's pair count, the start-hit and segment counts) each sit on a
// 128-byte line of their own: kernels read the grid fields and the error flag
// of the first line all the time, and a line under a stream of atomics queues
// those reads at its L2 slice.
struct Frame {
    unsigned zmin_key, zmax_key;   // order-preserving keys of the folded-z extrema, all frames
    float mzmin, minv_cs;          // merger grid (all frames)
    int mnz;
    int ny;                        // grid y-bins per z-cell
    unsigned total_cells;          // grid cells of all frames
    int err;                       // TPC_ERR_* set by kernels (0 = ok)
    int n_tracks, n_clus;
    int n_bad;                     // clusters rejected by validation
    int n_rejected;                // clusters rejected before the refit
    int n_loop_err;                // looper legs: a bounded union-find walk gave up (never expected)
    alignas(128) int n_starts;
    alignas(128) int n_seg;
    alignas(128) int trk_next;     // work queue heads of the tracklet constructor's two passes
    alignas(128) int trk_next2;
    alignas(128) int n_mpairs;     // merger: candidate pairs that passed the screen
    // work counters (params.profile): tracklet propagations, updates, window
    // candidates examined; refit propagations; merger chi2 evaluations
    alignas(128) unsigned long long w_prop;
    unsigned long long w_upd, w_cand, w_refit_prop, w_merge;
};

// per time frame: grid of that frame's clusters
struct FrameGrid {
    unsigned zmin_key, zmax_key;   // folded-z extrema of the frame
    float zmin, inv_cs;            // grid origin and 1 / z-cell length
    int nz;                        // z-cells per plane
    unsigned cell_base;            // first cell of this frame
};

// order-preserving float <-> uint32 key
__device__ __forceinline__ unsigned fkey(float f)
{
    unsigned u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float fkey_inv(unsigned k)
{
    unsigned u = (k & 0x80000000u) ? (k & 0x7fffffffu) : ~k;
    return __uint_as_float(u);
}

__device__ __forceinline__ int grid_cell(float zeta, float zmin, float inv_cs, int nz)
{
    float t = (zeta - zmin) * inv_cs;
    t = fminf(fmaxf(t, 0.0f), (float)(nz - 1));   // NaN -> 0
    return (int)t;
}

__host__ __device__ __forceinline__ uint64_t tracklet_weight(int nhits, int start_id)
{
    return ((uint64_t)(uint32_t)nhits << 32) | (uint64_t)(0xFFFFFFFFu - (uint32_t)start_id);
}

// merge partner sector of s: dir +1 / -1 the next / previous wedge of the same
// side, dir 0 the same wedge across the central membrane
__device__ __forceinline__ int neighbour_sector(int s, int dir, int n_sectors)
{
    if (n_sectors != 36) return -1;
    const int side = s / 18, w = s - side * 18;
    if (dir == 0) return (1 - side) * 18 + w;
    return side * 18 + (w + (dir > 0 ? 1 : 17)) % 18;
}

}  // namespace tpc
