// tpc_fit.cuh -- Kalman-fit steps of the tolerance path (refit and the
// calibration pass): helix propagation and frame rotation of a binary32
// state with compensated accumulation, returning the non-trivial entries of
// their Jacobians, and the covariance transport through the helix step.
// Included by translation units built with multiply-add contraction allowed;
// the decision path (tpc_dev.cuh) has its own, order-fixed versions.
#pragma once

#include "tpc_dev.cuh"

namespace tpc {
namespace fit {

// d = F c F^T for F = I + a e0e2 + b e0e4 + cc e1e2 + d e1e3 + e e1e4 + f e2e4
template <typename CT>
__device__ __forceinline__ void transport(CT* c, CT a, CT b, CT cc, CT d, CT e, CT f)
{
    CT C[5][5], D[5][5];
#pragma unroll
    for (int i = 0; i < 5; i++)
#pragma unroll
        for (int j = 0; j < 5; j++) C[i][j] = c[cidx(i, j)];
#pragma unroll
    for (int j = 0; j < 5; j++) {
        D[0][j] = C[0][j] + a * C[2][j] + b * C[4][j];
        D[1][j] = C[1][j] + cc * C[2][j] + d * C[3][j] + e * C[4][j];
        D[2][j] = C[2][j] + f * C[4][j];
        D[3][j] = C[3][j];
        D[4][j] = C[4][j];
    }
#pragma unroll
    for (int i = 0; i < 5; i++) {
        c[CI(i, 0)] = D[i][0] + a * D[i][2] + b * D[i][4];
        if (i >= 1) c[CI(i, 1)] = D[i][1] + cc * D[i][2] + d * D[i][3] + e * D[i][4];
        if (i >= 2) c[CI(i, 2)] = D[i][2] + f * D[i][4];
        if (i >= 3) c[CI(i, 3)] = D[i][3];
        if (i >= 4) c[CI(i, 4)] = D[i][4];
    }
}

// A(u) = asin(u)/u and A'(u); the arc length of a chord dl at curvature k is
// dl A(k dl / 2).  Taylor series of asin below |u| = 0.2.
__device__ __forceinline__ void asin_ratio(float u, float& A, float& Ap)
{
    const float u2 = u * u;
    if (fabsf(u) < 0.2f) {
        A = 1.0f + u2 * (1.0f / 6 + u2 * (3.0f / 40 + u2 * (5.0f / 112 + u2 * (35.0f / 1152 + u2 * (63.0f / 2816)))));
        Ap = u * (1.0f / 3 + u2 * (3.0f / 10 + u2 * (15.0f / 56 + u2 * (35.0f / 144 + u2 * (315.0f / 1408)))));
    } else {
        const float as = asinf(u);
        A = as / u;
        Ap = (u * rsqrtf((1.0f - u) * (1.0f + u)) - as) / u2;
    }
}

// Compensated binary32 accumulation of the state: p[i] + pl[i] carries the
// parameter with about twice the binary32 precision.  The sum is Knuth's
// error-free transformation (s + e == a + b exactly); it has no products, so
// multiply-add contraction cannot alter it.
__device__ __forceinline__ void acc(float& hi, float& lo, float d)
{
    const float s = hi + d;
    const float bb = s - hi;
    const float e = (hi - (s - bb)) + (d - bb);
    hi = s;
    lo += e;
}
__device__ __forceinline__ void renorm(float& hi, float& lo)
{
    const float s = hi + lo;
    lo = lo - (s - hi);
    hi = s;
}

// Jacobian of the helix step: F = I + a e0e2 + b e0e4 + c e1e2 + d e1e3 + e e1e4 + f e2e4
struct HelixJac {
    float a, b, c, d, e, f;
};

// Helix step of the state (y, z, sin(phi), tan(lambda), q/pT) from plane x to
// plane x2 in the field constant kb (d sin(phi)/dx per unit q/pT).  False
// (state unchanged) when |sin(phi)| would reach SNP_MAX or the chord exceeds
// the circle; dx == 0 gives the identity.
__device__ __forceinline__ bool helix_step(float& x, float* p, float* pl, float x2, float kb, HelixJac& J)
{
    const float dx = x2 - x;
    if (dx == 0.0f) {
        J.a = J.b = J.c = J.d = J.e = J.f = 0.0f;
        return true;
    }
    const float k = kb * p[4];
    const float kdx = k * dx;
    const float s1 = p[2], s2 = s1 + kdx;
    if (!(fabsf(s1) < SNP_MAX) || !(fabsf(s2) < SNP_MAX)) return false;
    const float c1 = sqrtf((1.0f - s1) * (1.0f + s1)), c2 = sqrtf((1.0f - s2) * (1.0f + s2));
    const float ss = s1 + s2, cc = c1 + c2;
    const float dy = dx * ss / cc;
    const float dl = copysignf(sqrtf(dx * dx + dy * dy), dx);
    const float u = 0.5f * k * dl;
    if (!(fabsf(u) < 1.0f)) return false;
    float A, Ap;
    asin_ratio(u, A, Ap);
    const float dS = dl * A;
    const float r1 = s1 / c1, r2 = s2 / c2;
    const float icc2 = 1.0f / (cc * cc);
    const float dy_ds = dx * (2.0f * cc + ss * (r1 + r2)) * icc2;
    const float dy_dk = dx * dx * (cc + ss * r2) * icc2;
    const float g = dy / dl;
    const float B = rsqrtf((1.0f - u) * (1.0f + u));
    const float dS_ds = B * g * dy_ds;
    const float dS_dk = B * g * dy_dk + 0.5f * dl * dl * Ap;
    J.a = dy_ds;
    J.b = dy_dk * kb;
    J.c = p[3] * dS_ds;
    J.d = dS;
    J.e = p[3] * dS_dk * kb;
    J.f = dx * kb;
    x = x2;
    acc(p[0], pl[0], dy);
    acc(p[1], pl[1], dS * p[3]);
    acc(p[2], pl[2], kdx);
#pragma unroll
    for (int i = 0; i < 3; i++) renorm(p[i], pl[i]);
    return true;
}

// Jacobian of the frame rotation: rows 0..2 are j00 e0, e1 + j10 e0,
// j22 e2 + j20 e0; rows 3, 4 are the identity
struct RotJac {
    float j00, j10, j20, j22;
};

// Rotation of the local frame by the angle (cs, sn) at fixed position.
__device__ __forceinline__ bool rotate_step(float& x, float* p, float* pl, float cs, float sn, float kb, RotJac& J)
{
    const float sp = p[2];
    const float cf = sqrtf((1.0f - sp) * (1.0f + sp));
    const float spn = sp * cs - cf * sn;
    const float cfn = cf * cs + sp * sn;
    if (!(fabsf(spn) < SNP_MAX) || !(cfn > 0.0f)) return false;
    const float k = kb * p[4];
    J.j00 = cf / cfn;
    J.j10 = -sn * p[3] / cfn;
    J.j20 = -k * sn;
    J.j22 = cfn / cf;
    const float xn = x * cs + p[0] * sn;
    const float yn = -x * sn + p[0] * cs;
    pl[0] = pl[0] * cs;
    pl[2] = pl[2] * (cfn / cf);
    x = xn;
    p[0] = yn;
    p[2] = spn;
    renorm(p[0], pl[0]);
    renorm(p[2], pl[2]);
    return true;
}

// c = J c J^T for the rotation Jacobian J
template <typename CT>
__device__ __forceinline__ void rotate_cov(CT* c, const RotJac& R)
{
    const CT J00 = R.j00, J10 = R.j10, J20 = R.j20, J22 = R.j22;
    CT C[5][5], D[5][5];
#pragma unroll
    for (int i = 0; i < 5; i++)
#pragma unroll
        for (int j = 0; j < 5; j++) C[i][j] = c[cidx(i, j)];
#pragma unroll
    for (int j = 0; j < 5; j++) {
        D[0][j] = J00 * C[0][j];
        D[1][j] = C[1][j] + J10 * C[0][j];
        D[2][j] = J22 * C[2][j] + J20 * C[0][j];
        D[3][j] = C[3][j];
        D[4][j] = C[4][j];
    }
#pragma unroll
    for (int i = 0; i < 5; i++) {
        c[CI(i, 0)] = J00 * D[i][0];
        if (i >= 1) c[CI(i, 1)] = D[i][1] + J10 * D[i][0];
        if (i >= 2) c[CI(i, 2)] = J22 * D[i][2] + J20 * D[i][0];
        if (i >= 3) c[CI(i, 3)] = D[i][3];
        if (i >= 4) c[CI(i, 4)] = D[i][4];
    }
}

__device__ __forceinline__ float sector_alpha_deg(int s, int ns) { return ns == 1 ? 10.0f : (float)((s % 18) * 20 + 10); }

// cos / sin of the rotation from sector s_from's frame to sector s_to's
__device__ __forceinline__ void frame_rotation(int s_from, int s_to, int ns, float& cs, float& sn)
{
    float da = sector_alpha_deg(s_to, ns) - sector_alpha_deg(s_from, ns);
    if (da > 180.0f) da -= 360.0f;
    if (da <= -180.0f) da += 360.0f;
    if (da == 20.0f) {
        cs = COS20;
        sn = SIN20;
    } else if (da == -20.0f) {
        cs = COS20;
        sn = -SIN20;
    } else {
        sincospif(da / 180.0f, &sn, &cs);
    }
}

}  // namespace fit
}  // namespace tpc
