// tpc_calib.cu -- calibration chi2 of the refit and its adjoint (the
// gradient with respect to drift velocity, t0 and the per-sector spline
// distortion map).  Paper: section "Tracking" (the collision time fixed by
// matching, the final refit applies the calibration under the primary-track
// assumption) and section "TPC Tracking" (online drift-velocity calibration);
// the model is stated in tpc_calib.h.
//
// One thread per track.  The forward kernel carries the reference helix (the
// tracker's output state) out to the outermost cluster, then runs the inward
// Kalman pass on the deviation from it and stores the pass state every
// TPC_CALIB_CKPT_STEPS steps.  The backward kernel walks the segments from the
// vertex end back: it recomputes one segment from its checkpoint into local
// memory (Jacobian entries, gain, inverse innovation covariance, innovation
// of every step), then sweeps it in reverse with the adjoint recursion
//   a_k = 2 W_k r_k + K_k^T lam_k        (d chi2 / d measurement k)
//   lam_{k-1} = F_k^T (lam_k - H^T a_k)  (d chi2 / d deviation before step k)
// and scatters a_k dm_k/dtheta into the gradient: the spline part through
// block-private binary64 shared-memory sums, v and t0 through per-track
// binary32 sums added to block-private binary64 sums, all flushed once per
// block into binary64 global sums.  Tolerance path: multiply-add
// contraction allowed.
#include "tpc_calib.h"
#include "tpc_dev.cuh"
#include "tpc_fit.cuh"

#include <cmath>
#include <cstring>

using namespace tpc;
using namespace tpc::fit;

namespace {

constexpr int NSPL = TPC_CALIB_NSPL;
constexpr int SEG = TPC_CALIB_CKPT_STEPS;
constexpr int CK_FLOATS = 32;          // x, sector, p[5], pl[5], dp[5], C[15]
constexpr int CALIB_BLOCK = 128;
constexpr int MAX_SPL_SECTORS = 36;
// workspace: a 256-byte header (int32 error flags at offset 0, bit 0: invalid
// track data, bit 1: a recomputed segment failed), then the checkpoints
constexpr size_t HDR_BYTES = 256;
// tracks whose reference reaches |sin(phi)| >= 0.9 at a cluster (nearly
// tangent to the pad rows, an ill-conditioned helix step) are left out
constexpr float SNP_CALIB = 0.9f;

struct CalibArgs {
    int T, ns, nr;
    int64_t ncl;
    float kb, vy, vz, vtx, c0s, c0t, c0q, v_nom, zmax, x_first, inv_dx;
    const int32_t* sector;
    const float* x;
    const float* param;
    const int32_t* off;
    const int32_t* clus;
    const float* tcoll;
    const uint8_t* cs;
    const uint8_t* cr;
    const float* cy;
    const float* ct;
    const float* theta;
    float* chi2;
    uint8_t* used;
    const uint8_t* used_in;
    const float* dchi2;
    double* grad;
    float4* ckpt;
    int32_t* err;
    float rowx[256];
};

// ---- uniform clamped cubic B-spline, 8 coefficients on [0, 1] ----------------
// knots 0,0,0,0, .2,.4,.6,.8, 1,1,1,1; triangular evaluation of the four
// non-zero basis functions of the knot span holding u, derivatives from the
// degree-2 functions.  Returns the index of the first of the four.
__device__ __forceinline__ float knot(int i) { return i <= 3 ? 0.0f : (i >= 8 ? 1.0f : (float)(i - 3) * 0.2f); }

__device__ __forceinline__ int bspline(float u, float* B, float* dB)
{
    u = fminf(fmaxf(u, 0.0f), 1.0f);
    int span = 3;
#pragma unroll
    for (int i = 4; i <= 7; i++)
        if (u >= knot(i)) span = i;
    float N[4], left[4], right[4], N2[3];
    N[0] = 1.0f;
#pragma unroll
    for (int j = 1; j <= 3; j++) {
        left[j] = u - knot(span + 1 - j);
        right[j] = knot(span + j) - u;
        float saved = 0.0f;
#pragma unroll
        for (int r = 0; r < j; r++) {
            const float tmp = N[r] / (right[r + 1] + left[j - r]);
            N[r] = saved + right[r + 1] * tmp;
            saved = left[j - r] * tmp;
        }
        N[j] = saved;
        if (j == 2) {
            N2[0] = N[0];
            N2[1] = N[1];
            N2[2] = N[2];
        }
    }
#pragma unroll
    for (int r = 0; r < 4; r++) {
        const int i = span - 3 + r;
        float d = 0.0f;
        if (r >= 1) {
            const float den = knot(i + 3) - knot(i);
            if (den > 0.0f) d += 3.0f * N2[r - 1] / den;
        }
        if (r <= 2) {
            const float den = knot(i + 4) - knot(i + 1);
            if (den > 0.0f) d -= 3.0f * N2[r] / den;
        }
        B[r] = N[r];
        dB[r] = d;
    }
    return span - 3;
}

// calibrated measurement of cluster c for collision time tc; with grad, the
// derivatives of (m_y, m_z) with respect to v and t0 and the basis values
struct Meas {
    float my, mz;
    float dy_v, dz_v, dy_t0, dz_t0;
    float sgn;
    int s, i0, j0;
    float Bu[4], Bw[4];
};

__device__ __forceinline__ void measure(const CalibArgs& A, const float* __restrict__ spl, int c, float tc, Meas& m)
{
    const int s = A.cs[c];
    const float v = A.theta[0], t0 = A.theta[1];
    const float tau = (A.ct[c] - tc) - t0;
    const float zl = A.zmax - v * tau;
    const float w = zl / A.zmax;
    const float dwdz = (w > 0.0f && w < 1.0f) ? 1.0f / A.zmax : 0.0f;
    float dBu[4], dBw[4];
    m.i0 = bspline((A.rowx[A.cr[c]] - A.x_first) * A.inv_dx, m.Bu, dBu);
    m.j0 = bspline(w, m.Bw, dBw);
    const float* cc = spl + (s * NSPL * NSPL + m.i0 * NSPL + m.j0) * 2;
    float dy = 0.0f, dz = 0.0f, dyw = 0.0f, dzw = 0.0f;
#pragma unroll
    for (int a = 0; a < 4; a++) {
        float ry = 0.0f, rz = 0.0f, ryw = 0.0f, rzw = 0.0f;
#pragma unroll
        for (int b = 0; b < 4; b++) {
            const float cy = cc[(a * NSPL + b) * 2], cz = cc[(a * NSPL + b) * 2 + 1];
            ry += m.Bw[b] * cy;
            rz += m.Bw[b] * cz;
            ryw += dBw[b] * cy;
            rzw += dBw[b] * cz;
        }
        dy += m.Bu[a] * ry;
        dz += m.Bu[a] * rz;
        dyw += m.Bu[a] * ryw;
        dzw += m.Bu[a] * rzw;
    }
    const float sgn = (A.ns == 36 && s >= 18) ? -1.0f : 1.0f;
    m.my = A.cy[c] - dy;
    m.mz = sgn * (zl - dz);
    // zl depends on v through -tau and on t0 through v
    const float ky = -dyw * dwdz, kz = sgn * (1.0f - dzw * dwdz);
    m.dy_v = ky * -tau;
    m.dz_v = kz * -tau;
    m.dy_t0 = ky * v;
    m.dz_t0 = kz * v;
    m.sgn = sgn;
    m.s = s;
}

// pass state: reference (x, sector, p + pl) and deviation (dp, C)
struct PassState {
    float x;
    int sec;
    float p[5], pl[5];
    float dp[5];
    float C[15];
};

// one step's record for the reverse sweep
struct StepRec {
    float j00, j10, j20, j22;      // rotation Jacobian (identity when no rotation)
    HelixJac h;
    float K[10];                   // K[2i + e]
    float W[3];                    // W00, W01, W11
    float r[2];
};

__device__ __forceinline__ bool ref_step(const CalibArgs& A, PassState& S, int s2, float x2, StepRec& R)
{
    R.j00 = 1.0f;
    R.j10 = 0.0f;
    R.j20 = 0.0f;
    R.j22 = 1.0f;
    if (s2 != S.sec) {
        float cs, sn;
        frame_rotation(S.sec, s2, A.ns, cs, sn);
        RotJac J;
        if (!rotate_step(S.x, S.p, S.pl, cs, sn, A.kb, J)) return false;
        R.j00 = J.j00;
        R.j10 = J.j10;
        R.j20 = J.j20;
        R.j22 = J.j22;
        S.sec = s2;
    }
    return helix_step(S.x, S.p, S.pl, x2, A.kb, R.h) && fabsf(S.p[2]) < SNP_CALIB;
}

// step to the primary vertex: rotate the frame about the origin onto the
// reference position (x' = r, y' = 0), then the helix to x = 0, where the
// track crosses at a small angle to the new axis
__device__ __forceinline__ bool vertex_step(const CalibArgs& A, PassState& S, StepRec& R)
{
    const float y = S.p[0] + S.pl[0];
    const float r = sqrtf(S.x * S.x + y * y);
    if (!(r > 0.0f)) return false;
    RotJac J;
    if (!rotate_step(S.x, S.p, S.pl, S.x / r, y / r, A.kb, J)) return false;
    R.j00 = J.j00;
    R.j10 = J.j10;
    R.j20 = J.j20;
    R.j22 = J.j22;
    return helix_step(S.x, S.p, S.pl, 0.0f, A.kb, R.h);
}

// prediction + update of step k >= 1 with measurement (my, mz) of variances
// (vy, vz); the reference has already been moved to the step's plane
__device__ __forceinline__ bool filter_step(PassState& S, StepRec& R, float my, float mz, float vy, float vz,
                                            float& chi2)
{
    // deviation through the rotation, then the helix
    float d0 = R.j00 * S.dp[0];
    float d1 = S.dp[1] + R.j10 * S.dp[0];
    float d2 = R.j22 * S.dp[2] + R.j20 * S.dp[0];
    const float d3 = S.dp[3], d4 = S.dp[4];
    d0 = d0 + R.h.a * d2 + R.h.b * d4;
    d1 = d1 + R.h.c * d2 + R.h.d * d3 + R.h.e * d4;
    d2 = d2 + R.h.f * d4;
    RotJac J{R.j00, R.j10, R.j20, R.j22};
    rotate_cov<float>(S.C, J);
    transport<float>(S.C, R.h.a, R.h.b, R.h.c, R.h.d, R.h.e, R.h.f);
    // innovation against reference + deviation
    const float r0 = ((my - S.p[0]) - S.pl[0]) - d0;
    const float r1 = ((mz - S.p[1]) - S.pl[1]) - d1;
    const float s00 = S.C[0] + vy, s01 = S.C[1], s11 = S.C[2] + vz;
    const float det = s00 * s11 - s01 * s01;
    if (!(det > 0.0f)) return false;
    const float idet = 1.0f / det;
    const float w00 = s11 * idet, w01 = -s01 * idet, w11 = s00 * idet;
    chi2 += r0 * (w00 * r0 + w01 * r1) + r1 * (w01 * r0 + w11 * r1);
    float K0[5], K1[5], c0[5], c1[5];
#pragma unroll
    for (int i = 0; i < 5; i++) {
        c0[i] = S.C[cidx(i, 0)];
        c1[i] = S.C[cidx(i, 1)];
        K0[i] = c0[i] * w00 + c1[i] * w01;
        K1[i] = c0[i] * w01 + c1[i] * w11;
        R.K[2 * i] = K0[i];
        R.K[2 * i + 1] = K1[i];
    }
    R.W[0] = w00;
    R.W[1] = w01;
    R.W[2] = w11;
    R.r[0] = r0;
    R.r[1] = r1;
    S.dp[0] = d0 + K0[0] * r0 + K1[0] * r1;
    S.dp[1] = d1 + K0[1] * r0 + K1[1] * r1;
    S.dp[2] = d2 + K0[2] * r0 + K1[2] * r1;
    S.dp[3] = d3 + K0[3] * r0 + K1[3] * r1;
    S.dp[4] = d4 + K0[4] * r0 + K1[4] * r1;
#pragma unroll
    for (int i = 0; i < 5; i++)
#pragma unroll
        for (int j = 0; j <= i; j++) S.C[CI(i, j)] -= K0[i] * c0[j] + K1[i] * c1[j];
    return true;
}

__device__ __forceinline__ void save_ckpt(float4* dst, const PassState& S)
{
    float v[CK_FLOATS];
    v[0] = S.x;
    v[1] = __int_as_float(S.sec);
#pragma unroll
    for (int i = 0; i < 5; i++) {
        v[2 + i] = S.p[i];
        v[7 + i] = S.pl[i];
        v[12 + i] = S.dp[i];
    }
#pragma unroll
    for (int i = 0; i < 15; i++) v[17 + i] = S.C[i];
#pragma unroll
    for (int q = 0; q < CK_FLOATS / 4; q++) dst[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
}

__device__ __forceinline__ void load_ckpt(const float4* src, PassState& S)
{
    float v[CK_FLOATS];
#pragma unroll
    for (int q = 0; q < CK_FLOATS / 4; q++) {
        const float4 t = src[q];
        v[4 * q] = t.x;
        v[4 * q + 1] = t.y;
        v[4 * q + 2] = t.z;
        v[4 * q + 3] = t.w;
    }
    S.x = v[0];
    S.sec = __float_as_int(v[1]);
#pragma unroll
    for (int i = 0; i < 5; i++) {
        S.p[i] = v[2 + i];
        S.pl[i] = v[7 + i];
        S.dp[i] = v[12 + i];
    }
#pragma unroll
    for (int i = 0; i < 15; i++) S.C[i] = v[17 + i];
}

// checkpoint slot of track r: clus_offset[r] / SEG + r (slots of consecutive
// tracks never overlap: a track of n clusters uses at most n / SEG + 1)
__device__ __forceinline__ int64_t ckpt_base(const CalibArgs& A, int r) { return (int64_t)A.off[r] / SEG + r; }

__device__ __forceinline__ bool track_ok(const CalibArgs& A, int r, int& off, int& n)
{
    off = A.off[r];
    n = A.off[r + 1] - off;
    if (n < 0 || off < 0 || (int64_t)off + n > A.ncl) {
        atomicOr(A.err, 1);
        return false;
    }
    for (int i = 0; i < n; i++) {
        const int c = A.clus[off + i];
        if (c < 0 || (int64_t)c >= A.ncl || A.cs[c] >= A.ns || A.cr[c] >= A.nr) {
            atomicOr(A.err, 1);
            return false;
        }
    }
    const int s0 = A.sector[r];
    if (s0 < 0 || s0 >= A.ns) {
        atomicOr(A.err, 1);
        return false;
    }
    return true;
}

// reference at the outermost cluster (start of the inward pass)
__device__ __forceinline__ bool ref_outward(const CalibArgs& A, int r, int off, int n, float tc, PassState& S)
{
    S.sec = A.sector[r];
    S.x = A.x[r];
#pragma unroll
    for (int k = 0; k < 5; k++) {
        S.p[k] = A.param[5 * (int64_t)r + k];
        S.pl[k] = 0.0f;
    }
    if (!(fabsf(S.p[2]) < SNP_CALIB)) return false;
    // tracker frame -> absolute z, compensated
    acc(S.p[1], S.pl[1], ((A.ns == 36 && S.sec >= 18) ? -A.v_nom : A.v_nom) * tc);
    renorm(S.p[1], S.pl[1]);
    StepRec R;
    for (int i = 1; i < n; i++) {
        const int c = A.clus[off + i];
        if (!ref_step(A, S, A.cs[c], A.rowx[A.cr[c]], R)) return false;
    }
    return true;
}

__device__ __forceinline__ void load_spline(const CalibArgs& A, float* spl)
{
    const int nc = A.ns * NSPL * NSPL * 2;
    for (int i = threadIdx.x; i < nc; i += blockDim.x) spl[i] = A.theta[2 + i];
}

__global__ void __launch_bounds__(CALIB_BLOCK) k_calib_fwd(CalibArgs A)
{
    __shared__ float spl[MAX_SPL_SECTORS * NSPL * NSPL * 2];
    load_spline(A, spl);
    __syncthreads();
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < A.T; r += gridDim.x * blockDim.x) {
        int off, n;
        const float tc = A.tcoll[r];
        float chi2 = 0.0f;
        bool ok = track_ok(A, r, off, n) && n >= 2 && !isnan(tc);
        PassState S;
        if (ok) ok = ref_outward(A, r, off, n, tc, S);
        float4* ck = A.ckpt + ckpt_base(A, r) * (CK_FLOATS / 4);
        if (ok) {
            Meas m;
            measure(A, spl, A.clus[off + n - 1], tc, m);
            S.dp[0] = (m.my - S.p[0]) - S.pl[0];
            S.dp[1] = (m.mz - S.p[1]) - S.pl[1];
            S.dp[2] = S.dp[3] = S.dp[4] = 0.0f;
#pragma unroll
            for (int i = 0; i < 15; i++) S.C[i] = 0.0f;
            S.C[0] = A.vy;
            S.C[2] = A.vz;
            S.C[CI(2, 2)] = A.c0s;
            S.C[CI(3, 3)] = A.c0t;
            S.C[CI(4, 4)] = A.c0q;
            save_ckpt(ck, S);
            StepRec R;
            for (int k = 1; k <= n && ok; k++) {
                float my, mz, vy, vz;
                if (k < n) {
                    const int c = A.clus[off + n - 1 - k];
                    ok = ref_step(A, S, A.cs[c], A.rowx[A.cr[c]], R);
                    if (!ok) break;
                    measure(A, spl, c, tc, m);
                    my = m.my;
                    mz = m.mz;
                    vy = A.vy;
                    vz = A.vz;
                } else {
                    ok = vertex_step(A, S, R);
                    if (!ok) break;
                    my = mz = 0.0f;
                    vy = vz = A.vtx;
                }
                ok = filter_step(S, R, my, mz, vy, vz, chi2);
                if (ok && k % SEG == 0 && k < n) save_ckpt(ck + (k / SEG) * (CK_FLOATS / 4), S);
            }
        }
        A.chi2[r] = ok ? chi2 : 0.0f;
        A.used[r] = ok ? 1 : 0;
    }
}

__device__ __forceinline__ void scatter_grad(const CalibArgs& A, const float* spl, double* gspl, int c, float tc,
                                             float a0, float a1, float& gv, float& gt0)
{
    Meas m;
    measure(A, spl, c, tc, m);
    gv += a0 * m.dy_v + a1 * m.dz_v;
    gt0 += a0 * m.dy_t0 + a1 * m.dz_t0;
    double* g = gspl + (m.s * NSPL * NSPL + m.i0 * NSPL + m.j0) * 2;
    const float ay = -a0, az = -a1 * m.sgn;
#pragma unroll
    for (int i = 0; i < 4; i++)
#pragma unroll
        for (int j = 0; j < 4; j++) {
            const float b = m.Bu[i] * m.Bw[j];
            atomicAdd(&g[(i * NSPL + j) * 2], (double)(ay * b));
            atomicAdd(&g[(i * NSPL + j) * 2 + 1], (double)(az * b));
        }
}

__global__ void __launch_bounds__(CALIB_BLOCK) k_calib_bwd(CalibArgs A)
{
    // dynamic shared memory: binary64 spline-gradient sums, then the spline
    extern __shared__ double smem[];
    __shared__ double gvt[2];
    const int nc = A.ns * NSPL * NSPL * 2;
    double* gspl = smem;
    float* spl = reinterpret_cast<float*>(smem + nc);
    load_spline(A, spl);
    for (int i = threadIdx.x; i < nc; i += blockDim.x) gspl[i] = 0.0;
    if (threadIdx.x < 2) gvt[threadIdx.x] = 0.0;
    __syncthreads();
    StepRec rec[SEG];
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < A.T; r += gridDim.x * blockDim.x) {
        if (!A.used_in[r]) continue;
        const float wr = A.dchi2[r];
        int off, n;
        if (wr == 0.0f || !track_ok(A, r, off, n) || n < 1) continue;
        const float tc = A.tcoll[r];
        const float4* ck = A.ckpt + ckpt_base(A, r) * (CK_FLOATS / 4);
        float lam[5] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
        float gv = 0.0f, gt0 = 0.0f;
        const int nseg = (n + SEG - 1) / SEG;
        for (int sgi = nseg - 1; sgi >= 0; sgi--) {
            PassState S;
            load_ckpt(ck + sgi * (CK_FLOATS / 4), S);
            const int k0 = sgi * SEG + 1, k1 = min(sgi * SEG + SEG, n);
            float chi2 = 0.0f;
            bool ok = true;
            for (int k = k0; k <= k1; k++) {
                StepRec& R = rec[k - k0];
                float my, mz, vy, vz;
                if (k < n) {
                    const int c = A.clus[off + n - 1 - k];
                    ok = ok && ref_step(A, S, A.cs[c], A.rowx[A.cr[c]], R);
                    Meas m;
                    measure(A, spl, c, tc, m);
                    my = m.my;
                    mz = m.mz;
                    vy = A.vy;
                    vz = A.vz;
                } else {
                    ok = ok && vertex_step(A, S, R);
                    my = mz = 0.0f;
                    vy = vz = A.vtx;
                }
                ok = ok && filter_step(S, R, my, mz, vy, vz, chi2);
            }
            if (!ok) atomicOr(A.err, 2);   // the forward pass succeeded on the same data
            for (int k = k1; k >= k0; k--) {
                const StepRec& R = rec[k - k0];
                float a0 = 2.0f * (R.W[0] * R.r[0] + R.W[1] * R.r[1]);
                float a1 = 2.0f * (R.W[1] * R.r[0] + R.W[2] * R.r[1]);
#pragma unroll
                for (int i = 0; i < 5; i++) {
                    a0 += R.K[2 * i] * lam[i];
                    a1 += R.K[2 * i + 1] * lam[i];
                }
                // mu = lam - H^T a; lam = Jr^T Jh^T mu
                const float m0 = lam[0] - a0, m1 = lam[1] - a1, m2 = lam[2], m3 = lam[3], m4 = lam[4];
                const float n0 = m0, n1 = m1;
                const float n2 = m2 + R.h.a * m0 + R.h.c * m1;
                const float n3 = m3 + R.h.d * m1;
                const float n4 = m4 + R.h.b * m0 + R.h.e * m1 + R.h.f * m2;
                lam[0] = R.j00 * n0 + R.j10 * n1 + R.j20 * n2;
                lam[1] = n1;
                lam[2] = R.j22 * n2;
                lam[3] = n3;
                lam[4] = n4;
                if (k < n) scatter_grad(A, spl, gspl, A.clus[off + n - 1 - k], tc, wr * a0, wr * a1, gv, gt0);
            }
        }
        // step 0: the deviation was set from the outermost measurement
        scatter_grad(A, spl, gspl, A.clus[off + n - 1], tc, wr * lam[0], wr * lam[1], gv, gt0);
        atomicAdd(&gvt[0], (double)gv);
        atomicAdd(&gvt[1], (double)gt0);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nc; i += blockDim.x)
        if (gspl[i] != 0.0) atomicAdd(&A.grad[2 + i], gspl[i]);
    if (threadIdx.x < 2 && gvt[threadIdx.x] != 0.0) atomicAdd(&A.grad[threadIdx.x], gvt[threadIdx.x]);
}

int fill_args(const tpc_params* p, const tpc_geometry* g, float bz, float v_nominal, float vertex_var,
              const tpc_calib_tracks* tr, const float* theta, CalibArgs& A)
{
    if (!p || !g || !g->row_x || !tr || !theta) return TPC_ERR_ARG;
    if (!g->continuous || !(g->n_sectors == 36 || g->n_sectors == 1)) return TPC_ERR_ARG;
    if (g->n_rows < 2 || g->n_rows > 255) return TPC_ERR_ARG;
    if (tr->n_tracks < 0 || tr->n_clusters < 0 || tr->n_clusters > (int64_t)INT32_MAX) return TPC_ERR_ARG;
    if (!(vertex_var > 0.0f) || !(g->z_max > 0.0f)) return TPC_ERR_ARG;
    if (tr->n_tracks > 0 && (!tr->sector || !tr->x || !tr->param || !tr->clus_offset || !tr->clus_index ||
                             !tr->t_coll || !tr->cl_sector || !tr->cl_row || !tr->cl_y || !tr->cl_t))
        return TPC_ERR_ARG;
    memset(&A, 0, sizeof(A));
    A.T = tr->n_tracks;
    A.ns = g->n_sectors;
    A.nr = g->n_rows;
    A.ncl = tr->n_clusters;
    volatile float kb = KB_C * bz;
    volatile float vy = p->sigma_y * p->sigma_y;
    volatile float vz = p->sigma_z * p->sigma_z;
    A.kb = kb;
    A.vy = vy;
    A.vz = vz;
    A.vtx = vertex_var;
    A.c0s = p->c0_snp;
    A.c0t = p->c0_tgl;
    A.c0q = p->c0_qpt;
    A.v_nom = v_nominal;
    A.zmax = g->z_max;
    A.x_first = g->row_x[0];
    A.inv_dx = 1.0f / (g->row_x[g->n_rows - 1] - g->row_x[0]);
    for (int i = 0; i < g->n_rows; i++) A.rowx[i] = g->row_x[i];
    A.sector = tr->sector;
    A.x = tr->x;
    A.param = tr->param;
    A.off = tr->clus_offset;
    A.clus = tr->clus_index;
    A.tcoll = tr->t_coll;
    A.cs = tr->cl_sector;
    A.cr = tr->cl_row;
    A.cy = tr->cl_y;
    A.ct = tr->cl_t;
    A.theta = theta;
    return TPC_OK;
}

size_t ckpt_slots(int32_t T, int64_t ncl) { return (size_t)(ncl / SEG) + (size_t)T + 1; }

int calib_grid(int T)
{
    const int want = (T + CALIB_BLOCK - 1) / CALIB_BLOCK;
    return want < 1 ? 1 : (want > 148 * 8 ? 148 * 8 : want);
}

}  // namespace

extern "C" {

int tpc_calib_workspace_size(const tpc_geometry* g, int32_t n_tracks, int64_t n_clusters, size_t* bytes)
{
    if (!g || !bytes || n_tracks < 0 || n_clusters < 0 || n_clusters > (int64_t)INT32_MAX) return TPC_ERR_ARG;
    *bytes = HDR_BYTES + ckpt_slots(n_tracks, n_clusters) * CK_FLOATS * sizeof(float);
    return TPC_OK;
}

int tpc_calib_forward(const tpc_params* p, const tpc_geometry* g, float bz, float v_nominal, float vertex_var,
                      const tpc_calib_tracks* tr, const float* theta, float* chi2, uint8_t* used, void* workspace,
                      size_t ws_bytes, void* stream)
{
    CalibArgs A;
    int rc = fill_args(p, g, bz, v_nominal, vertex_var, tr, theta, A);
    if (rc) return rc;
    size_t need;
    if ((rc = tpc_calib_workspace_size(g, tr->n_tracks, tr->n_clusters, &need))) return rc;
    if (!workspace || ws_bytes < need) return TPC_ERR_CAPACITY;
    if (tr->n_tracks > 0 && (!chi2 || !used)) return TPC_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaMemsetAsync(workspace, 0, HDR_BYTES, st) != cudaSuccess) return TPC_ERR_CUDA;
    A.err = static_cast<int32_t*>(workspace);
    A.ckpt = reinterpret_cast<float4*>(static_cast<char*>(workspace) + HDR_BYTES);
    A.chi2 = chi2;
    A.used = used;
    if (A.T == 0) return TPC_OK;
    k_calib_fwd<<<calib_grid(A.T), CALIB_BLOCK, 0, st>>>(A);
    return cudaGetLastError() == cudaSuccess ? TPC_OK : TPC_ERR_CUDA;
}

int tpc_calib_backward(const tpc_params* p, const tpc_geometry* g, float bz, float v_nominal, float vertex_var,
                       const tpc_calib_tracks* tr, const float* theta, const float* dchi2, const uint8_t* used,
                       const void* workspace, size_t ws_bytes, double* grad, void* stream)
{
    CalibArgs A;
    int rc = fill_args(p, g, bz, v_nominal, vertex_var, tr, theta, A);
    if (rc) return rc;
    size_t need;
    if ((rc = tpc_calib_workspace_size(g, tr->n_tracks, tr->n_clusters, &need))) return rc;
    if (!grad || (tr->n_tracks > 0 && (!dchi2 || !used))) return TPC_ERR_ARG;
    if (!workspace || ws_bytes < need) return TPC_ERR_CAPACITY;
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaMemsetAsync(grad, 0, sizeof(double) * TPC_CALIB_N_THETA(g->n_sectors), st) != cudaSuccess)
        return TPC_ERR_CUDA;
    char* ws = static_cast<char*>(const_cast<void*>(workspace));
    A.err = reinterpret_cast<int32_t*>(ws);
    A.ckpt = reinterpret_cast<float4*>(ws + HDR_BYTES);
    A.used_in = used;
    A.dchi2 = dchi2;
    A.grad = grad;
    if (A.T == 0) return TPC_OK;
    const size_t smem = (size_t)TPC_CALIB_N_THETA(A.ns) * (sizeof(double) + sizeof(float));
    if (cudaFuncSetAttribute(k_calib_bwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return TPC_ERR_CUDA;
    k_calib_bwd<<<calib_grid(A.T), CALIB_BLOCK, smem, st>>>(A);
    return cudaGetLastError() == cudaSuccess ? TPC_OK : TPC_ERR_CUDA;
}

int tpc_calib_status(const void* workspace, int32_t* err, void* stream)
{
    if (!workspace || !err) return TPC_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaMemcpyAsync(err, workspace, sizeof(int32_t), cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return TPC_ERR_CUDA;
    return cudaStreamSynchronize(st) == cudaSuccess ? TPC_OK : TPC_ERR_CUDA;
}

}  // extern "C"
