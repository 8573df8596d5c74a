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
// TPC_CALIB_CKPT_STEPS steps and its final deviation.  The backward kernel
// walks the segments from the vertex end back: it recomputes one segment's
// reference from its checkpoint into local memory (Jacobian entries and
// reference position of every step), then sweeps the smoothed deviation back
// through the inverse Jacobians; the derivative of the chi2 with respect to
// each measurement is twice its weighted smoothed residual (k_calib_bwd
// states why), and a_k dm_k/dtheta goes into the gradient: the spline part through
// per-thread register sums over the clusters that share a spline support,
// added to the binary64 global sums, v and t0 through per-track
// binary32 sums added to block-private binary64 sums, all flushed once per
// block into binary64 global sums.  Tolerance path: multiply-add
// contraction allowed.
#include "tpc_calib.h"
#include "tpc_dev.cuh"
#include "tpc_fit.cuh"

#include <cmath>
#include <cstring>
#include <algorithm>
#include <vector>

using namespace tpc;
using namespace tpc::fit;

namespace {

constexpr int NSPL = TPC_CALIB_NSPL;
constexpr int SEG = TPC_CALIB_CKPT_STEPS;
constexpr int CK_FLOATS = 12;          // reference: x, sector, p[5], pl[5]
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
    const float* tgl;                   // [T] dip angle of the matched inner track (NaN: none), may be null
    float tvar;
    float* chi2;
    uint8_t* used;
    const uint8_t* used_in;
    const float* dchi2;
    double* grad;
    float4* ckpt;
    float4* dfin;                       // [T][2]: deviation after the vertex step
    int32_t* order;                     // [T]: tracks by decreasing cluster count
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
    // error scale of m_z (the drift-time error through the map): es = (v /
    // v_nom) (1 - d dz / d zl at the nominal position); d es / d c[i0+a]
    // [j0n+b][z] = -(v / v_nom) Bu[a] dBn[b]
    float es;
    int j0n;
    float dBn[4];
};

// per-row u-basis table in shared memory: ub[4 r + a] the four non-zero
// basis values at row r's u, ui[r] the index of the first
struct RowBasis {
    float* ub;
    int* ui;
};

__device__ __forceinline__ void load_row_basis(const CalibArgs& A, RowBasis rb)
{
    for (int r = threadIdx.x; r < A.nr; r += blockDim.x) {
        float B[4], dB[4];
        rb.ui[r] = bspline((A.rowx[r] - A.x_first) * A.inv_dx, B, dB);
#pragma unroll
        for (int a = 0; a < 4; a++) rb.ub[4 * r + a] = B[a];
    }
}

__device__ __forceinline__ void measure(const CalibArgs& A, const float* __restrict__ spl, RowBasis rb, int c,
                                        float tc, Meas& m)
{
    const int s = A.cs[c];
    const int row = A.cr[c];
    const float v = A.theta[0], t0 = A.theta[1];
    const float tau = (A.ct[c] - tc) - t0;
    const float zl = A.zmax - v * tau;
    const float w = zl / A.zmax;
    const float dwdz = (w > 0.0f && w < 1.0f) ? 1.0f / A.zmax : 0.0f;
    float dBw[4];
    m.i0 = rb.ui[row];
#pragma unroll
    for (int a = 0; a < 4; a++) m.Bu[a] = rb.ub[4 * row + a];
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
    // the slope of the map at the nominal position (v_nom, no t0)
    const float wn = (A.zmax - A.v_nom * (A.ct[c] - tc)) / A.zmax;
    const float dwn = (wn > 0.0f && wn < 1.0f) ? 1.0f / A.zmax : 0.0f;
    float Bn[4], dBn[4];
    m.j0n = bspline(wn, Bn, dBn);
    const float* cn = spl + (s * NSPL * NSPL + m.i0 * NSPL + m.j0n) * 2;
    float dzn = 0.0f;
#pragma unroll
    for (int a = 0; a < 4; a++) {
        float rz = 0.0f;
#pragma unroll
        for (int b = 0; b < 4; b++) rz += dBn[b] * cn[(a * NSPL + b) * 2 + 1];
        dzn += m.Bu[a] * rz;
    }
    m.es = (v / A.v_nom) * (1.0f - dzn * dwn);
#pragma unroll
    for (int b = 0; b < 4; b++) m.dBn[b] = dBn[b] * dwn;
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
    dst[0] = make_float4(S.x, __int_as_float(S.sec), S.p[0], S.p[1]);
    dst[1] = make_float4(S.p[2], S.p[3], S.p[4], S.pl[0]);
    dst[2] = make_float4(S.pl[1], S.pl[2], S.pl[3], S.pl[4]);
}

__device__ __forceinline__ void load_ckpt(const float4* src, PassState& S)
{
    const float4 a = src[0], b = src[1], c = src[2];
    S.x = a.x;
    S.sec = __float_as_int(a.y);
    S.p[0] = a.z;
    S.p[1] = a.w;
    S.p[2] = b.x;
    S.p[3] = b.y;
    S.p[4] = b.z;
    S.pl[0] = b.w;
    S.pl[1] = c.x;
    S.pl[2] = c.y;
    S.pl[3] = c.z;
    S.pl[4] = c.w;
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
    __shared__ float ub[4 * 256];
    __shared__ int ui[256];
    const RowBasis rb{ub, ui};
    load_spline(A, spl);
    load_row_basis(A, rb);
    __syncthreads();
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < A.T; i += gridDim.x * blockDim.x) {
        const int r = A.order[i];               // longest tracks first: similar lengths share a warp
        int off, n;
        const float tc = A.tcoll[r];
        float chi2 = 0.0f;
        bool ok = track_ok(A, r, off, n) && n >= 2 && !isnan(tc);
        PassState S;
        if (ok) ok = ref_outward(A, r, off, n, tc, S);
        float4* ck = A.ckpt + ckpt_base(A, r) * (CK_FLOATS / 4);
        if (ok) {
            Meas m;
            measure(A, spl, rb, A.clus[off + n - 1], tc, m);
            S.dp[0] = (m.my - S.p[0]) - S.pl[0];
            S.dp[1] = (m.mz - S.p[1]) - S.pl[1];
            S.dp[2] = S.dp[3] = S.dp[4] = 0.0f;
#pragma unroll
            for (int i = 0; i < 15; i++) S.C[i] = 0.0f;
            S.C[0] = A.vy;
            S.C[2] = A.vz * m.es * m.es;
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
                    measure(A, spl, rb, c, tc, m);
                    my = m.my;
                    mz = m.mz;
                    vy = A.vy;
                    vz = A.vz * m.es * m.es;
                } else {
                    ok = vertex_step(A, S, R);
                    if (!ok) break;
                    my = mz = 0.0f;
                    vy = vz = A.vtx;
                }
                ok = filter_step(S, R, my, mz, vy, vz, chi2);
                if (ok && k % SEG == 0 && k < n) save_ckpt(ck + (k / SEG) * (CK_FLOATS / 4), S);
            }
            // the dip angle of the matched inner track: one more update at the
            // vertex (H selects tan(lambda)); no covariance is needed after it
            const float tm = (ok && A.tgl) ? A.tgl[r] : __int_as_float(0x7fc00000);
            if (!isnan(tm)) {
                const float rr = ((tm - S.p[3]) - S.pl[3]) - S.dp[3];
                const float sv = S.C[CI(3, 3)] + A.tvar;
                if (!(sv > 0.0f)) {
                    ok = false;
                } else {
                    const float w = 1.0f / sv;
                    chi2 += rr * w * rr;
#pragma unroll
                    for (int i = 0; i < 5; i++) S.dp[i] += S.C[cidx(i, 3)] * w * rr;
                }
            }
            if (ok) {
                A.dfin[2 * (int64_t)r] = make_float4(S.dp[0], S.dp[1], S.dp[2], S.dp[3]);
                A.dfin[2 * (int64_t)r + 1] = make_float4(S.dp[4], 0.0f, 0.0f, 0.0f);
            }
        }
        A.chi2[r] = ok ? chi2 : 0.0f;
        A.used[r] = ok ? 1 : 0;
    }
}

// Spline-gradient sums of one thread: the 4 x 4 (dy, dz) coefficients of
// the current support (sector, first u index, first w index) are summed in
// registers and added to the binary64 global gradient only when the support
// changes (consecutive clusters of a track mostly share it).
struct GradAcc {
    int key;             // s * 64 + i0 * 8 + j0, -1: empty
    float g[32];         // [(i * 4 + j) * 2 + k]
};

__device__ __forceinline__ void flush(GradAcc& G, double* grad)
{
    if (G.key < 0) return;
    const int s = G.key >> 6, i0 = (G.key >> 3) & 7, j0 = G.key & 7;
    double* g = grad + 2 + (s * NSPL * NSPL + i0 * NSPL + j0) * 2;
#pragma unroll
    for (int i = 0; i < 4; i++)
#pragma unroll
        for (int j = 0; j < 4; j++) {
            atomicAdd(&g[(i * NSPL + j) * 2], (double)G.g[(i * 4 + j) * 2]);
            atomicAdd(&g[(i * NSPL + j) * 2 + 1], (double)G.g[(i * 4 + j) * 2 + 1]);
        }
#pragma unroll
    for (int q = 0; q < 32; q++) G.g[q] = 0.0f;
    G.key = -1;
}

// Sums of the error-scale term of the z coefficients (support of the
// nominal-position slope), flushed like GradAcc
struct SlopeAcc {
    int key;
    float g[16];         // [i * 4 + j]
};

__device__ __forceinline__ void flush(SlopeAcc& G, double* grad)
{
    if (G.key < 0) return;
    const int s = G.key >> 6, i0 = (G.key >> 3) & 7, j0 = G.key & 7;
    double* g = grad + 2 + (s * NSPL * NSPL + i0 * NSPL + j0) * 2;
#pragma unroll
    for (int i = 0; i < 4; i++)
#pragma unroll
        for (int j = 0; j < 4; j++) atomicAdd(&g[(i * NSPL + j) * 2 + 1], (double)G.g[i * 4 + j]);
#pragma unroll
    for (int q = 0; q < 16; q++) G.g[q] = 0.0f;
    G.key = -1;
}

// the derivative through the variance of m_z: with V = vz es^2 and the
// smoothed residual r1, d chi2 / d es = -2 r1^2 / (V es) (weight wr)
__device__ __forceinline__ void scatter_var(const CalibArgs& A, SlopeAcc& G, const Meas& m, float wr, float r1,
                                            float iv, float& gv, double* grad)
{
    const float q = -2.0f * wr * r1 * r1 * iv / m.es;
    gv += q * m.es / A.theta[0];
    const int key = m.s * 64 + m.i0 * 8 + m.j0n;
    if (key != G.key) {
        flush(G, grad);
        G.key = key;
    }
    const float f = -q * A.theta[0] / A.v_nom;
#pragma unroll
    for (int i = 0; i < 4; i++)
#pragma unroll
        for (int j = 0; j < 4; j++) G.g[i * 4 + j] += f * m.Bu[i] * m.dBn[j];
}

// adds a0 dm_y/dtheta + a1 dm_z/dtheta of measurement m
__device__ __forceinline__ void scatter_grad(const CalibArgs& A, const float* spl, RowBasis rb, GradAcc& G,
                                             const Meas& m, float a0, float a1, float& gv, float& gt0, double* grad)
{
    gv += a0 * m.dy_v + a1 * m.dz_v;
    gt0 += a0 * m.dy_t0 + a1 * m.dz_t0;
    const int key = m.s * 64 + m.i0 * 8 + m.j0;
    if (key != G.key) {
        flush(G, grad);
        G.key = key;
    }
    const float ay = -a0, az = -a1 * m.sgn;      // m_y = y - dy, m_z = sgn (zl - dz)
#pragma unroll
    for (int i = 0; i < 4; i++) {
        const float by = ay * m.Bu[i], bz = az * m.Bu[i];
#pragma unroll
        for (int j = 0; j < 4; j++) {
            G.g[(i * 4 + j) * 2] += by * m.Bw[j];
            G.g[(i * 4 + j) * 2 + 1] += bz * m.Bw[j];
        }
    }
}

// reference of one step for the backward sweep: the step's Jacobians and
// the reference (y, z) as compensated pairs
struct BackRec {
    float j00, j10, j20, j22;
    HelixJac h;
    float y, yl, z, zl;
};

// v <- F^-1 v for F = Jh Jr: back substitution through the unit upper
// triangular helix Jacobian, then the lower triangular rotation Jacobian
__device__ __forceinline__ void inv_step(const BackRec& R, float* v)
{
    const float u4 = v[4], u3 = v[3];
    const float u2 = v[2] - R.h.f * u4;
    const float u1 = v[1] - R.h.c * u2 - R.h.d * u3 - R.h.e * u4;
    const float u0 = v[0] - R.h.a * u2 - R.h.b * u4;
    v[0] = u0 / R.j00;
    v[1] = u1 - R.j10 * v[0];
    v[2] = (u2 - R.j20 * v[0]) / R.j22;
    v[3] = u3;
    v[4] = u4;
}

// The pass is a linear least-squares problem in the deviation at step 0
// (prior at step 0, no process noise), its chi2 the minimum of that problem.
// By the envelope theorem the derivative of the minimum with respect to a
// cluster measurement m_k is the partial derivative at the optimum:
//   d chi2 / d m_k = 2 V_k^-1 (m_k - h_k - H dev*_k),
// with dev*_k the smoothed deviation.  Without process noise the smoothed
// track is deterministic: dev*_{k-1} = F_k^-1 dev*_k, starting from the
// filtered deviation after the last (vertex) step.  Step 0 is the prior
// centred on the outermost measurement, which enters the same way with
// V_0 = diag(sigma_y^2, sigma_z^2).  The backward kernel therefore
// recomputes only the reference of each segment from its checkpoint (no
// covariance work) and sweeps the smoothed deviation back.
__global__ void __launch_bounds__(CALIB_BLOCK) k_calib_bwd(CalibArgs A)
{
    // dynamic shared memory: the spline, then the per-row u-basis table
    extern __shared__ float smem[];
    __shared__ double gvt[2];
    const int nc = A.ns * NSPL * NSPL * 2;
    float* spl = smem;
    const RowBasis rb{spl + nc, reinterpret_cast<int*>(spl + nc + 4 * 256)};
    load_spline(A, spl);
    load_row_basis(A, rb);
    if (threadIdx.x < 2) gvt[threadIdx.x] = 0.0;
    __syncthreads();
    const float ivy = 1.0f / A.vy, ivz = 1.0f / A.vz;
    BackRec rec[SEG];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < A.T; i += gridDim.x * blockDim.x) {
        const int r = A.order[i];               // longest tracks first: similar lengths share a warp
        if (!A.used_in[r]) continue;
        const float wr = A.dchi2[r];
        int off, n;
        if (wr == 0.0f || !track_ok(A, r, off, n) || n < 1) continue;
        const float tc = A.tcoll[r];
        const float4* ck = A.ckpt + ckpt_base(A, r) * (CK_FLOATS / 4);
        const float4 d0 = A.dfin[2 * (int64_t)r], d1 = A.dfin[2 * (int64_t)r + 1];
        float dev[5] = {d0.x, d0.y, d0.z, d0.w, d1.x};
        float gv = 0.0f, gt0 = 0.0f;
        GradAcc G;
        G.key = -1;
#pragma unroll
        for (int q = 0; q < 32; q++) G.g[q] = 0.0f;
        SlopeAcc GS;
        GS.key = -1;
#pragma unroll
        for (int q = 0; q < 16; q++) GS.g[q] = 0.0f;
        const int nseg = (n + SEG - 1) / SEG;
        bool ok = true;
        float hy = 0.0f, hyl = 0.0f, hz = 0.0f, hzl = 0.0f;
        for (int sgi = nseg - 1; sgi >= 0; sgi--) {
            PassState S;
            load_ckpt(ck + sgi * (CK_FLOATS / 4), S);
            hy = S.p[0];
            hyl = S.pl[0];
            hz = S.p[1];
            hzl = S.pl[1];
            const int k0 = sgi * SEG + 1, k1 = min(sgi * SEG + SEG, n);
            for (int k = k0; k <= k1; k++) {
                BackRec& R = rec[k - k0];
                StepRec J;
                if (k < n) {
                    const int c = A.clus[off + n - 1 - k];
                    ok = ok && ref_step(A, S, A.cs[c], A.rowx[A.cr[c]], J);
                } else {
                    ok = ok && vertex_step(A, S, J);
                }
                R.j00 = J.j00;
                R.j10 = J.j10;
                R.j20 = J.j20;
                R.j22 = J.j22;
                R.h = J.h;
                R.y = S.p[0];
                R.yl = S.pl[0];
                R.z = S.p[1];
                R.zl = S.pl[1];
            }
            for (int k = k1; k >= k0; k--) {
                const BackRec& R = rec[k - k0];
                if (k < n) {
                    const int c = A.clus[off + n - 1 - k];
                    Meas m;
                    measure(A, spl, rb, c, tc, m);
                    const float r0 = ((m.my - R.y) - R.yl) - dev[0];
                    const float r1 = ((m.mz - R.z) - R.zl) - dev[1];
                    const float iv = ivz / (m.es * m.es);
                    scatter_grad(A, spl, rb, G, m, 2.0f * wr * ivy * r0, 2.0f * wr * iv * r1, gv, gt0, A.grad);
                    scatter_var(A, GS, m, wr, r1, iv, gv, A.grad);
                }
                inv_step(R, dev);
            }
        }
        if (!ok) atomicOr(A.err, 2);       // the forward pass succeeded on the same data
        // step 0: the prior centred on the outermost measurement
        {
            const int c = A.clus[off + n - 1];
            Meas m;
            measure(A, spl, rb, c, tc, m);
            const float r0 = ((m.my - hy) - hyl) - dev[0];
            const float r1 = ((m.mz - hz) - hzl) - dev[1];
            const float iv = ivz / (m.es * m.es);
            scatter_grad(A, spl, rb, G, m, 2.0f * wr * ivy * r0, 2.0f * wr * iv * r1, gv, gt0, A.grad);
            scatter_var(A, GS, m, wr, r1, iv, gv, A.grad);
        }
        flush(G, A.grad);
        flush(GS, A.grad);
        atomicAdd(&gvt[0], (double)gv);
        atomicAdd(&gvt[1], (double)gt0);
    }
    __syncthreads();
    if (threadIdx.x < 2 && gvt[threadIdx.x] != 0.0) atomicAdd(&A.grad[threadIdx.x], gvt[threadIdx.x]);
}

// One block: counting sort of the tracks by decreasing cluster count into
// A.order (schedule only; every track's results are independent of it).
constexpr int ORDER_BUCKETS = 1024;
__global__ void __launch_bounds__(ORDER_BUCKETS) k_calib_order(CalibArgs A)
{
    __shared__ unsigned cnt[ORDER_BUCKETS];
    cnt[threadIdx.x] = 0;
    __syncthreads();
    auto bucket = [&](int r) {
        const int n = A.off[r + 1] - A.off[r];
        return ORDER_BUCKETS - 1 - min(max(n, 0), ORDER_BUCKETS - 1);
    };
    for (int r = threadIdx.x; r < A.T; r += blockDim.x) atomicAdd(&cnt[bucket(r)], 1u);
    __syncthreads();
    // exclusive scan of the bucket counts (Hillis-Steele on the inclusive sums)
    unsigned v = cnt[threadIdx.x];
    for (int o = 1; o < ORDER_BUCKETS; o <<= 1) {
        __syncthreads();
        const unsigned add = threadIdx.x >= (unsigned)o ? cnt[threadIdx.x - o] : 0u;
        __syncthreads();
        cnt[threadIdx.x] += add;
    }
    __syncthreads();
    const unsigned excl = cnt[threadIdx.x] - v;
    __syncthreads();
    cnt[threadIdx.x] = excl;
    __syncthreads();
    for (int r = threadIdx.x; r < A.T; r += blockDim.x) A.order[atomicAdd(&cnt[bucket(r)], 1u)] = r;
}

// Calibration track selection: one thread per track, NaN marks a track the
// calibration passes leave out (failed refit or |q/pT| > qpt_max).
__global__ void k_calib_select(int T, const float* t_coll, const int32_t* __restrict__ status,
                               const float* __restrict__ param, float qpt_max, float* t_sel)
{
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < T; r += gridDim.x * blockDim.x) {
        const bool keep = status[r] == 0 && fabsf(param[5 * r + 4]) <= qpt_max;
        t_sel[r] = keep ? t_coll[r] : __int_as_float(0x7fc00000);
    }
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
    A.tgl = tr->tgl_ext;
    A.tvar = tr->tgl_var;
    if (A.tgl && !(A.tvar > 0.0f)) return TPC_ERR_ARG;
    return TPC_OK;
}

size_t ckpt_slots(int32_t T, int64_t ncl) { return (size_t)(ncl / SEG) + (size_t)T + 1; }
// workspace: header, checkpoints (CK_FLOATS per slot), final deviations (8
// floats per track), the track order (1 int per track, 16-byte padded)
size_t dfin_offset(int32_t T, int64_t ncl) { return HDR_BYTES + ckpt_slots(T, ncl) * CK_FLOATS * sizeof(float); }
size_t order_offset(int32_t T, int64_t ncl) { return dfin_offset(T, ncl) + (size_t)T * 8 * sizeof(float); }

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
    *bytes = order_offset(n_tracks, n_clusters) + ((size_t)n_tracks + 3) / 4 * 16;
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
    A.dfin = reinterpret_cast<float4*>(static_cast<char*>(workspace) + dfin_offset(A.T, A.ncl));
    A.order = reinterpret_cast<int32_t*>(static_cast<char*>(workspace) + order_offset(A.T, A.ncl));
    A.chi2 = chi2;
    A.used = used;
    if (A.T == 0) return TPC_OK;
    k_calib_order<<<1, ORDER_BUCKETS, 0, st>>>(A);        // the backward pass reuses this order
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
    A.dfin = reinterpret_cast<float4*>(ws + dfin_offset(A.T, A.ncl));
    A.order = reinterpret_cast<int32_t*>(ws + order_offset(A.T, A.ncl));
    A.used_in = used;
    A.dchi2 = dchi2;
    A.grad = grad;
    if (A.T == 0) return TPC_OK;
    const size_t smem = (size_t)TPC_CALIB_N_THETA(A.ns) * sizeof(float) + 256 * (4 * sizeof(float) + sizeof(int));
    if (cudaFuncSetAttribute(k_calib_bwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return TPC_ERR_CUDA;
    k_calib_bwd<<<calib_grid(A.T), CALIB_BLOCK, smem, st>>>(A);
    return cudaGetLastError() == cudaSuccess ? TPC_OK : TPC_ERR_CUDA;
}

int tpc_calib_select(int32_t n_tracks, const float* t_coll, const int32_t* status, const float* param,
                     float qpt_max, float* t_sel, void* stream)
{
    if (n_tracks < 0 || qpt_max != qpt_max) return TPC_ERR_ARG;
    if (n_tracks == 0) return TPC_OK;
    if (!t_coll || !status || !param || !t_sel) return TPC_ERR_ARG;
    const int grid = calib_grid(n_tracks);
    k_calib_select<<<grid, CALIB_BLOCK, 0, (cudaStream_t)stream>>>(n_tracks, t_coll, status, param, qpt_max, t_sel);
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

// ---------------------------------------------------------------------------
// Closed-loop calibration (tpc_calib_fit): selection kernels and the host
// L-BFGS over theta
// ---------------------------------------------------------------------------
namespace {

// binary64 sum of chi2 over the used tracks (one block)
__global__ void __launch_bounds__(1024) k_fit_sum(const float* __restrict__ chi2, const uint8_t* __restrict__ used,
                                                  int T, double* __restrict__ out)
{
    __shared__ double part[32];
    double s = 0.0;
    for (int r = threadIdx.x; r < T; r += blockDim.x)
        if (used[r]) s += (double)chi2[r];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); k++) t += part[k];
        *out = t;
    }
}

__global__ void k_fit_fill(float* __restrict__ a, int n, float v)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) a[i] = v;
}

// selection at the current theta: a track is kept when its pass without the
// dip angle is used and chi2 / (2 n) < ndf_cut; its dip angle when given and
// its chi2 contribution (with - without) < anchor_cut.  counts[0] tracks,
// counts[1] dip angles kept.
__global__ void k_fit_select(int T, const int32_t* __restrict__ off, const float* __restrict__ t_coll,
                             const float* __restrict__ tgl, const float* __restrict__ chi2_f,
                             const uint8_t* __restrict__ used_f, const float* __restrict__ chi2_a,
                             const uint8_t* __restrict__ used_a, float ndf_cut, float anchor_cut,
                             float* __restrict__ tsel, float* __restrict__ tgl_sel, int* __restrict__ counts)
{
    const float NaN = __int_as_float(0x7fc00000);
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < T; r += gridDim.x * blockDim.x) {
        const float ndf = 2.0f * (float)(off[r + 1] - off[r]);
        const bool keep = used_f[r] && chi2_f[r] < ndf_cut * ndf;
        tsel[r] = keep ? t_coll[r] : NaN;
        bool anc = false;
        if (tgl) {
            anc = keep && used_a[r] && !isnan(tgl[r]) && chi2_a[r] - chi2_f[r] < anchor_cut;
            tgl_sel[r] = anc ? tgl[r] : NaN;
        }
        if (keep) atomicAdd(&counts[0], 1);
        if (anc) atomicAdd(&counts[1], 1);
    }
}

struct FitLayout {
    size_t tsel, tgl, chi2a, chi2f, useda, usedf, ones, grad, theta, sum, counts, total;
};

FitLayout fit_layout(size_t calib_ws, int32_t T, int n_theta)
{
    FitLayout L;
    size_t o = (calib_ws + 255) / 256 * 256;
    auto take = [&](size_t b) { size_t r = o; o = (o + std::max<size_t>(b, 1) + 255) / 256 * 256; return r; };
    L.tsel = take(4 * (size_t)T);
    L.tgl = take(4 * (size_t)T);
    L.chi2a = take(4 * (size_t)T);
    L.chi2f = take(4 * (size_t)T);
    L.useda = take((size_t)T);
    L.usedf = take((size_t)T);
    L.ones = take(4 * (size_t)T);
    L.grad = take(8 * (size_t)n_theta);
    L.theta = take(4 * (size_t)n_theta);
    L.sum = take(8);
    L.counts = take(8);
    L.total = o;
    return L;
}

}  // namespace

extern "C" {

int tpc_calib_fit_defaults(tpc_calib_fit_opts* o)
{
    if (!o) return TPC_ERR_ARG;
    o->prior_sigma = 0.3f;
    o->scale_v = 0.01f;
    o->scale_t0 = 0.1f;
    o->max_iter = 300;
    o->rounds = 2;
    o->chi2ndf_first = 10.0f;
    o->anchor_cut_first = 100.0f;
    o->chi2ndf_cut = 2.5f;
    o->anchor_cut = 16.0f;
    o->ftol = 1e-10;
    return TPC_OK;
}

int tpc_calib_fit_workspace_size(const tpc_geometry* g, int32_t n_tracks, int64_t n_clusters, size_t* bytes)
{
    size_t cw = 0;
    int rc = tpc_calib_workspace_size(g, n_tracks, n_clusters, &cw);
    if (rc) return rc;
    *bytes = fit_layout(cw, n_tracks, TPC_CALIB_N_THETA(g->n_sectors)).total;
    return TPC_OK;
}

int tpc_calib_fit(const tpc_params* p, const tpc_geometry* g, float bz, float v_nominal, float vertex_var,
                  const tpc_calib_tracks* tr, const tpc_calib_fit_opts* opt, float* theta, void* workspace,
                  size_t ws_bytes, float* t_used, float* tgl_used, tpc_calib_fit_report* rep, void* stream)
{
    if (!p || !g || !tr || !opt || !theta) return TPC_ERR_ARG;
    {
        CalibArgs A;
        const int rc = fill_args(p, g, bz, v_nominal, vertex_var, tr, theta, A);
        if (rc) return rc;
    }
    if (!(opt->prior_sigma > 0.0f) || !(opt->scale_v > 0.0f) || !(opt->scale_t0 > 0.0f) || opt->max_iter < 1 ||
        opt->rounds < 0 || !(opt->ftol >= 0.0))
        return TPC_ERR_ARG;
    size_t cw = 0, need = 0;
    int rc = tpc_calib_workspace_size(g, tr->n_tracks, tr->n_clusters, &cw);
    if (rc) return rc;
    const int T = tr->n_tracks, NT = TPC_CALIB_N_THETA(g->n_sectors);
    const FitLayout L = fit_layout(cw, T, NT);
    need = L.total;
    if (!workspace || ws_bytes < need) return TPC_ERR_CAPACITY;
    cudaStream_t st = (cudaStream_t)stream;
    char* ws = static_cast<char*>(workspace);
    float* tsel = reinterpret_cast<float*>(ws + L.tsel);
    float* tgls = reinterpret_cast<float*>(ws + L.tgl);
    float* chi2a = reinterpret_cast<float*>(ws + L.chi2a);
    float* chi2f = reinterpret_cast<float*>(ws + L.chi2f);
    uint8_t* useda = reinterpret_cast<uint8_t*>(ws + L.useda);
    uint8_t* usedf = reinterpret_cast<uint8_t*>(ws + L.usedf);
    float* ones = reinterpret_cast<float*>(ws + L.ones);
    double* gradd = reinterpret_cast<double*>(ws + L.grad);
    float* thd = reinterpret_cast<float*>(ws + L.theta);
    double* sumd = reinterpret_cast<double*>(ws + L.sum);
    int* cnt = reinterpret_cast<int*>(ws + L.counts);
#define FCK(x) do { if ((x) != cudaSuccess) return TPC_ERR_CUDA; } while (0)
    const int grid = calib_grid(std::max(T, 1));
    if (T > 0) k_fit_fill<<<grid, CALIB_BLOCK, 0, st>>>(ones, T, 1.0f);
    // the start
    std::vector<float> th32(NT);
    FCK(cudaMemcpyAsync(th32.data(), theta, 4 * (size_t)NT, cudaMemcpyDeviceToHost, st));
    FCK(cudaStreamSynchronize(st));
    std::vector<double> th0(th32.begin(), th32.end());
    std::vector<double> D(NT, (double)opt->prior_sigma);
    D[0] = opt->scale_v;
    D[1] = opt->scale_t0;
    const double ip2 = 1.0 / ((double)opt->prior_sigma * opt->prior_sigma);
    tpc_calib_tracks tf = *tr;          // the fit's view: selected tracks and dip angles
    tf.t_coll = tsel;
    tf.tgl_ext = tr->tgl_ext ? tgls : nullptr;
    int evals = 0;
    // F and dF/dtheta at theta (host, binary64) with the current selection
    auto evaluate = [&](const std::vector<double>& th, double& F, std::vector<double>& gth) -> int {
        for (int i = 0; i < NT; i++) th32[i] = (float)th[i];
        FCK(cudaMemcpyAsync(thd, th32.data(), 4 * (size_t)NT, cudaMemcpyHostToDevice, st));
        int r2 = tpc_calib_forward(p, g, bz, v_nominal, vertex_var, &tf, thd, chi2a, useda, workspace, cw, stream);
        if (r2) return r2;
        if (T > 0) k_fit_sum<<<1, 1024, 0, st>>>(chi2a, useda, T, sumd);
        else FCK(cudaMemsetAsync(sumd, 0, 8, st));
        r2 = tpc_calib_backward(p, g, bz, v_nominal, vertex_var, &tf, thd, ones, useda, workspace, cw, gradd,
                                stream);
        if (r2) return r2;
        double s = 0.0;
        gth.assign(NT, 0.0);
        FCK(cudaMemcpyAsync(&s, sumd, 8, cudaMemcpyDeviceToHost, st));
        FCK(cudaMemcpyAsync(gth.data(), gradd, 8 * (size_t)NT, cudaMemcpyDeviceToHost, st));
        FCK(cudaStreamSynchronize(st));
        F = s;
        for (int i = 2; i < NT; i++) {
            F += th[i] * th[i] * ip2;
            gth[i] += 2.0 * th[i] * ip2;
        }
        evals++;
        return TPC_OK;
    };
    // selection at th
    auto select = [&](const std::vector<double>& th, float ndf_cut, float anchor_cut, int& ntr, int& nanc) -> int {
        for (int i = 0; i < NT; i++) th32[i] = (float)th[i];
        FCK(cudaMemcpyAsync(thd, th32.data(), 4 * (size_t)NT, cudaMemcpyHostToDevice, st));
        tpc_calib_tracks tfree = *tr;
        tfree.tgl_ext = nullptr;
        int r2 = tpc_calib_forward(p, g, bz, v_nominal, vertex_var, &tfree, thd, chi2f, usedf, workspace, cw, stream);
        if (r2) return r2;
        if (tr->tgl_ext) {
            r2 = tpc_calib_forward(p, g, bz, v_nominal, vertex_var, tr, thd, chi2a, useda, workspace, cw, stream);
            if (r2) return r2;
        }
        FCK(cudaMemsetAsync(cnt, 0, 8, st));
        if (T > 0)
            k_fit_select<<<grid, CALIB_BLOCK, 0, st>>>(T, tr->clus_offset, tr->t_coll, tr->tgl_ext, chi2f, usedf,
                                                       chi2a, useda, ndf_cut, anchor_cut, tsel, tgls, cnt);
        FCK(cudaGetLastError());
        int c[2] = {0, 0};
        FCK(cudaMemcpyAsync(c, cnt, 8, cudaMemcpyDeviceToHost, st));
        FCK(cudaStreamSynchronize(st));
        ntr = c[0];
        nanc = c[1];
        return TPC_OK;
    };
    std::vector<double> th = th0, gth, gx(NT), x(NT), xn(NT), gn(NT), thn(NT), d(NT);
    int ntr = 0, nanc = 0, rounds = 0;
    double F = 0.0, f_start = 0.0;
    for (int round = 0; round <= opt->rounds; round++) {
        rc = select(th, round == 0 ? opt->chi2ndf_first : opt->chi2ndf_cut,
                    round == 0 ? opt->anchor_cut_first : opt->anchor_cut, ntr, nanc);
        if (rc) return rc;
        rounds++;
        // L-BFGS in x = (theta - base) / D from x = 0
        const std::vector<double> base = th;
        std::fill(x.begin(), x.end(), 0.0);
        if ((rc = evaluate(th, F, gth))) return rc;
        if (round == 0) f_start = F;
        for (int i = 0; i < NT; i++) gx[i] = D[i] * gth[i];
        constexpr int M = 10;
        std::vector<std::vector<double>> S, Y;
        std::vector<double> rho;
        for (int it = 0; it < opt->max_iter; it++) {
            // two-loop recursion: d = -H gx
            std::vector<double> q = gx, alpha(S.size());
            for (int k = (int)S.size() - 1; k >= 0; k--) {
                double a = 0.0;
                for (int i = 0; i < NT; i++) a += S[k][i] * q[i];
                a *= rho[k];
                alpha[k] = a;
                for (int i = 0; i < NT; i++) q[i] -= a * Y[k][i];
            }
            double gamma = 1.0;
            if (!S.empty()) {
                double sy = 0.0, yy = 0.0;
                for (int i = 0; i < NT; i++) {
                    sy += S.back()[i] * Y.back()[i];
                    yy += Y.back()[i] * Y.back()[i];
                }
                gamma = sy / yy;
            } else {
                double gg = 0.0;
                for (int i = 0; i < NT; i++) gg += gx[i] * gx[i];
                gamma = gg > 0.0 ? 1.0 / std::sqrt(gg) : 1.0;
            }
            for (int i = 0; i < NT; i++) q[i] *= gamma;
            for (int k = 0; k < (int)S.size(); k++) {
                double b = 0.0;
                for (int i = 0; i < NT; i++) b += Y[k][i] * q[i];
                b *= rho[k];
                for (int i = 0; i < NT; i++) q[i] += S[k][i] * (alpha[k] - b);
            }
            double dg = 0.0;
            for (int i = 0; i < NT; i++) {
                d[i] = -q[i];
                dg += d[i] * gx[i];
            }
            if (!(dg < 0.0)) {              // not a descent direction: restart from the gradient
                S.clear(); Y.clear(); rho.clear();
                double gg = 0.0;
                for (int i = 0; i < NT; i++) gg += gx[i] * gx[i];
                const double sc = gg > 0.0 ? 1.0 / std::sqrt(gg) : 0.0;
                dg = 0.0;
                for (int i = 0; i < NT; i++) {
                    d[i] = -gx[i] * sc;
                    dg += d[i] * gx[i];
                }
                if (!(dg < 0.0)) break;
            }
            double step = 1.0, Fn = 0.0;
            bool ok = false;
            for (int ls = 0; ls < 40; ls++) {
                for (int i = 0; i < NT; i++) {
                    xn[i] = x[i] + step * d[i];
                    thn[i] = base[i] + D[i] * xn[i];
                }
                std::vector<double> gthn;
                if ((rc = evaluate(thn, Fn, gthn))) return rc;
                if (Fn <= F + 1e-4 * step * dg) {
                    for (int i = 0; i < NT; i++) gn[i] = D[i] * gthn[i];
                    ok = true;
                    break;
                }
                step *= 0.5;
            }
            if (!ok) break;
            std::vector<double> s(NT), y(NT);
            double sy = 0.0, ss = 0.0, yy = 0.0;
            for (int i = 0; i < NT; i++) {
                s[i] = xn[i] - x[i];
                y[i] = gn[i] - gx[i];
                sy += s[i] * y[i];
                ss += s[i] * s[i];
                yy += y[i] * y[i];
            }
            if (sy > 1e-12 * std::sqrt(ss * yy)) {
                if ((int)S.size() == M) {
                    S.erase(S.begin()); Y.erase(Y.begin()); rho.erase(rho.begin());
                }
                S.push_back(s); Y.push_back(y); rho.push_back(1.0 / sy);
            }
            const double dec = F - Fn;
            x = xn;
            gx = gn;
            F = Fn;
            for (int i = 0; i < NT; i++) th[i] = base[i] + D[i] * x[i];
            if (dec < opt->ftol * std::fabs(F)) break;
        }
        int32_t e = 0;
        if ((rc = tpc_calib_status(workspace, &e, stream))) return rc;
        if (e) return TPC_ERR_DATA;
    }
#undef FCK
    for (int i = 0; i < NT; i++) th32[i] = (float)th[i];
    if (T > 0 && t_used && cudaMemcpyAsync(t_used, tsel, 4 * (size_t)T, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
        return TPC_ERR_CUDA;
    if (T > 0 && tgl_used) {
        if (tr->tgl_ext) {
            if (cudaMemcpyAsync(tgl_used, tgls, 4 * (size_t)T, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
                return TPC_ERR_CUDA;
        } else {
            k_fit_fill<<<grid, CALIB_BLOCK, 0, st>>>(tgl_used, T, __builtin_nanf(""));
        }
    }
    if (cudaMemcpyAsync(theta, th32.data(), 4 * (size_t)NT, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return TPC_ERR_CUDA;
    if (rep) {
        rep->f_start = f_start;
        rep->f_final = F;
        rep->evaluations = evals;
        rep->rounds = rounds;
        rep->tracks = ntr;
        rep->anchors = nanc;
    }
    return TPC_OK;
}

}  // extern "C"
