// tpc_refit.cu -- multi-pass Kalman refit of merged tracks (paper section
// "TPC Tracking": several features of the offline fit were brought in, among
// them multiple fit iterations; section "Tracking": the preliminary fit is
// followed by a refit of the full track).
//
// One thread per track.  Pass 1 runs from the outermost cluster inwards,
// pass 2 outwards, pass 3 inwards again; each pass restarts from the previous
// fit's state with y, z set to the first measurement (variance sigma^2, no
// correlations) and the sin(phi), tan(lambda), q/pT covariance block of the
// previous fit multiplied by refit_inflate (pass 1: the tracklet's outer-end
// fit).  The state parameters are accumulated with compensated binary32
// sums (a high and a low part), so small curvature increments are not lost
// against sin(phi) and y.  Clusters of a neighbouring sector are reached by
// rotating the local frame.  Parameters are binary32; the covariance is
// binary32, or -- with fp64_final -- binary64 during the final pass with a
// Joseph-form update and a binary64 chi2 sum.  This is the tolerance path
// (compared with a binary64 fit within 1e-4 relative), so it uses the exact
// arcsine and lets the compiler contract multiply-adds.
#include "tpc_dev.cuh"
#include "tpc_track.h"

#include <cmath>

using namespace tpc;

namespace {

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
// parameter with about twice the binary32 precision.  two_sum is Knuth's
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

template <typename CT>
__device__ __forceinline__ bool prop(float& x, float* p, float* pl, CT* c, float x2, float kb)
{
    const float dx = x2 - x;
    if (dx == 0.0f) return true;
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
    transport<CT>(c, (CT)dy_ds, (CT)(dy_dk * kb), (CT)(p[3] * dS_ds), (CT)dS, (CT)(p[3] * dS_dk * kb), (CT)(dx * kb));
    x = x2;
    acc(p[0], pl[0], dy);
    acc(p[1], pl[1], dS * p[3]);
    acc(p[2], pl[2], kdx);
#pragma unroll
    for (int i = 0; i < 3; i++) renorm(p[i], pl[i]);
    return true;
}

template <typename CT>
__device__ __forceinline__ bool rot(float& x, float* p, float* pl, CT* c, float cs, float sn, float kb)
{
    const float sp = p[2];
    const float cf = sqrtf((1.0f - sp) * (1.0f + sp));
    const float spn = sp * cs - cf * sn;
    const float cfn = cf * cs + sp * sn;
    if (!(fabsf(spn) < SNP_MAX) || !(cfn > 0.0f)) return false;
    const float k = kb * p[4];
    const CT J00 = cf / cfn, J10 = -sn * p[3] / cfn, J20 = -k * sn, J22 = cfn / cf;
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

// standard-form update (binary32 covariance)
__device__ __forceinline__ bool update(float* p, float* pl, float* c, float my, float mz, float vy, float vz,
                                       double& chi2)
{
    const float r0 = (my - p[0]) - pl[0], r1 = (mz - p[1]) - pl[1];
    const float s00 = c[0] + vy, s01 = c[1], s11 = c[2] + vz;
    const float det = s00 * s11 - s01 * s01;
    if (!(det > 0.0f)) return false;
    const float idet = 1.0f / det;
    const float i00 = s11 * idet, i01 = -s01 * idet, i11 = s00 * idet;
    chi2 += (double)(r0 * (i00 * r0 + i01 * r1) + r1 * (i01 * r0 + i11 * r1));
    float K0[5], K1[5], row0[5], row1[5];
#pragma unroll
    for (int i = 0; i < 5; i++) {
        const float c0 = c[cidx(i, 0)], c1 = c[cidx(i, 1)];
        K0[i] = c0 * i00 + c1 * i01;
        K1[i] = c0 * i01 + c1 * i11;
        row0[i] = c0;
        row1[i] = c1;
    }
#pragma unroll
    for (int i = 0; i < 5; i++) {
        acc(p[i], pl[i], K0[i] * r0 + K1[i] * r1);
        renorm(p[i], pl[i]);
    }
#pragma unroll
    for (int i = 0; i < 5; i++)
#pragma unroll
        for (int j = 0; j <= i; j++) c[CI(i, j)] -= K0[i] * row0[j] + K1[i] * row1[j];
    return true;
}

// Joseph-form update with a binary64 covariance and chi2:
// C+ = (I - K H) C (I - K H)^T + K V K^T
__device__ __forceinline__ bool update(float* p, float* pl, double* c, float my, float mz, float vy, float vz,
                                       double& chi2)
{
    const double r0 = ((double)my - p[0]) - pl[0], r1 = ((double)mz - p[1]) - pl[1];
    const double s00 = c[0] + vy, s01 = c[1], s11 = c[2] + vz;
    const double det = s00 * s11 - s01 * s01;
    if (!(det > 0.0)) return false;
    const double i00 = s11 / det, i01 = -s01 / det, i11 = s00 / det;
    chi2 += r0 * (i00 * r0 + i01 * r1) + r1 * (i01 * r0 + i11 * r1);
    double K0[5], K1[5], C[5][5];
#pragma unroll
    for (int i = 0; i < 5; i++)
#pragma unroll
        for (int j = 0; j < 5; j++) C[i][j] = c[cidx(i, j)];
#pragma unroll
    for (int i = 0; i < 5; i++) {
        K0[i] = C[i][0] * i00 + C[i][1] * i01;
        K1[i] = C[i][0] * i01 + C[i][1] * i11;
    }
#pragma unroll
    for (int i = 0; i < 5; i++) {
        acc(p[i], pl[i], (float)(K0[i] * r0 + K1[i] * r1));
        renorm(p[i], pl[i]);
    }
    // A = I - K H (only columns 0, 1 differ from I); M = A C
    double M[5][5];
#pragma unroll
    for (int i = 0; i < 5; i++)
#pragma unroll
        for (int j = 0; j < 5; j++) M[i][j] = C[i][j] - K0[i] * C[0][j] - K1[i] * C[1][j];
#pragma unroll
    for (int i = 0; i < 5; i++)
#pragma unroll
        for (int j = 0; j <= i; j++) {
            const double mat = M[i][j] - M[i][0] * K0[j] - M[i][1] * K1[j];
            c[CI(i, j)] = mat + K0[i] * vy * K0[j] + K1[i] * vz * K1[j];
        }
    return true;
}

__device__ __forceinline__ float sector_alpha_deg(int s, int ns) { return ns == 1 ? 10.0f : (float)((s % 18) * 20 + 10); }

struct RefitArgs {
    const void* frame;
    const uint8_t* sector;
    const uint8_t* row;
    const float* y;
    const float* zlin;
    const float* rowtab;
    const int32_t* ttail;
    const float* t_top;
    int ns, passes, fp64, max_tracks, prof;
    float kb, vy, vz, inflate;
    tpc_tracks out;
};

template <typename CT>
__device__ bool run_pass(const RefitArgs& R, int off, int n, bool inward, int& sec, float& x, float* p, float* pl,
                         CT* c, double& chi2, unsigned& nprop, float zref)
{
    chi2 = 0.0;
    for (int q = 0; q < n; q++) {
        const int i = inward ? n - 1 - q : q;
        const int id = R.out.clus_index[off + i];
        const int s = R.sector[id];
        if (s != sec) {
            float da = sector_alpha_deg(s, R.ns) - sector_alpha_deg(sec, R.ns);
            if (da > 180.0f) da -= 360.0f;
            if (da <= -180.0f) da += 360.0f;
            float sn, cs;
            if (da == 20.0f) { cs = COS20; sn = SIN20; }
            else if (da == -20.0f) { cs = COS20; sn = -SIN20; }
            else sincospif(da / 180.0f, &sn, &cs);
            if (!rot<CT>(x, p, pl, c, cs, sn, R.kb)) return false;
            sec = s;
        }
        if (!prop<CT>(x, p, pl, c, R.rowtab[R.row[id] * ROWTAB], R.kb)) return false;
        nprop++;
        const float my = R.y[id], mz = R.zlin[id] - zref;
        if (q == 0) {
            // restart: y, z from the measurement; angles and curvature keep the
            // previous covariance block times refit_inflate
            p[0] = my;
            p[1] = mz;
            pl[0] = 0.0f;
            pl[1] = 0.0f;
            c[0] = (CT)R.vy;
            c[1] = (CT)0;
            c[2] = (CT)R.vz;
#pragma unroll
            for (int a = 2; a < 5; a++) {
                c[CI(a, 0)] = (CT)0;
                c[CI(a, 1)] = (CT)0;
#pragma unroll
                for (int b = 2; b <= a; b++) c[CI(a, b)] *= (CT)R.inflate;
            }
        } else if (!update(p, pl, c, my, mz, R.vy, R.vz, chi2)) {
            return false;
        }
    }
    return true;
}

__global__ void __launch_bounds__(128) k_refit(RefitArgs R)
{
    Frame* f = static_cast<Frame*>(const_cast<void*>(R.frame));
    if (f->err) return;
    unsigned nprop = 0;
    const int T = min(f->n_tracks, R.max_tracks);
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < T; r += gridDim.x * blockDim.x) {
        const int off = R.out.clus_offset[r];
        const int n = R.out.nclus[r];
        const float* ts = R.t_top + (int64_t)R.ttail[r] * NST;
        float x = ts[0];
        float p[5], pl[5] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
        float c[15];
        // z relative to the first cluster of the track: same-track z values
        // subtract exactly and the binary32 state keeps small magnitudes
        const float zref = R.zlin[R.out.clus_index[off]];
#pragma unroll
        for (int k = 0; k < 5; k++) p[k] = ts[1 + k];
        p[1] = p[1] - zref;
#pragma unroll
        for (int k = 0; k < 15; k++) c[k] = ts[6 + k];
        int sec = R.sector[R.out.clus_index[off + n - 1]];
        double chi2 = 0.0;
        bool ok = true;
        const int nfloat = R.fp64 ? R.passes - 1 : R.passes;
        for (int pass = 0; pass < nfloat && ok; pass++) ok = run_pass<float>(R, off, n, (pass % 2) == 0, sec, x, p, pl, c, chi2, nprop, zref);
        double c64[15];
        if (R.fp64 && ok) {
#pragma unroll
            for (int k = 0; k < 15; k++) c64[k] = c[k];
            ok = run_pass<double>(R, off, n, ((R.passes - 1) % 2) == 0, sec, x, p, pl, c64, chi2, nprop, zref);
#pragma unroll
            for (int k = 0; k < 15; k++) c[k] = (float)c64[k];
        }
#pragma unroll
        for (int k = 0; k < 5; k++) p[k] = p[k] + pl[k];
        p[1] = p[1] + zref;
        R.out.sector[r] = R.sector[R.out.clus_index[off]];
        R.out.x[r] = x;
#pragma unroll
        for (int k = 0; k < 5; k++) R.out.param[5 * r + k] = p[k];
#pragma unroll
        for (int k = 0; k < 15; k++) R.out.cov[15 * (int64_t)r + k] = c[k];
        R.out.chi2[r] = (float)chi2;
        R.out.ndf[r] = 2 * n - 5;
        R.out.status[r] = ok ? 0 : 1;
        if (R.fp64) {
#pragma unroll
            for (int k = 0; k < 15; k++) R.out.cov64[15 * (int64_t)r + k] = c64[k];
            R.out.chi2_64[r] = chi2;
        }
    }
    if (R.prof) atomicAdd(&f->w_refit_prop, (unsigned long long)nprop);
}

}  // namespace

int tpc_launch_refit(const tpc_params* p, const tpc_geometry* g, float bz, const tpc_clusters* cl,
                     const float* zlin, const float* rowtab, const void* frame, const int32_t* ttail,
                     const float* t_top, tpc_tracks* out, int max_tracks, cudaStream_t st)
{
    RefitArgs R;
    R.frame = frame;
    R.sector = cl->sector;
    R.row = cl->row;
    R.y = cl->y;
    R.zlin = zlin;
    R.rowtab = rowtab;
    R.ttail = ttail;
    R.t_top = t_top;
    R.ns = g->n_sectors;
    R.passes = p->refit_passes;
    R.fp64 = p->fp64_final;
    R.max_tracks = max_tracks;
    R.prof = p->profile;
    volatile float kb = KB_C * bz;
    volatile float vy = p->sigma_y * p->sigma_y;
    volatile float vz = p->sigma_z * p->sigma_z;
    R.kb = kb;
    R.vy = vy;
    R.vz = vz;
    R.inflate = p->refit_inflate;
    R.out = *out;
    const int64_t want = (max_tracks + 127) / 128;
    const int grid = (int)(want < 1 ? 1 : (want > 148 * 16 ? 148 * 16 : want));
    k_refit<<<grid, 128, 0, st>>>(R);
    return cudaGetLastError() == cudaSuccess ? TPC_OK : TPC_ERR_CUDA;
}
