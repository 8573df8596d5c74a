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
// arcsine, lets the compiler contract multiply-adds, and is built with the
// approximate division and square root (a few ulp).
#include "tpc_dev.cuh"
#include "tpc_fit.cuh"
#include "tpc_track.h"

#include <cmath>
#include <type_traits>

using namespace tpc;
using namespace tpc::fit;

namespace {

template <typename CT>
__device__ __forceinline__ bool prop(float& x, float* p, float* pl, CT* c, float x2, float kb)
{
    if (x2 - x == 0.0f) return true;
    HelixJac J;
    if (!helix_step(x, p, pl, x2, kb, J)) return false;
    transport<CT>(c, (CT)J.a, (CT)J.b, (CT)J.c, (CT)J.d, (CT)J.e, (CT)J.f);
    return true;
}

template <typename CT>
__device__ __forceinline__ bool rot(float& x, float* p, float* pl, CT* c, float cs, float sn, float kb)
{
    RotJac R;
    if (!rotate_step(x, p, pl, cs, sn, kb, R)) return false;
    rotate_cov<CT>(c, R);
    return true;
}

// chi2 of a binary32 pass: a compensated binary32 sum (TwoSum), far inside
// the 1e-3 the pass's chi2 is held to, without a binary64 add per step (the
// FP64 pipe of this GPU is narrow)
struct Chi2Sum {
    float s, e;
    __device__ __forceinline__ void add(float v)
    {
        const float t = s + v, bp = t - s;
        e += (s - (t - bp)) + (v - bp);
        s = t;
    }
};
__device__ __forceinline__ double chi2_value(const Chi2Sum& a) { return (double)a.s + (double)a.e; }
__device__ __forceinline__ double chi2_value(double a) { return a; }

// standard-form update (binary32 covariance)
__device__ __forceinline__ bool update(float* p, float* pl, float* c, float my, float mz, float vy, float vz,
                                       Chi2Sum& chi2)
{
    const float r0 = (my - p[0]) - pl[0], r1 = (mz - p[1]) - pl[1];
    const float s00 = c[0] + vy, s01 = c[1], s11 = c[2] + vz;
    const float det = s00 * s11 - s01 * s01;
    if (!(det > 0.0f)) return false;
    const float idet = 1.0f / det;
    const float i00 = s11 * idet, i01 = -s01 * idet, i11 = s00 * idet;
    chi2.add(r0 * (i00 * r0 + i01 * r1) + r1 * (i01 * r0 + i11 * r1));
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

// standard-form update (binary32 covariance), chi2 summed in binary64
__device__ __forceinline__ bool update(float* p, float* pl, float* c, float my, float mz, float vy, float vz,
                                       double& chi2)
{
    Chi2Sum d{0.0f, 0.0f};
    if (!update(p, pl, c, my, mz, vy, vz, d)) return false;
    chi2 += (double)d.s;
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
    const double idet = 1.0 / det;       // one binary64 division (the FP64 pipe is the bound here)
    const double i00 = s11 * idet, i01 = -s01 * idet, i11 = s00 * idet;
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
    // A = I - K H (only columns 0, 1 differ from I); M = A C, of which the
    // lower triangle and columns 0, 1 are used (16 entries)
    double M[5][5];
#pragma unroll
    for (int i = 0; i < 5; i++)
#pragma unroll
        for (int j = 0; j < 5; j++)
            if (j <= i || j < 2) M[i][j] = C[i][j] - K0[i] * C[0][j] - K1[i] * C[1][j];
    // C+ = M A^T + K V K^T, V = diag(vy, vz)
    double VK0[5], VK1[5];
#pragma unroll
    for (int j = 0; j < 5; j++) {
        VK0[j] = vy * K0[j];
        VK1[j] = vz * K1[j];
    }
#pragma unroll
    for (int i = 0; i < 5; i++)
#pragma unroll
        for (int j = 0; j <= i; j++)
            c[CI(i, j)] = M[i][j] - M[i][0] * K0[j] - M[i][1] * K1[j] + K0[i] * VK0[j] + K1[i] * VK1[j];
    return true;
}


// |q/pT| (c/GeV) from which the binary64 mode 2 treats a track as a looper
// (pT below 0.2 GeV/c)
constexpr float LOOPER_QPT = 5.0f;

struct RefitArgs {
    const void* frame;
    const float4* tcl;      // track clusters in track order: y, z, row x, sector (int bits)
    const int32_t* order;   // tracks by decreasing cluster count (nullable)
    const int32_t* ttail;
    const float* t_top;
    int ns, nr, passes, fp64, max_tracks, prof;
    float kb, vy, vz, inflate;
    tpc_tracks out;
};

template <typename CT, typename ACC>
__device__ __forceinline__ bool run_steps(const RefitArgs& R, int off, int n, bool inward, int& sec, float& x, float* p,
                                          float* pl, CT* c, ACC& chi2, unsigned& nprop, float zref)
{
    for (int q = 0; q < n; q++) {
        const int i = inward ? n - 1 - q : q;
        const float4 cl = R.tcl[off + i];
        const int s = __float_as_int(cl.w);
        if (s != sec) {
            float sn, cs;
            frame_rotation(sec, s, R.ns, cs, sn);
            if (!rot<CT>(x, p, pl, c, cs, sn, R.kb)) return false;
            sec = s;
        }
        if (!prop<CT>(x, p, pl, c, cl.z, R.kb)) return false;
        nprop++;
        const float my = cl.x, mz = cl.y - zref;
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

// ACC: the chi2 accumulator -- a compensated binary32 sum for the binary32
// passes, binary64 for the final pass of the binary64 modes
template <typename CT, typename ACC = typename std::conditional<std::is_same<CT, float>::value, Chi2Sum, double>::type>
__device__ bool run_pass(const RefitArgs& R, int off, int n, bool inward, int& sec, float& x, float* p, float* pl,
                         CT* c, double& chi2, unsigned& nprop, float zref)
{
    ACC acc{};
    const bool ok = run_steps<CT>(R, off, n, inward, sec, x, p, pl, c, acc, nprop, zref);
    chi2 = chi2_value(acc);
    return ok;
}

// FP64: the final pass in binary64 (a separate instance, so that the
// binary32-only refit is not held to the binary64 pass's register count)
template <bool FP64>
__global__ void __launch_bounds__(128) k_refit(RefitArgs R)
{
    Frame* f = static_cast<Frame*>(const_cast<void*>(R.frame));
    if (f->err) return;
    unsigned nprop = 0;
    const int T = min(f->n_tracks, R.max_tracks);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < T; i += gridDim.x * blockDim.x) {
        const int r = R.order ? R.order[i] : i;       // longest tracks first: similar lengths share a warp
        const int off = R.out.clus_offset[r];
        const int n = R.out.nclus[r];
        const float* ts = R.t_top + (int64_t)R.ttail[r] * NST;
        float x = ts[0];
        float p[5], pl[5] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
        float c[15];
        // z relative to the first cluster of the track: same-track z values
        // subtract exactly and the binary32 state keeps small magnitudes
        const float zref = R.tcl[off].y;
#pragma unroll
        for (int k = 0; k < 5; k++) p[k] = ts[1 + k];
        p[1] = p[1] - zref;
#pragma unroll
        for (int k = 0; k < 15; k++) c[k] = ts[6 + k];
        int sec = __float_as_int(R.tcl[off + n - 1].w);
        double chi2 = 0.0;
        bool ok = true;
        const int nfloat = FP64 ? R.passes - 1 : R.passes;
        for (int pass = 0; pass < nfloat && ok; pass++) ok = run_pass<float>(R, off, n, (pass % 2) == 0, sec, x, p, pl, c, chi2, nprop, zref);
        double c64[15];
        if (FP64) {
            // mode 1: the binary64 Joseph update for every track; mode 2: for
            // long looping low-pT tracks only (|q/pT| >= LOOPER_QPT after the
            // earlier passes, or more clusters than pad rows), the binary32
            // update for the others; the final pass's chi2 in binary64 always
            const bool inward_last = ((R.passes - 1) % 2) == 0;
            const bool joseph = R.fp64 == 1 || fabsf(p[4] + pl[4]) >= LOOPER_QPT || n > R.nr;
            if (joseph) {
#pragma unroll
                for (int k = 0; k < 15; k++) c64[k] = c[k];
                if (ok) ok = run_pass<double>(R, off, n, inward_last, sec, x, p, pl, c64, chi2, nprop, zref);
#pragma unroll
                for (int k = 0; k < 15; k++) c[k] = (float)c64[k];
            } else {
                if (ok) ok = run_pass<float, double>(R, off, n, inward_last, sec, x, p, pl, c, chi2, nprop, zref);
#pragma unroll
                for (int k = 0; k < 15; k++) c64[k] = c[k];
            }
        }
#pragma unroll
        for (int k = 0; k < 5; k++) p[k] = p[k] + pl[k];
        p[1] = p[1] + zref;
        R.out.sector[r] = __float_as_int(R.tcl[off].w);
        R.out.x[r] = x;
#pragma unroll
        for (int k = 0; k < 5; k++) R.out.param[5 * r + k] = p[k];
#pragma unroll
        for (int k = 0; k < 15; k++) R.out.cov[15 * (int64_t)r + k] = c[k];
        R.out.chi2[r] = (float)chi2;
        R.out.ndf[r] = 2 * n - 5;
        R.out.status[r] = ok ? 0 : 1;
        if (FP64) {
#pragma unroll
            for (int k = 0; k < 15; k++) R.out.cov64[15 * (int64_t)r + k] = c64[k];
            R.out.chi2_64[r] = chi2;
        }
    }
    if (R.prof) {
        // one atomic per warp (every thread of the block gets here)
        nprop = __reduce_add_sync(0xffffffffu, nprop);
        if ((threadIdx.x & 31) == 0) atomicAdd(&f->w_refit_prop, (unsigned long long)nprop);
    }
}

}  // namespace

int tpc_launch_refit(const tpc_params* p, const tpc_geometry* g, float bz, const float4* tcl, const int32_t* order,
                     const void* frame, const int32_t* ttail, const float* t_top, tpc_tracks* out, int max_tracks,
                     cudaStream_t st)
{
    RefitArgs R;
    R.frame = frame;
    R.tcl = tcl;
    R.order = order;
    R.ttail = ttail;
    R.t_top = t_top;
    R.ns = g->n_sectors;
    R.nr = g->n_rows;
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
    if (R.fp64) k_refit<true><<<grid, 128, 0, st>>>(R);
    else k_refit<false><<<grid, 128, 0, st>>>(R);
    return cudaGetLastError() == cudaSuccess ? TPC_OK : TPC_ERR_CUDA;
}
