// Entropy coder of the cluster compression: rANS of byte symbols with one
// static 12-bit table per stream, in independent chunks (paper, section
// "TPC Data Compression", step 4; the format is stated in tpc_compress.h).
//
// Kernels: k_rans_hist (block histograms in shared memory, one global add
// per bin and block), k_rans_table (one block of 256 threads: the
// largest-remainder normalisation), k_rans_chunks (one thread per chunk: the
// chunk is coded last symbol first into its own scratch slot, bytes written
// from the slot's end backward, so they come out in decode order; the
// division by the symbol frequency by a magic multiplier), a scan of the
// chunk sizes and k_rans_copy (one block per chunk) packing the chunks back
// to back.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>

#include "tpc_compress.h"
#include "tpc_track.h"

namespace {

constexpr uint32_t RANS_L = 1u << 23;
constexpr int RANS_BITS = 12;
constexpr uint32_t RANS_M = 1u << RANS_BITS;

struct RansLayout {
    size_t hist, freq, cum, len, off, err, scratch, total;
};

size_t al(size_t x) { return (x + 255) & ~(size_t)255; }

RansLayout rans_layout(int64_t n, int32_t chunk)
{
    const int64_t nch = n > 0 ? (n + chunk - 1) / chunk : 0;
    RansLayout L;
    size_t o = 0;
    L.hist = o; o = al(o + 4 * 256);
    L.freq = o; o = al(o + 4 * 256);
    L.cum = o; o = al(o + 4 * 257);
    L.len = o; o = al(o + 4 * (size_t)std::max<int64_t>(nch, 1));
    L.off = o; o = al(o + 8 * (size_t)(nch + 1));
    L.err = o; o = al(o + 4);
    L.scratch = o; o = al(o + (size_t)std::max<int64_t>(nch, 1) * (4 + 2 * (size_t)chunk));
    L.total = o;
    return L;
}

template <typename T>
T* at(void* ws, size_t off) { return reinterpret_cast<T*>(static_cast<char*>(ws) + off); }

__global__ void k_rans_hist(const uint8_t* __restrict__ sym, int64_t n, uint32_t* __restrict__ hist)
{
    __shared__ uint32_t h[256];
    for (int s = threadIdx.x; s < 256; s += blockDim.x) h[s] = 0;
    __syncthreads();
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(&h[sym[i]], 1u);
    __syncthreads();
    for (int s = threadIdx.x; s < 256; s += blockDim.x)
        if (h[s]) atomicAdd(&hist[s], h[s]);
}

// One block of 256 threads, thread s for symbol s: the table (largest
// remainders) and its cumulative sums.  The missing units go to the present
// symbols ranked first by (remainder descending, symbol ascending) -- the
// order in which repeatedly taking the largest remainder, ties to the
// smaller symbol, hands them out; the surplus after raising absent-looking
// present symbols to 1 is taken back one unit at a time from the largest
// frequency above 1 (ties to the smaller symbol), each by a block argmax.
constexpr int TABLE_THREADS = 256;

__global__ void __launch_bounds__(TABLE_THREADS) k_rans_table(const uint32_t* __restrict__ hist,
                                                              uint32_t* __restrict__ freq,
                                                              uint32_t* __restrict__ cum, int* __restrict__ err)
{
    __shared__ unsigned long long rem_sh[256];
    __shared__ uint32_t f_sh[256];
    __shared__ unsigned long long red64[TABLE_THREADS / 32];
    __shared__ uint32_t red32[TABLE_THREADS / 32];
    const int s = threadIdx.x, lane = s & 31, w = s >> 5;
    const uint32_t h = hist[s];
    // total
    unsigned long long t = h;
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (lane == 0) red64[w] = t;
    __syncthreads();
    unsigned long long total = 0;
    for (int k = 0; k < TABLE_THREADS / 32; k++) total += red64[k];
    if (total == 0) {
        freq[s] = 0;
        cum[s] = 0;
        if (s == 0) cum[256] = 0;
        return;
    }
    const unsigned long long m = (unsigned long long)h * RANS_M;
    uint32_t f = (uint32_t)(m / total);
    const unsigned long long rem = m % total;
    rem_sh[s] = rem;
    uint32_t fs = f;
    for (int o = 16; o > 0; o >>= 1) fs += __shfl_xor_sync(0xffffffffu, fs, o);
    __syncthreads();                       // red64 read by every thread above
    if (lane == 0) red32[w] = fs;
    __syncthreads();
    uint32_t sum = 0;
    for (int k = 0; k < TABLE_THREADS / 32; k++) sum += red32[k];
    const uint32_t missing = RANS_M - sum;  // fewer than the present symbols
    if (h > 0) {
        uint32_t rank = 0;
        for (int q = 0; q < 256; q++) {
            if (hist[q] == 0) continue;
            const unsigned long long rq = rem_sh[q];
            rank += (rq > rem || (rq == rem && q < s));
        }
        if (rank < missing) f++;
        if (f == 0) f = 1;
    }
    f_sh[s] = f;
    __syncthreads();
    // the sum after the raises, then the surplus taken back
    uint32_t fs2 = f;
    for (int o = 16; o > 0; o >>= 1) fs2 += __shfl_xor_sync(0xffffffffu, fs2, o);
    if (lane == 0) red32[w] = fs2;
    __syncthreads();
    uint32_t sum2 = 0;
    for (int k = 0; k < TABLE_THREADS / 32; k++) sum2 += red32[k];
    __syncthreads();
    for (uint32_t it = 0; sum2 > RANS_M && it < 256; it++, sum2--) {
        // argmax of (freq, -symbol) over freq > 1
        const uint32_t fv = f_sh[s];
        uint32_t key = fv > 1 ? (fv << 8) | (uint32_t)(255 - s) : 0u;
        for (int o = 16; o > 0; o >>= 1) key = max(key, __shfl_xor_sync(0xffffffffu, key, o));
        if (lane == 0) red32[w] = key;
        __syncthreads();
        uint32_t best = 0;
        for (int k = 0; k < TABLE_THREADS / 32; k++) best = max(best, red32[k]);
        if (best == 0) {
            if (s == 0) *err = 1;
            return;
        }
        if (s == 255 - (int)(best & 0xFF)) f_sh[s] = fv - 1;
        __syncthreads();
    }
    if (sum2 > RANS_M) {
        if (s == 0) *err = 1;
        return;
    }
    // cumulative sums: an exclusive scan over the 256 frequencies
    const uint32_t fv = f_sh[s];
    freq[s] = fv;
    uint32_t inc = fv;
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) red32[w] = inc;
    __syncthreads();
    uint32_t base = 0;
    for (int k = 0; k < w; k++) base += red32[k];
    cum[s] = base + inc - fv;
    if (s == 255) cum[256] = base + inc;
}

// One thread per chunk; slot c holds 4 + 2 chunk bytes, filled from its end.
// Codes the chunks of blocks bi, bi + nb, ... (blockDim.x chunks per block)
// of one stream.
__device__ void code_chunks(const uint8_t* __restrict__ sym, int64_t n, int32_t chunk,
                            const uint32_t* __restrict__ freq_g, const uint32_t* __restrict__ cum_g,
                            uint8_t* __restrict__ scratch, int32_t* __restrict__ len, const int* __restrict__ err,
                            int64_t bi, int64_t nb)
{
    // x / f by multiplication (Granlund and Montgomery, division by invariant
    // integers): l = ceil(log2 f), m = ceil(2^(32 + l) / f) <= 2^33; for x <
    // 2^32, x / f = (x m) >> (32 + l) exactly.  With m = 2^32 m_hi + m_lo and
    // x < 2^31: (x m) >> 32 = umulhi(x, m_lo) + x m_hi < 2^32, so q =
    // (umulhi(x, m_lo) + x m_hi) >> l in 32-bit arithmetic.  Per symbol one
    // 16-byte entry: f | l << 16 | m_hi << 24, the cumulative frequency, m_lo,
    // the renormalisation bound.
    __shared__ uint4 tab[256];
    for (int s = threadIdx.x; s < 256; s += blockDim.x) {
        const uint32_t f = freq_g[s];
        uint32_t l = 0;
        while (l < 12 && (1u << l) < f) l++;
        const unsigned long long m = f ? (((1ull << (32 + l)) - 1ull) / f + 1ull) : 0ull;
        tab[s] = make_uint4(f | (l << 16) | ((uint32_t)(m >> 32) << 24), cum_g[s], (uint32_t)m,
                            ((RANS_L >> RANS_BITS) << 8) * f);
    }
    __syncthreads();
    if (*err) return;
    const int64_t nch = (n + chunk - 1) / chunk;
    const size_t cap = 4 + 2 * (size_t)chunk;
    for (int64_t c = bi * (int64_t)blockDim.x + threadIdx.x; c < nch; c += nb * blockDim.x) {
        const int64_t a = c * chunk;
        const int64_t m = min((int64_t)chunk, n - a);
        uint8_t* base = scratch + (size_t)c * cap;
        size_t p = cap;
        uint32_t x = RANS_L;
        // the entry of the next symbol is loaded a step ahead: the state chain
        // does not wait for the table
        uint4 en = tab[sym[a + m - 1]];
        for (int64_t i = a + m - 1; i >= a; i--) {
            const uint4 e = en;
            if (i > a) en = tab[sym[i - 1]];
            while (x >= e.w) {
                base[--p] = (uint8_t)(x & 0xFF);
                x >>= 8;
            }
            const uint32_t f = e.x & 0xFFFFu, l = (e.x >> 16) & 0xFFu, mh = e.x >> 24;
            const uint32_t q = (__umulhi(x, e.z) + x * mh) >> l;
            x = (q << RANS_BITS) + (x - q * f) + e.y;
        }
        base[--p] = (uint8_t)(x & 0xFF);
        base[--p] = (uint8_t)((x >> 8) & 0xFF);
        base[--p] = (uint8_t)((x >> 16) & 0xFF);
        base[--p] = (uint8_t)(x >> 24);
        len[c] = (int32_t)(cap - p);
    }
}

__global__ void __launch_bounds__(128) k_rans_chunks(const uint8_t* __restrict__ sym, int64_t n, int32_t chunk,
                                                     const uint32_t* __restrict__ freq_g,
                                                     const uint32_t* __restrict__ cum_g,
                                                     uint8_t* __restrict__ scratch, int32_t* __restrict__ len,
                                                     const int* __restrict__ err)
{
    code_chunks(sym, n, chunk, freq_g, cum_g, scratch, len, err, blockIdx.x, gridDim.x);
}

// Several streams in one launch: the blocks [block0, block0 + blocks) of job
// j code stream j's chunks (each block loads one stream's table).
struct ChunkJob {
    const uint8_t* sym;
    int64_t n;
    const uint32_t* freq;
    const uint32_t* cum;
    uint8_t* scratch;
    int32_t* len;
    const int* err;
    int32_t block0, blocks;
};
constexpr int MAX_CHUNK_JOBS = 16;
struct ChunkJobs {
    ChunkJob j[MAX_CHUNK_JOBS];
    int32_t njobs, chunk;
};

__global__ void __launch_bounds__(128) k_rans_chunks_multi(const ChunkJobs J)
{
    int k = 0;
    while (k + 1 < J.njobs && (int)blockIdx.x >= J.j[k + 1].block0) k++;
    const ChunkJob& q = J.j[k];
    const int64_t bi = (int64_t)blockIdx.x - q.block0;
    if (bi < 0 || bi >= q.blocks) return;
    code_chunks(q.sym, q.n, J.chunk, q.freq, q.cum, q.scratch, q.len, q.err, bi, q.blocks);
}

// one block: exclusive scan of the chunk sizes (off[nch] = total)
__global__ void k_rans_scan(const int32_t* __restrict__ len, int64_t nch, long long* __restrict__ off,
                            const int* __restrict__ err)
{
    __shared__ long long part[1024];
    if (*err) return;
    const int64_t per = (nch + blockDim.x - 1) / blockDim.x;
    const int64_t a = threadIdx.x * per, b = min(nch, a + per);
    long long s = 0;
    for (int64_t i = a; i < b; i++) s += len[i];
    part[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        long long run = 0;
        for (int t = 0; t < (int)blockDim.x; t++) {
            const long long v = part[t];
            part[t] = run;
            run += v;
        }
        off[nch] = run;
    }
    __syncthreads();
    long long o = part[threadIdx.x];
    for (int64_t i = a; i < b; i++) {
        off[i] = o;
        o += len[i];
    }
}

// one block per chunk: its bytes to their place in out
__global__ void k_rans_copy(const uint8_t* __restrict__ scratch, int32_t chunk, int64_t nch,
                            const int32_t* __restrict__ len, const long long* __restrict__ off,
                            uint8_t* __restrict__ out, int64_t out_cap, int32_t* __restrict__ chunk_bytes,
                            const int* __restrict__ err)
{
    if (*err) return;
    const size_t cap = 4 + 2 * (size_t)chunk;
    for (int64_t c = blockIdx.x; c < nch; c += gridDim.x) {
        const int32_t l = len[c];
        const uint8_t* src = scratch + (size_t)c * cap + (cap - (size_t)l);
        const long long o = off[c];
        if (o + l > out_cap) continue;          // the host bound makes this unreachable
        for (int32_t k = threadIdx.x; k < l; k += blockDim.x) out[o + k] = src[k];
        if (threadIdx.x == 0) chunk_bytes[c] = l;
    }
}

int grid_cap(int64_t work, int block)
{
    const int64_t g = (work + block - 1) / block;
    return (int)std::max<int64_t>(1, std::min<int64_t>(g, 148 * 16));
}

}  // namespace

extern "C" int tpc_rans_workspace_size(int64_t n, int32_t chunk, size_t* bytes)
{
    if (!bytes || n < 0 || n >= TPC_RANS_MAX_SYMBOLS || chunk < 1 || chunk > TPC_RANS_MAX_CHUNK) return TPC_ERR_ARG;
    *bytes = rans_layout(n, chunk).total;
    return TPC_OK;
}

extern "C" int tpc_rans_max_bytes(int64_t n, int32_t chunk, int64_t* bytes)
{
    if (!bytes || n < 0 || n >= TPC_RANS_MAX_SYMBOLS || chunk < 1 || chunk > TPC_RANS_MAX_CHUNK) return TPC_ERR_ARG;
    const int64_t nch = n > 0 ? (n + chunk - 1) / chunk : 0;
    *bytes = 4 * nch + 2 * n;
    return TPC_OK;
}

extern "C" int tpc_rans_encode(const uint8_t* sym, int64_t n, int32_t chunk, void* workspace, size_t ws_bytes,
                               uint32_t* freq, int32_t* chunk_bytes, uint8_t* out, int64_t out_cap, int64_t* total,
                               void* stream)
{
    size_t need = 0;
    int rc = tpc_rans_workspace_size(n, chunk, &need);
    if (rc) return rc;
    int64_t maxb = 0;
    tpc_rans_max_bytes(n, chunk, &maxb);
    if (!workspace || ws_bytes < need || !freq || (n > 0 && (!sym || !chunk_bytes || !out || out_cap < maxb)))
        return TPC_ERR_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const RansLayout L = rans_layout(n, chunk);
    const int64_t nch = n > 0 ? (n + chunk - 1) / chunk : 0;
    uint32_t* hist = at<uint32_t>(workspace, L.hist);
    uint32_t* cum = at<uint32_t>(workspace, L.cum);
    int32_t* len = at<int32_t>(workspace, L.len);
    long long* off = at<long long>(workspace, L.off);
    int* err = at<int>(workspace, L.err);
#define CK(x) do { if ((x) != cudaSuccess) return TPC_ERR_CUDA; } while (0)
    CK(cudaMemsetAsync(hist, 0, 4 * 256, st));
    CK(cudaMemsetAsync(err, 0, 4, st));
    k_rans_hist<<<grid_cap(n, 256), 256, 0, st>>>(sym, n, hist);
    k_rans_table<<<1, TABLE_THREADS, 0, st>>>(hist, freq, cum, err);
    if (nch > 0) {
        k_rans_chunks<<<grid_cap(nch, 128), 128, 0, st>>>(sym, n, chunk, freq, cum, at<uint8_t>(workspace, L.scratch),
                                                          len, err);
        k_rans_scan<<<1, 1024, 0, st>>>(len, nch, off, err);
        k_rans_copy<<<(int)std::min<int64_t>(nch, 148 * 32), 128, 0, st>>>(at<uint8_t>(workspace, L.scratch), chunk,
                                                                           nch, len, off, out, out_cap, chunk_bytes,
                                                                           err);
    }
    CK(cudaGetLastError());
    if (total) {
        long long t = 0;
        int e = 0;
        if (nch > 0) CK(cudaMemcpyAsync(&t, off + nch, sizeof(t), cudaMemcpyDeviceToHost, st));
        CK(cudaMemcpyAsync(&e, err, sizeof(e), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        if (e) return TPC_ERR_ARG;
        *total = t;
    }
#undef CK
    return TPC_OK;
}

// ---------------------------------------------------------------------------
// The compressed cluster format (tpc_compress.h): integer fields, per-track
// run streams, per-plane streams of the other clusters, then each stream
// symbolised (escapes) and coded into its container.
//
// Kernels: k_cq (quantisation, plane counts of the other clusters, checks),
// k_ct_count (per track: clusters, runs), multi-block scans of the per-track
// and per-plane counts (k_tile_sum, k_scan1, k_tile_apply), k_ct_fill (one
// warp per track writes its values at the scanned offsets), k_cu_scatter /
// k_cu_plane (the other clusters by plane, then one block per plane ranks
// them by (qt, qy, index) and writes the plane's values), k_sym_count /
// k_sym_write (escape split), the coder's histogram and table per stream,
// k_rans_chunks_multi (the chunks of all streams in one launch: each chunk is
// a serial chain, so the streams' chains run side by side), k_rans_scan /
// k_rans_copy per stream, k_pack_head / k_pack_copy (the container).
// ---------------------------------------------------------------------------
namespace {

enum { CS_NT, CS_HS, CS_HR, CS_HY, CS_HT, CS_DS, CS_DR, CS_RY, CS_RT, CS_UN, CS_UT, CS_UY, CS_N };
static_assert(CS_N == TPC_CMP_N_STREAMS, "stream count");
constexpr int CU_SMEM = 4096;           // keys of a plane's other clusters held in shared memory

__device__ __forceinline__ uint32_t zz32(long long v)
{
    return v >= 0 ? (uint32_t)(2 * v) : (uint32_t)(-2 * v - 1);
}

struct CmpArgs {
    int64_t n;
    int ns, nr, np, T;
    int64_t na;
    const uint8_t* sector;
    const uint8_t* row;
    const float* y;
    const float* zt;
    const int32_t* off;
    const int32_t* clus;
    const int32_t* assign;
    float sy, st;                 // 2^ey, 2^et
    int4* rec;                    // [n] per cluster: qy, qt, sector | row << 8, 0 (one gather per cluster)
    uint32_t* tcnt;               // [4][T + 1]: has clusters, runs, clusters - 1, clusters - runs (then scanned)
    uint32_t* pcnt;               // [np + 1] other clusters per plane (then scanned)
    uint32_t* pfill;              // [np] fill cursors
    int32_t* uord;                // [n] other clusters by plane (arbitrary order inside)
    int32_t* usort;               // [n] sorted inside each plane
    uint32_t* vals;               // stream values, stream s from vbase[s]
    int64_t vbase[CS_N + 1];
    int* err;
};

__global__ void k_cq(CmpArgs A)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < A.n; i += (int64_t)gridDim.x * blockDim.x) {
        const int s = A.sector[i], r = A.row[i];
        if (s >= A.ns || r >= A.nr) {
            atomicExch(A.err, 1);
            continue;
        }
        A.rec[i] = make_int4(__float2int_rn(A.y[i] * A.sy), __float2int_rn(A.zt[i] * A.st), s | (r << 8), 0);
        if (A.assign[i] < 0) atomicAdd(&A.pcnt[s * A.nr + r], 1u);
    }
}

// per track: [0] 1 if it has clusters, [1] runs, [2] clusters - 1, [3] clusters - runs
__global__ void k_ct_count(CmpArgs A)
{
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < A.T; t += gridDim.x * blockDim.x) {
        const int a = A.off[t], b = A.off[t + 1];
        uint32_t runs = 0;
        if (a < 0 || b < a || (int64_t)b > A.na) {
            atomicExch(A.err, 1);
        } else {
            int sec = -1;
            for (int k = a; k < b; k++) {
                const int c = A.clus[k];
                if (c < 0 || (int64_t)c >= A.n) {
                    atomicExch(A.err, 1);
                    break;
                }
                const int s = A.sector[c];
                runs += (k == a || s != sec);
                sec = s;
            }
        }
        const uint32_t m = (a >= 0 && b >= a) ? (uint32_t)(b - a) : 0u;
        const int64_t T1 = (int64_t)A.T + 1;
        A.tcnt[t] = m > 0;
        A.tcnt[T1 + t] = runs;
        A.tcnt[2 * T1 + t] = m > 0 ? m - 1 : 0;
        A.tcnt[3 * T1 + t] = m >= runs ? m - runs : 0;
    }
}

// one block: in[0..n) -> exclusive sums in place, in[n] = total
__global__ void __launch_bounds__(1024) k_scan1(uint32_t* a, int64_t n)
{
    __shared__ uint32_t part[1024];
    const int64_t per = (n + blockDim.x - 1) / blockDim.x;
    const int64_t lo = threadIdx.x * per, hi = min(n, lo + per);
    uint32_t s = 0;
    for (int64_t i = lo; i < hi; i++) s += a[i];
    part[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t run = 0;
        for (int t = 0; t < (int)blockDim.x; t++) {
            const uint32_t v = part[t];
            part[t] = run;
            run += v;
        }
        a[n] = run;
    }
    __syncthreads();
    uint32_t o = part[threadIdx.x];
    for (int64_t i = lo; i < hi; i++) {
        const uint32_t v = a[i];
        a[i] = o;
        o += v;
    }
}

// prediction of a run's next value from its previous one or two clusters
__device__ __forceinline__ long long predict(int nprev, long long v0, int r0, long long v1, int r1, int r)
{
    if (nprev < 2 || r1 == r0) return v1;
    return v1 + ((v1 - v0) * (long long)(r - r1)) / (long long)(r1 - r0);
}

// One warp per track: lane j takes the clusters a + 32 i + j.  A cluster
// starts a run when it is the track's first or its sector differs from the
// previous cluster's; its residuals use the previous two clusters (a line
// when neither the cluster nor the previous one starts a run).  Positions in
// the head and residual streams are the counts of run starts and of the
// other clusters before it (ballots), so each warp writes its track's values
// contiguously.  The previous chunk's last two clusters carry over in
// registers.
__global__ void k_ct_fill(CmpArgs A)
{
    if (*A.err) return;
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    const int64_t T1 = (int64_t)A.T + 1;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int t = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; t < A.T; t += nw) {
        const int a = A.off[t], b = A.off[t + 1];
        if (lane == 0) A.vals[A.vbase[CS_NT] + t] = (uint32_t)(b - a);
        if (b <= a) continue;
        uint32_t* hr = A.vals + A.vbase[CS_HR] + A.tcnt[T1 + t];
        uint32_t* hy = A.vals + A.vbase[CS_HY] + A.tcnt[T1 + t];
        uint32_t* ht = A.vals + A.vbase[CS_HT] + A.tcnt[T1 + t];
        uint32_t* ds = A.vals + A.vbase[CS_DS] + A.tcnt[2 * T1 + t];
        uint32_t* dr = A.vals + A.vbase[CS_DR] + A.tcnt[3 * T1 + t];
        uint32_t* ry = A.vals + A.vbase[CS_RY] + A.tcnt[3 * T1 + t];
        uint32_t* rt = A.vals + A.vbase[CS_RT] + A.tcnt[3 * T1 + t];
        if (lane == 0) A.vals[A.vbase[CS_HS] + A.tcnt[t]] = (uint32_t)A.sector[A.clus[a]];
        // the cluster before the chunk (c1) and the one before that (c2)
        int s1 = 0, r1 = 0, r2 = 0;
        long long y1 = 0, t1 = 0, y2 = 0, t2 = 0;
        bool st1 = false;
        uint32_t nh = 0, nres = 0;
        for (int k0 = a; k0 < b; k0 += 32) {
            const int k = k0 + lane;
            const bool valid = k < b;
            int sk = 0, rk = 0;
            long long yk = 0, tk = 0;
            if (valid) {
                const int4 e = A.rec[A.clus[k]];
                sk = e.z & 0xFF;
                rk = e.z >> 8;
                yk = e.x;
                tk = e.y;
            }
            // previous and second previous cluster of each lane
            int sp = __shfl_up_sync(FULL, sk, 1), rp = __shfl_up_sync(FULL, rk, 1);
            long long yp = __shfl_up_sync(FULL, yk, 1), tp = __shfl_up_sync(FULL, tk, 1);
            int rpp = __shfl_up_sync(FULL, rk, 2);
            long long ypp = __shfl_up_sync(FULL, yk, 2), tpp = __shfl_up_sync(FULL, tk, 2);
            if (lane == 0) { sp = s1; rp = r1; yp = y1; tp = t1; rpp = r2; ypp = y2; tpp = t2; }
            if (lane == 1) { rpp = r1; ypp = y1; tpp = t1; }
            const bool start = valid && (k == a || sk != sp);
            bool stp = __shfl_up_sync(FULL, start, 1);
            if (lane == 0) stp = st1;
            const unsigned mh = __ballot_sync(FULL, start);
            const unsigned mr = __ballot_sync(FULL, valid && !start);
            if (valid && k > a) ds[k - a - 1] = zz32((long long)sk - sp);
            if (start) {
                const uint32_t o = nh + __popc(mh & lt);
                hr[o] = (uint32_t)rk;
                hy[o] = zz32(yk);
                ht[o] = zz32(tk);
            } else if (valid) {
                const uint32_t o = nres + __popc(mr & lt);
                const int nprev = stp ? 1 : 2;      // clusters of the run before this one (2: two or more)
                dr[o] = zz32((long long)rk - rp);
                ry[o] = zz32(yk - predict(nprev, ypp, rpp, yp, rp, rk));
                rt[o] = zz32(tk - predict(nprev, tpp, rpp, tp, rp, rk));
            }
            nh += __popc(mh);
            nres += __popc(mr);
            // carry the chunk's last two clusters (the loop ends after a partial chunk)
            s1 = __shfl_sync(FULL, sk, 31);
            r1 = __shfl_sync(FULL, rk, 31);
            y1 = __shfl_sync(FULL, yk, 31);
            t1 = __shfl_sync(FULL, tk, 31);
            st1 = __shfl_sync(FULL, start, 31);
            r2 = __shfl_sync(FULL, rk, 30);
            y2 = __shfl_sync(FULL, yk, 30);
            t2 = __shfl_sync(FULL, tk, 30);
        }
    }
}

// the other clusters to their plane's range (order inside: the atomics')
__global__ void k_cu_scatter(CmpArgs A)
{
    if (*A.err) return;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < A.n; i += (int64_t)gridDim.x * blockDim.x) {
        if (A.assign[i] >= 0) continue;
        const int s = A.sector[i], r = A.row[i];
        if (s >= A.ns || r >= A.nr) continue;
        const int p = s * A.nr + r;
        A.uord[A.pcnt[p] + atomicAdd(&A.pfill[p], 1u)] = (int32_t)i;
    }
}

__device__ __forceinline__ bool cu_less(int32_t ta, int32_t ya, int32_t ia, int32_t tb, int32_t yb, int32_t ib)
{
    return ta < tb || (ta == tb && (ya < yb || (ya == yb && ia < ib)));
}

// one block per plane: its other clusters ranked by (qt, qy, index) (keys in
// shared memory when they fit, else read from global memory), then the
// plane's values
__global__ void __launch_bounds__(256) k_cu_plane(CmpArgs A)
{
    __shared__ int32_t kt[CU_SMEM], ky[CU_SMEM], ki[CU_SMEM];
    if (*A.err) return;
    for (int p = blockIdx.x; p < A.np; p += gridDim.x) {
        const uint32_t ps = A.pcnt[p];
        const int m = (int)(A.pcnt[p + 1] - ps);
        if (threadIdx.x == 0) A.vals[A.vbase[CS_UN] + p] = (uint32_t)m;
        const bool sh = m <= CU_SMEM;
        __syncthreads();                    // the previous plane is done with the keys
        if (sh)
            for (int k = threadIdx.x; k < m; k += blockDim.x) {
                const int c = A.uord[ps + k];
                const int4 e = A.rec[c];
                kt[k] = e.y;
                ky[k] = e.x;
                ki[k] = c;
            }
        __syncthreads();
        for (int k = threadIdx.x; k < m; k += blockDim.x) {
            int32_t t, yv, iv;
            if (sh) {
                t = kt[k]; yv = ky[k]; iv = ki[k];
            } else {
                iv = A.uord[ps + k];
                const int4 e = A.rec[iv];
                t = e.y;
                yv = e.x;
            }
            int rank = 0;
            if (sh) {
                for (int j = 0; j < m; j++) rank += cu_less(kt[j], ky[j], ki[j], t, yv, iv);
            } else {
                for (int j = 0; j < m; j++) {
                    const int c = A.uord[ps + j];
                    const int4 e = A.rec[c];
                    rank += cu_less(e.y, e.x, c, t, yv, iv);
                }
            }
            A.usort[ps + rank] = iv;
        }
        __syncthreads();                    // usort of the plane complete (global writes of this block)
        for (int k = threadIdx.x; k < m; k += blockDim.x) {
            const int c = A.usort[ps + k];
            const int4 e = A.rec[c];
            const int32_t t = e.y;
            A.vals[A.vbase[CS_UT] + ps + k] = k == 0 ? zz32(t) : (uint32_t)(t - A.rec[A.usort[ps + k - 1]].y);
            A.vals[A.vbase[CS_UY] + ps + k] = zz32(e.x);
        }
    }
}

// ---- symbolisation: values >= 252 become an escape symbol plus raw bytes
__device__ __forceinline__ int esc_bytes(uint32_t v)
{
    if (v < 252u) return 0;
    const uint32_t w = v - 252u;
    return w < (1u << 8) ? 1 : w < (1u << 16) ? 2 : w < (1u << 24) ? 3 : 4;
}

__global__ void k_sym_count(const uint32_t* __restrict__ v, int64_t n, uint32_t* __restrict__ rawn)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        rawn[i] = (uint32_t)esc_bytes(v[i]);
}

// rawo: exclusive sums of the escape byte counts (rawo[n] = nraw)
__global__ void k_sym_write(const uint32_t* __restrict__ v, int64_t n, const uint32_t* __restrict__ rawo,
                            uint8_t* __restrict__ sym, uint8_t* __restrict__ raw)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t x = v[i];
        const int k = esc_bytes(x);
        if (k == 0) {
            sym[i] = (uint8_t)x;
            continue;
        }
        sym[i] = (uint8_t)(251 + k);
        const uint32_t w = x - 252u;
        uint8_t* o = raw + rawo[i];
        for (int b = 0; b < k; b++) o[b] = (uint8_t)(w >> (8 * b));
    }
}

// ---- exclusive scan of n uint32 in place (a[n] receives the total): tile
// sums, one-block scan of the tile sums, tiles rescanned with their offsets
constexpr int SC_BLOCK = 256, SC_ITEMS = 16, SC_TILE = SC_BLOCK * SC_ITEMS;

__global__ void __launch_bounds__(SC_BLOCK) k_tile_sum(const uint32_t* __restrict__ a, int64_t n,
                                                       uint32_t* __restrict__ sums)
{
    __shared__ uint32_t w[SC_BLOCK / 32];
    const int64_t base = (int64_t)blockIdx.x * SC_TILE;
    uint32_t s = 0;
    for (int k = threadIdx.x; k < SC_TILE; k += SC_BLOCK) {
        const int64_t i = base + k;
        if (i < n) s += a[i];
    }
    s = __reduce_add_sync(0xffffffffu, s);
    if ((threadIdx.x & 31) == 0) w[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t t = 0;
        for (int k = 0; k < SC_BLOCK / 32; k++) t += w[k];
        sums[blockIdx.x] = t;
    }
}

__global__ void __launch_bounds__(SC_BLOCK) k_tile_apply(uint32_t* __restrict__ a, int64_t n,
                                                         const uint32_t* __restrict__ sums)
{
    __shared__ uint32_t w[SC_BLOCK / 32];
    const int64_t base = (int64_t)blockIdx.x * SC_TILE + (int64_t)threadIdx.x * SC_ITEMS;
    uint32_t v[SC_ITEMS];
    uint32_t run = 0;
#pragma unroll
    for (int j = 0; j < SC_ITEMS; j++) {
        const int64_t i = base + j;
        v[j] = i < n ? a[i] : 0u;
        run += v[j];
    }
    // exclusive prefix of the thread sums within the block
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    uint32_t inc = run;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += t;
    }
    if (lane == 31) w[wid] = inc;
    __syncthreads();
    uint32_t off = sums[blockIdx.x];
    for (int k = 0; k < wid; k++) off += w[k];
    off += inc - run;
#pragma unroll
    for (int j = 0; j < SC_ITEMS; j++) {
        const int64_t i = base + j;
        if (i < n) a[i] = off;
        off += v[j];
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == SC_BLOCK - 1) a[n] = off;
}

// a[0..n] (n + 1 entries; a[n] overwritten with the total); tmp holds
// ceil(n / SC_TILE) + 1 entries
void scan_n(uint32_t* a, int64_t n, uint32_t* tmp, cudaStream_t st)
{
    const int64_t nt = std::max<int64_t>(1, (n + SC_TILE - 1) / SC_TILE);
    k_tile_sum<<<(unsigned)nt, SC_BLOCK, 0, st>>>(a, n, tmp);
    k_scan1<<<1, 1024, 0, st>>>(tmp, nt);
    k_tile_apply<<<(unsigned)nt, SC_BLOCK, 0, st>>>(a, n, tmp);
}

int64_t scan_tmp_elems(int64_t n) { return (n + SC_TILE - 1) / SC_TILE + 2; }

}  // namespace

namespace {

// container header of one stream: n, chunk, nraw, the table as u16, the
// chunk sizes; the coded total goes to *coded (one block)
__global__ void __launch_bounds__(256) k_pack_head(uint8_t* __restrict__ cont, uint32_t n, int32_t chunk,
                                                   const uint32_t* __restrict__ nraw,
                                                   const uint32_t* __restrict__ freq,
                                                   const int32_t* __restrict__ chunk_bytes, int64_t nch,
                                                   long long* __restrict__ coded)
{
    __shared__ long long part[256];
    auto put32 = [&](int64_t o, uint32_t v) {
        for (int b = 0; b < 4; b++) cont[o + b] = (uint8_t)(v >> (8 * b));
    };
    if (threadIdx.x == 0) {
        put32(0, n);
        put32(4, (uint32_t)chunk);
        put32(8, *nraw);
    }
    for (int s = threadIdx.x; s < 256; s += blockDim.x) {
        const uint32_t f = n > 0 ? freq[s] : 0u;
        cont[12 + 2 * s] = (uint8_t)(f & 0xFF);
        cont[13 + 2 * s] = (uint8_t)(f >> 8);
    }
    long long t = 0;
    for (int64_t c = threadIdx.x; c < nch; c += blockDim.x) {
        put32(524 + 4 * c, (uint32_t)chunk_bytes[c]);
        t += chunk_bytes[c];
    }
    part[threadIdx.x] = t;
    __syncthreads();
    if (threadIdx.x == 0) {
        long long sum = 0;
        for (int k = 0; k < (int)blockDim.x; k++) sum += part[k];
        *coded = sum;
    }
}

// the coded chunks and the escape bytes after the header; *size = the
// container's bytes
__global__ void k_pack_copy(uint8_t* __restrict__ cont, int64_t nch, const uint8_t* __restrict__ coded_bytes,
                            const long long* __restrict__ coded, const uint8_t* __restrict__ raw,
                            const uint32_t* __restrict__ nraw, long long* __restrict__ size)
{
    const long long nc = *coded, nr = *nraw;
    const long long o1 = 524 + 4 * nch, o2 = o1 + nc;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nc + nr;
         i += (long long)gridDim.x * blockDim.x)
        cont[o1 + i] = i < nc ? coded_bytes[i] : raw[i - nc];
    if (blockIdx.x == 0 && threadIdx.x == 0) *size = o2 + nr;
}

// per stream, its own coding regions: the streams are coded side by side
struct StreamRegions {
    size_t rawn, sym, raw, rans, cout, cbytes, freq, stmp, coded, cont;
    int64_t cap;                  // values the stream can hold
};

struct CmpLayout {
    size_t err, rec, tcnt, pcnt, pfill, uord, usort, stmp, sizes;   // fields
    size_t vals;                                                        // the streams' values
    StreamRegions st[CS_N];                                             // coding (frame only)
    int64_t max_vals, max_stream, max_cont_total;
    size_t total;
};

int64_t n_chunks(int64_t m, int32_t chunk) { return m > 0 ? (m + chunk - 1) / chunk : 0; }
int64_t cont_max(int64_t m, int32_t chunk) { return 524 + 8 * n_chunks(m, chunk) + 6 * m; }

int check_in(const tpc_compress_in* in)
{
    if (!in || in->n < 0 || in->n > (int64_t)INT32_MAX || in->n_tracks < 0 || in->n_attached < 0 ||
        in->n_attached > (int64_t)INT32_MAX || in->n_sectors < 1 || in->n_sectors > 255 || in->n_rows < 1 ||
        in->n_rows > 255)
        return TPC_ERR_ARG;
    if (in->n > 0 && (!in->sector || !in->row || !in->y || !in->zt || !in->assign)) return TPC_ERR_ARG;
    if (!in->clus_offset || (in->n_attached > 0 && !in->clus_index)) return TPC_ERR_ARG;
    return TPC_OK;
}

CmpLayout cmp_layout(const tpc_compress_in* in, int32_t chunk)
{
    CmpLayout L;
    const int64_t n = in->n, T = in->n_tracks, na = in->n_attached;
    const int64_t np = (int64_t)in->n_sectors * in->n_rows;
    L.max_vals = 2 * T + 7 * na + np + 2 * n;
    L.max_stream = std::max<int64_t>({T, na, np, n, 1});
    L.max_cont_total = 0;
    const int64_t per[CS_N] = {T, T, na, na, na, na, na, na, na, np, n, n};
    for (int s = 0; s < CS_N; s++) L.max_cont_total += (cont_max(per[s], chunk) + 15) / 16 * 16;
    size_t o = 0;
    auto take = [&](size_t b) { size_t r = o; o = al(o + std::max<size_t>(b, 1)); return r; };
    L.err = take(4);
    L.rec = take(16 * (size_t)n);
    L.tcnt = take(4 * 4 * (size_t)(T + 1));
    L.pcnt = take(4 * (size_t)(np + 1));
    L.pfill = take(4 * (size_t)np);
    L.uord = take(4 * (size_t)n);
    L.usort = take(4 * (size_t)n);
    L.stmp = take(4 * (size_t)scan_tmp_elems(std::max<int64_t>(L.max_stream, 4 * (T + 1)) + 1));
    L.sizes = take(8 * CS_N);
    L.vals = take(4 * (size_t)L.max_vals);
    for (int k = 0; k < CS_N; k++) {
        StreamRegions& R = L.st[k];
        const int64_t c = per[k];
        R.cap = c;
        R.rawn = take(4 * (size_t)(c + 1));
        R.sym = take((size_t)c);
        R.raw = take(4 * (size_t)c);
        R.rans = take(rans_layout(c, chunk).total);
        R.cout = take(4 * (size_t)n_chunks(c, chunk) + 2 * (size_t)c);
        R.cbytes = take(4 * (size_t)std::max<int64_t>(n_chunks(c, chunk), 1));
        R.freq = take(4 * 256);
        R.stmp = take(4 * (size_t)scan_tmp_elems(c + 1));
        R.coded = take(8);
        R.cont = take((size_t)cont_max(c, chunk));      // the container, packed at the end
    }
    L.total = o;
    return L;
}

}  // namespace

namespace {

#define CCK(x) do { if ((x) != cudaSuccess) return TPC_ERR_CUDA; } while (0)

// the 12 integer streams into vals (stream s from its worst-case base in
// vbase); counts (host) read back.  Synchronises the stream.
int run_fields(const tpc_compress_in* in, int32_t ey, int32_t et, void* ws, const CmpLayout& L, int64_t* counts,
               int64_t* vbase, cudaStream_t st)
{
    CmpArgs A;
    memset(&A, 0, sizeof(A));
    A.n = in->n;
    A.ns = in->n_sectors;
    A.nr = in->n_rows;
    A.np = A.ns * A.nr;
    A.T = in->n_tracks;
    A.na = in->n_attached;
    A.sector = in->sector; A.row = in->row; A.y = in->y; A.zt = in->zt;
    A.off = in->clus_offset; A.clus = in->clus_index; A.assign = in->assign;
    A.sy = ldexpf(1.0f, ey);
    A.st = ldexpf(1.0f, et);
    A.rec = at<int4>(ws, L.rec);
    A.tcnt = at<uint32_t>(ws, L.tcnt);
    A.pcnt = at<uint32_t>(ws, L.pcnt);
    A.pfill = at<uint32_t>(ws, L.pfill);
    A.uord = at<int32_t>(ws, L.uord);
    A.usort = at<int32_t>(ws, L.usort);
    A.err = at<int>(ws, L.err);
    A.vals = at<uint32_t>(ws, L.vals);
    // worst-case stream bases: NT, HS: T; HR .. RT: n_attached each; UN: planes; UT, UY: n
    const int64_t per[CS_N] = {A.T, A.T, A.na, A.na, A.na, A.na, A.na, A.na, A.na, A.np, A.n, A.n};
    A.vbase[0] = 0;
    for (int k = 0; k < CS_N; k++) A.vbase[k + 1] = A.vbase[k] + per[k];
    uint32_t* stmp = at<uint32_t>(ws, L.stmp);
    const int64_t T1 = (int64_t)A.T + 1;
    CCK(cudaMemsetAsync(A.err, 0, 4, st));
    CCK(cudaMemsetAsync(A.pcnt, 0, 4 * ((size_t)A.np + 1), st));
    CCK(cudaMemsetAsync(A.pfill, 0, 4 * (size_t)A.np, st));
    // the offset table must start at 0 and end at n_attached
    if (A.n > 0) k_cq<<<grid_cap(A.n, 256), 256, 0, st>>>(A);
    if (A.T > 0) k_ct_count<<<grid_cap(A.T, 128), 128, 0, st>>>(A);
    for (int k = 0; k < 4; k++) scan_n(A.tcnt + k * T1, A.T, stmp, st);
    scan_n(A.pcnt, A.np, stmp, st);
    k_ct_fill<<<grid_cap(32 * (int64_t)std::max(A.T, 1), 256), 256, 0, st>>>(A);
    if (A.n > 0) k_cu_scatter<<<grid_cap(A.n, 256), 256, 0, st>>>(A);
    k_cu_plane<<<(unsigned)std::min(A.np, 148 * 8), 256, 0, st>>>(A);
    CCK(cudaGetLastError());
    // read back: error flag, offset table ends, stream lengths
    uint32_t tc[4] = {0, 0, 0, 0}, pc = 0;
    int32_t ends[2] = {0, 0};
    int e = 0;
    CCK(cudaMemcpyAsync(&e, A.err, 4, cudaMemcpyDeviceToHost, st));
    for (int k = 0; k < 4; k++) CCK(cudaMemcpyAsync(&tc[k], A.tcnt + k * T1 + A.T, 4, cudaMemcpyDeviceToHost, st));
    CCK(cudaMemcpyAsync(&pc, A.pcnt + A.np, 4, cudaMemcpyDeviceToHost, st));
    CCK(cudaMemcpyAsync(&ends[0], A.off, 4, cudaMemcpyDeviceToHost, st));
    CCK(cudaMemcpyAsync(&ends[1], A.off + A.T, 4, cudaMemcpyDeviceToHost, st));
    CCK(cudaStreamSynchronize(st));
    if (e || ends[0] != 0 || (int64_t)ends[1] != A.na) return TPC_ERR_DATA;
    const int64_t cnt[CS_N] = {A.T, tc[0], tc[1], tc[1], tc[1], tc[2], tc[3], tc[3], tc[3], A.np, pc, pc};
    for (int k = 0; k < CS_N; k++) {
        counts[k] = cnt[k];
        vbase[k] = A.vbase[k];
    }
    return TPC_OK;
}

}  // namespace

extern "C" int tpc_compress_workspace_size(const tpc_compress_in* in, int32_t chunk, size_t* bytes)
{
    if (check_in(in) || !bytes || chunk < 1 || chunk > TPC_RANS_MAX_CHUNK) return TPC_ERR_ARG;
    *bytes = cmp_layout(in, chunk).total;
    return TPC_OK;
}

extern "C" int tpc_compress_max_size(const tpc_compress_in* in, int32_t chunk, int64_t* max_values,
                                     int64_t* max_bytes)
{
    if (check_in(in) || chunk < 1 || chunk > TPC_RANS_MAX_CHUNK) return TPC_ERR_ARG;
    const CmpLayout L = cmp_layout(in, chunk);
    if (max_values) *max_values = L.max_vals;
    if (max_bytes) *max_bytes = L.max_cont_total;
    return TPC_OK;
}

extern "C" int tpc_compress_fields(const tpc_compress_in* in, int32_t ey, int32_t et, void* workspace,
                                   size_t ws_bytes, uint32_t* vals, int64_t vals_cap, int64_t* counts, void* stream)
{
    if (check_in(in) || !counts || !workspace || ey < -30 || ey > 30 || et < -30 || et > 30) return TPC_ERR_ARG;
    const CmpLayout L = cmp_layout(in, 4096);     // the fields' regions do not depend on the chunk
    if (ws_bytes < L.vals + 4 * (size_t)L.max_vals || (L.max_vals > 0 && (!vals || vals_cap < L.max_vals)))
        return TPC_ERR_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int64_t vbase[CS_N];
    int rc = run_fields(in, ey, et, workspace, L, counts, vbase, st);
    if (rc) return rc;
    int64_t o = 0;
    for (int k = 0; k < CS_N; k++) {
        if (counts[k] > 0)
            CCK(cudaMemcpyAsync(vals + o, at<uint32_t>(workspace, L.vals) + vbase[k], 4 * (size_t)counts[k],
                                cudaMemcpyDeviceToDevice, st));
        o += counts[k];
    }
    CCK(cudaStreamSynchronize(st));
    return TPC_OK;
}

extern "C" int tpc_compress_frame(const tpc_compress_in* in, int32_t ey, int32_t et, int32_t chunk, void* workspace,
                                  size_t ws_bytes, uint8_t* out, int64_t out_cap, int64_t* bytes, void* stream)
{
    if (check_in(in) || !bytes || !workspace || !out || chunk < 1 || chunk > TPC_RANS_MAX_CHUNK || ey < -30 ||
        ey > 30 || et < -30 || et > 30)
        return TPC_ERR_ARG;
    const CmpLayout L = cmp_layout(in, chunk);
    if (ws_bytes < L.total || out_cap < L.max_cont_total) return TPC_ERR_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int64_t counts[CS_N], vbase[CS_N];
    int rc = run_fields(in, ey, et, workspace, L, counts, vbase, st);
    if (rc) return rc;
    uint32_t* vals = at<uint32_t>(workspace, L.vals);
    long long* sizes = at<long long>(workspace, L.sizes);
    // per stream: symbols and escape bytes, histogram and table
    ChunkJobs J;
    memset(&J, 0, sizeof(J));
    J.chunk = chunk;
    int32_t nblocks = 0;
    int64_t nchs[CS_N];
    for (int k = 0; k < CS_N; k++) {
        const StreamRegions& R = L.st[k];
        const int64_t m = counts[k], nch = n_chunks(m, chunk);
        nchs[k] = nch;
        if (m > R.cap) return TPC_ERR_DATA;
        const uint32_t* v = vals + vbase[k];
        uint32_t* rawn = at<uint32_t>(workspace, R.rawn);
        uint8_t* sym = at<uint8_t>(workspace, R.sym);
        uint8_t* raw = at<uint8_t>(workspace, R.raw);
        if (m > 0) k_sym_count<<<grid_cap(m, 256), 256, 0, st>>>(v, m, rawn);
        scan_n(rawn, m, at<uint32_t>(workspace, R.stmp), st);          // rawn[m] = escape bytes
        if (m == 0) continue;
        k_sym_write<<<grid_cap(m, 256), 256, 0, st>>>(v, m, rawn, sym, raw);
        const RansLayout RL = rans_layout(R.cap, chunk);
        void* rw = at<void>(workspace, R.rans);
        CCK(cudaMemsetAsync(at<uint32_t>(rw, RL.hist), 0, 4 * 256, st));
        CCK(cudaMemsetAsync(at<int>(rw, RL.err), 0, 4, st));
        k_rans_hist<<<grid_cap(m, 256), 256, 0, st>>>(sym, m, at<uint32_t>(rw, RL.hist));
        k_rans_table<<<1, TABLE_THREADS, 0, st>>>(at<uint32_t>(rw, RL.hist), at<uint32_t>(workspace, R.freq),
                                                  at<uint32_t>(rw, RL.cum), at<int>(rw, RL.err));
        ChunkJob& q = J.j[J.njobs++];
        q.sym = sym;
        q.n = m;
        q.freq = at<uint32_t>(workspace, R.freq);
        q.cum = at<uint32_t>(rw, RL.cum);
        q.scratch = at<uint8_t>(rw, RL.scratch);
        q.len = at<int32_t>(rw, RL.len);
        q.err = at<int>(rw, RL.err);
        q.block0 = nblocks;
        q.blocks = (int32_t)std::min<int64_t>((nch + 127) / 128, 148 * 16);
        nblocks += q.blocks;
    }
    CCK(cudaGetLastError());
    // every stream's chunks in one launch: the serial chunk chains run side by side
    if (J.njobs > 0) k_rans_chunks_multi<<<nblocks, 128, 0, st>>>(J);
    // per stream: chunk offsets, the chunks back to back, the container
    for (int k = 0; k < CS_N; k++) {
        const StreamRegions& R = L.st[k];
        const int64_t m = counts[k], nch = nchs[k];
        uint32_t* rawn = at<uint32_t>(workspace, R.rawn);
        const RansLayout RL = rans_layout(R.cap, chunk);
        void* rw = at<void>(workspace, R.rans);
        int32_t* cbytes = at<int32_t>(workspace, R.cbytes);
        uint8_t* cout = at<uint8_t>(workspace, R.cout);
        if (nch > 0) {
            k_rans_scan<<<1, 1024, 0, st>>>(at<int32_t>(rw, RL.len), nch, at<long long>(rw, RL.off), at<int>(rw, RL.err));
            k_rans_copy<<<(int)std::min<int64_t>(nch, 148 * 32), 128, 0, st>>>(
                at<uint8_t>(rw, RL.scratch), chunk, nch, at<int32_t>(rw, RL.len), at<long long>(rw, RL.off), cout,
                4 * nch + 2 * m, cbytes, at<int>(rw, RL.err));
        }
        long long* coded = at<long long>(workspace, R.coded);
        uint8_t* cont = at<uint8_t>(workspace, R.cont);
        k_pack_head<<<1, 256, 0, st>>>(cont, (uint32_t)m, chunk, rawn + m, at<uint32_t>(workspace, R.freq), cbytes,
                                       nch, coded);
        k_pack_copy<<<grid_cap(2 * m + 4 * nch + 1, 256), 256, 0, st>>>(cont, nch, cout, coded,
                                                                       at<uint8_t>(workspace, R.raw), rawn + m,
                                                                       sizes + k);
    }
    CCK(cudaGetLastError());
    long long sz[CS_N];
    CCK(cudaMemcpyAsync(sz, sizes, sizeof(sz), cudaMemcpyDeviceToHost, st));
    CCK(cudaStreamSynchronize(st));
    int64_t p = 0;
    for (int k = 0; k < CS_N; k++) {
        CCK(cudaMemcpyAsync(out + p, at<uint8_t>(workspace, L.st[k].cont), (size_t)sz[k], cudaMemcpyDeviceToDevice,
                            st));
        bytes[k] = sz[k];
        p += sz[k];
    }
    CCK(cudaStreamSynchronize(st));
    return TPC_OK;
}
