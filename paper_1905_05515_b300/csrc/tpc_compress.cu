// Entropy coder of the cluster compression: rANS of byte symbols with one
// static 12-bit table per stream, in independent chunks (paper, section
// "TPC Data Compression", step 4; the format is stated in tpc_compress.h).
//
// Kernels: k_rans_hist (block histograms in shared memory, one global add
// per bin and block), k_rans_table (one thread: the largest-remainder
// normalisation over 256 symbols), k_rans_chunks (one thread per chunk: the
// chunk is coded last symbol first into its own scratch slot, bytes written
// from the slot's end backward, so they come out in decode order), a scan of
// the chunk sizes and k_rans_copy (one block per chunk) packing the chunks
// back to back.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

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

// one thread: the table (largest remainders), its cumulative sums
__global__ void k_rans_table(const uint32_t* __restrict__ hist, uint32_t* __restrict__ freq,
                             uint32_t* __restrict__ cum, int* __restrict__ err)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    unsigned long long total = 0;
    for (int s = 0; s < 256; s++) total += hist[s];
    if (total == 0) {
        for (int s = 0; s < 256; s++) freq[s] = 0;
        for (int s = 0; s <= 256; s++) cum[s] = 0;
        return;
    }
    unsigned long long rem[256];
    bool got[256];
    long long sum = 0;
    for (int s = 0; s < 256; s++) {
        const unsigned long long m = (unsigned long long)hist[s] * RANS_M;
        freq[s] = (uint32_t)(m / total);
        rem[s] = m % total;
        got[s] = false;
        sum += freq[s];
    }
    while (sum < (long long)RANS_M) {
        int best = -1;
        for (int s = 0; s < 256; s++) {
            if (hist[s] == 0 || got[s]) continue;
            if (best < 0 || rem[s] > rem[best]) best = s;
        }
        if (best < 0) { *err = 1; return; }
        freq[best]++;
        got[best] = true;
        sum++;
    }
    for (int s = 0; s < 256; s++)
        if (hist[s] > 0 && freq[s] == 0) { freq[s] = 1; sum++; }
    while (sum > (long long)RANS_M) {
        int best = -1;
        for (int s = 0; s < 256; s++) {
            if (freq[s] <= 1) continue;
            if (best < 0 || freq[s] > freq[best]) best = s;
        }
        if (best < 0) { *err = 1; return; }
        freq[best]--;
        sum--;
    }
    cum[0] = 0;
    for (int s = 0; s < 256; s++) cum[s + 1] = cum[s] + freq[s];
}

// one thread per chunk; slot c holds 4 + 2 chunk bytes, filled from its end
__global__ void __launch_bounds__(128) k_rans_chunks(const uint8_t* __restrict__ sym, int64_t n, int32_t chunk,
                                                     const uint32_t* __restrict__ freq_g,
                                                     const uint32_t* __restrict__ cum_g,
                                                     uint8_t* __restrict__ scratch, int32_t* __restrict__ len,
                                                     const int* __restrict__ err)
{
    __shared__ uint32_t freq[256], cum[256];
    for (int s = threadIdx.x; s < 256; s += blockDim.x) {
        freq[s] = freq_g[s];
        cum[s] = cum_g[s];
    }
    __syncthreads();
    if (*err) return;
    const int64_t nch = (n + chunk - 1) / chunk;
    const size_t cap = 4 + 2 * (size_t)chunk;
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < nch; c += (int64_t)gridDim.x * blockDim.x) {
        const int64_t a = c * chunk;
        const int64_t m = min((int64_t)chunk, n - a);
        uint8_t* base = scratch + (size_t)c * cap;
        size_t p = cap;
        uint32_t x = RANS_L;
        for (int64_t i = a + m - 1; i >= a; i--) {
            const uint32_t s = sym[i];
            const uint32_t f = freq[s];
            const uint32_t xmax = ((RANS_L >> RANS_BITS) << 8) * f;
            while (x >= xmax) {
                base[--p] = (uint8_t)(x & 0xFF);
                x >>= 8;
            }
            x = ((x / f) << RANS_BITS) + (x % f) + cum[s];
        }
        base[--p] = (uint8_t)(x & 0xFF);
        base[--p] = (uint8_t)((x >> 8) & 0xFF);
        base[--p] = (uint8_t)((x >> 16) & 0xFF);
        base[--p] = (uint8_t)(x >> 24);
        len[c] = (int32_t)(cap - p);
    }
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
    k_rans_table<<<1, 32, 0, st>>>(hist, freq, cum, err);
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
