// tpc_probe.cu -- fused multiply-add throughput probes (include/tpc_probe.h):
// the measured binary32 / binary64 rates the Kalman stages' rooflines divide by.
#include <cuda_runtime.h>

#include "tpc_probe.h"
#include "tpc_track.h"

namespace {

constexpr int CHAINS = 8;

// Eight independent chains per thread hide the multiply-add latency; a and b
// keep every chain finite (|a| < 1).  One value per block leaves the kernel.
template <typename T>
__global__ void k_fma_probe(int iters, T a, T b, T* __restrict__ out)
{
    T x[CHAINS];
#pragma unroll
    for (int c = 0; c < CHAINS; c++) x[c] = (T)(threadIdx.x + c) * (T)1e-3;
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int c = 0; c < CHAINS; c++) x[c] = fma(x[c], a, b);
    }
    T s = 0;
#pragma unroll
    for (int c = 0; c < CHAINS; c++) s += x[c];
    __shared__ T red[32];
    // any lane's value makes the chains live; one store per block
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        T t = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) t += red[w];
        out[blockIdx.x] = t;
    }
}

}  // namespace

extern "C" int tpc_probe_fma(int32_t precision, int32_t blocks, int32_t threads, int32_t iters, void* out,
                             int64_t* flops, void* stream)
{
    if ((precision != 32 && precision != 64) || blocks < 1 || blocks > (1 << 20) || threads < 32 ||
        threads > 1024 || threads % 32 || iters < 1 || iters > (1 << 24) || !out || !flops)
        return TPC_ERR_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (precision == 32)
        k_fma_probe<float><<<blocks, threads, 0, st>>>(iters, 0.9999f, 1e-4f, static_cast<float*>(out));
    else
        k_fma_probe<double><<<blocks, threads, 0, st>>>(iters, 0.9999, 1e-4, static_cast<double*>(out));
    if (cudaGetLastError() != cudaSuccess) return TPC_ERR_CUDA;
    *flops = 2LL * CHAINS * (int64_t)iters * (int64_t)blocks * (int64_t)threads;
    return TPC_OK;
}
