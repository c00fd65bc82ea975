// The integer ceiling of the walk kernels, measured.  Their unit of work is
// one pivot word pair: a 32-bit AND of a row word with a label word, its
// population count, and the add into the member's neighbour count.  This
// kernel runs that triple on independent register chains, with no memory
// traffic, on every SM, and reports how many triples per second the GPU
// sustains: the denominator of the walks' roofline.
#include <algorithm>

#include "pvt_internal.cuh"

namespace pvt {
namespace {

constexpr int RATE_CHAINS = 8;      // independent chains per thread
constexpr int RATE_THREADS = 256;
constexpr int RATE_BLOCKS_PER_SM = 8;
constexpr int RATE_ITERS = 1 << 15;

// Each iteration advances one label word m (a linear congruential step,
// shared by the chains) and adds popc(x_j & m) into chain j: the label
// changes every iteration, so nothing can be hoisted.  The sums go to sink
// so that no chain is dead.
__global__ void __launch_bounds__(RATE_THREADS) k_popc_rate(unsigned *sink, int iters, unsigned seed)
{
    const unsigned gid = blockIdx.x * blockDim.x + threadIdx.x;
    unsigned x[RATE_CHAINS], c[RATE_CHAINS];
#pragma unroll
    for (int j = 0; j < RATE_CHAINS; ++j) {
        x[j] = gid * 0x9E3779B9u + (unsigned)j * 0x85EBCA6Bu + seed;
        c[j] = 0;
    }
    unsigned m = seed | 1u;
    for (int it = 0; it < iters; ++it) {
        m = m * 1664525u + 1013904223u;
#pragma unroll
        for (int j = 0; j < RATE_CHAINS; ++j) c[j] += __popc(x[j] & m);
    }
    unsigned s = 0;
#pragma unroll
    for (int j = 0; j < RATE_CHAINS; ++j) s += c[j];
    sink[gid] = s;
}

}  // namespace
}  // namespace pvt

extern "C" pvt_status pvt_measure_popc_rate(double *pairs_per_s, void *stream)
{
    using namespace pvt;
    const HostRange range("pvt_measure_popc_rate");
    if (!pairs_per_s) {
        set_error("pvt_measure_popc_rate: NULL argument");
        return PVT_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0, sms = 0;
    PVT_CK(cudaGetDevice(&dev));
    PVT_CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const unsigned blocks = (unsigned)std::max(sms, 1) * RATE_BLOCKS_PER_SM;
    unsigned *sink = nullptr;
    PVT_CK(cudaMallocAsync(&sink, (size_t)blocks * RATE_THREADS * sizeof(unsigned), s));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    pvt_status st = PVT_OK;
    float best = 0.f;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) st = PVT_ECUDA;
    // one warm-up launch, then the fastest of three timed ones
    for (int rep = 0; rep < 4 && st == PVT_OK; ++rep) {
        if (cudaEventRecord(e0, s) != cudaSuccess) st = PVT_ECUDA;
        k_popc_rate<<<blocks, RATE_THREADS, 0, s>>>(sink, RATE_ITERS, 0x2545F491u + (unsigned)rep);
        if (cudaGetLastError() != cudaSuccess || cudaEventRecord(e1, s) != cudaSuccess ||
            cudaEventSynchronize(e1) != cudaSuccess)
            st = PVT_ECUDA;
        float ms = 0.f;
        if (st == PVT_OK && cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) st = PVT_ECUDA;
        if (st == PVT_OK && rep > 0 && (best == 0.f || ms < best)) best = ms;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFreeAsync(sink, s);
    if (st != PVT_OK) {
        set_error("pvt_measure_popc_rate: CUDA error");
        return st;
    }
    const double pairs = (double)blocks * RATE_THREADS * (double)RATE_ITERS * RATE_CHAINS;
    *pairs_per_s = best > 0.f ? pairs / (best * 1e-3) : 0.0;
    return PVT_OK;
}
