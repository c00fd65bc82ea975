// Frequency distribution of one column of a local count table: the paper's
// experiments ("Demonstrations of Pivoter", the per-vertex clique
// distributions) plot f_k(b), the number of vertices that take part in
// exactly b k-cliques; the same function over edges comes from the per-edge
// table.  Values are exact W-word integers, so the distribution is
// built by exact-key aggregation in a device hash table (linear probing,
// at least twice as many slots as rows), then compacted.
#include <string>

#include "pvt_internal.cuh"

namespace pvt {
namespace {

constexpr uint32_t SLOT_EMPTY = 0xFFFFFFFFu;

// SplitMix64 finaliser (Steele, Lea and Flood 2014) as the slot hash.
__device__ __forceinline__ unsigned long long mix64(unsigned long long z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Rows with equal values inside a warp are grouped first (one match per
// word), so a value shared by many rows (zero, typically) costs one insert
// per warp; the group's leader inserts the row index of its first member
// and adds the group size.
__global__ void k_freq_insert(const unsigned long long *__restrict__ t, int64_t rows, int K, int W, int k,
                              uint32_t *owner, unsigned long long *cnt, uint64_t mask, unsigned *err)
{
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = blockIdx.x * (int64_t)blockDim.x + threadIdx.x - lane; base < rows; base += stride) {
        const int64_t r = base + lane;
        const bool valid = r < rows;
        const unsigned act = __ballot_sync(0xFFFFFFFFu, valid);
        if (!valid) continue;
        const unsigned long long *key = t + ((size_t)r * K + k) * W;
        unsigned peers = act;
        unsigned long long h = 0x9E3779B97F4A7C15ull;
        for (int w = 0; w < W; ++w) {
            const unsigned long long x = key[w];
            peers &= __match_any_sync(act, x);
            h = mix64(h ^ x);
        }
        if (lane != __ffs(peers) - 1) continue;  // not the group's leader
        const unsigned long long add = (unsigned long long)__popc(peers);
        uint64_t s = h & mask;
        for (uint64_t probe = 0;; ++probe) {
            if (probe > mask) {
                atomicOr(err, DERR_RANGE);
                break;
            }
            const uint32_t o = atomicCAS(&owner[s], SLOT_EMPTY, (uint32_t)r);
            bool same = o == SLOT_EMPTY;
            if (!same) {
                const unsigned long long *ok = t + ((size_t)o * K + k) * W;
                same = true;
                for (int w = 0; w < W; ++w) same = same && ok[w] == key[w];
            }
            if (same) {
                atomicAdd(&cnt[s], add);
                break;
            }
            s = (s + 1) & mask;
        }
    }
}

// Occupied slots -> (value, count) pairs, in slot order within a warp.
__global__ void k_freq_compact(const uint32_t *__restrict__ owner, const unsigned long long *__restrict__ cnt,
                               uint64_t cap, const unsigned long long *__restrict__ t, int K, int W, int k,
                               unsigned long long *values, unsigned long long *counts, unsigned long long *n_out)
{
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = blockIdx.x * (int64_t)blockDim.x + threadIdx.x - lane; base < (int64_t)cap;
         base += stride) {
        const int64_t s = base + lane;
        const bool occ = s < (int64_t)cap && owner[s] != SLOT_EMPTY;
        const unsigned b = __ballot_sync(0xFFFFFFFFu, occ);
        if (!b) continue;
        unsigned long long at = 0;
        if (lane == 0) at = atomicAdd(n_out, (unsigned long long)__popc(b));
        at = __shfl_sync(0xFFFFFFFFu, at, 0);
        if (occ) {
            const unsigned long long i = at + __popc(b & ((1u << lane) - 1u));
            const unsigned long long *key = t + ((size_t)owner[s] * K + k) * W;
            for (int w = 0; w < W; ++w) values[i * W + w] = key[w];
            counts[i] = cnt[s];
        }
    }
}

}  // namespace
}  // namespace pvt

using namespace pvt;

extern "C" pvt_status pvt_local_distribution(const uint64_t *table, int64_t rows, int32_t K, int32_t W, int32_t k,
                                             uint64_t *values, uint64_t *counts, int64_t *n_distinct,
                                             void *stream)
{
    const pvt::HostRange range("pvt_local_distribution");
    if (rows < 0 || rows > 0xFFFFFFFEll || K < 1 || k < 0 || k >= K || W < 1 || W > WMAX || !n_distinct ||
        (rows > 0 && (!table || !values || !counts))) {
        set_error("pvt_local_distribution: invalid argument");
        return PVT_EINVAL;
    }
    *n_distinct = 0;
    if (rows == 0) return PVT_OK;
    cudaStream_t s = (cudaStream_t)stream;
    uint64_t cap = 1024;
    while (cap < 2 * (uint64_t)rows) cap <<= 1;
    unsigned char *scratch = nullptr;
    const size_t bytes = cap * sizeof(uint32_t) + cap * sizeof(unsigned long long) + 16;
    PVT_CK(cudaMallocAsync(&scratch, bytes, s));
    unsigned long long *cnt = reinterpret_cast<unsigned long long *>(scratch);
    uint32_t *owner = reinterpret_cast<uint32_t *>(scratch + cap * sizeof(unsigned long long));
    unsigned long long *n_out = reinterpret_cast<unsigned long long *>(scratch + bytes - 16);
    unsigned *err = reinterpret_cast<unsigned *>(n_out + 1);
    pvt_status st = PVT_OK;
    cudaError_t e = cudaMemsetAsync(cnt, 0, cap * sizeof(unsigned long long), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(owner, 0xFF, cap * sizeof(uint32_t), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(n_out, 0, 16, s);
    int dev = 0, sms = 1;
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) {
        const int grid = sms * 8;
        k_freq_insert<<<grid, 256, 0, s>>>(reinterpret_cast<const unsigned long long *>(table), rows, K, W, k,
                                           owner, cnt, cap - 1, err);
        k_freq_compact<<<grid, 256, 0, s>>>(owner, cnt, cap, reinterpret_cast<const unsigned long long *>(table), K,
                                            W, k, reinterpret_cast<unsigned long long *>(values),
                                            reinterpret_cast<unsigned long long *>(counts), n_out);
        e = cudaGetLastError();
    }
    unsigned long long host[2] = {0, 0};
    if (e == cudaSuccess) e = cudaMemcpyAsync(host, n_out, 16, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) st = cuda_fail(e, "pvt_local_distribution");
    cudaFreeAsync(scratch, s);
    if (st != PVT_OK) return st;
    if ((unsigned)(host[1] & 0xFFFFFFFFull)) {
        set_error("pvt_local_distribution: hash table overflow");
        return PVT_EINTERNAL;
    }
    *n_distinct = (int64_t)host[0];
    return PVT_OK;
}
