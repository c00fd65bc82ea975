// Host drivers of the clique counts (global, per-vertex, per-edge), the
// batched form, the combine kernels and the allocation-free entry point.
// The walk kernels themselves live in walk.cuh, instantiated per bitset
// width in walk_nw*.cu.
#include <algorithm>
#include <mutex>
#include <string>

#include "walk.cuh"

namespace pvt {

extern template pvt_status launch_class<1, MODE_GLOBAL, true>(pvt_dag *, const CountArgs &, int, cudaStream_t);
extern template pvt_status launch_class<1, MODE_VERTEX, false>(pvt_dag *, const CountArgs &, int, cudaStream_t);
extern template pvt_status launch_class<1, MODE_EDGE, false>(pvt_dag *, const CountArgs &, int, cudaStream_t);
extern template pvt_status launch_class<2, MODE_GLOBAL, true>(pvt_dag *, const CountArgs &, int, cudaStream_t);
extern template pvt_status launch_class<2, MODE_VERTEX, false>(pvt_dag *, const CountArgs &, int, cudaStream_t);
extern template pvt_status launch_class<2, MODE_EDGE, false>(pvt_dag *, const CountArgs &, int, cudaStream_t);
extern template pvt_status launch_class<4, MODE_GLOBAL, true>(pvt_dag *, const CountArgs &, int, cudaStream_t);
extern template pvt_status launch_class<4, MODE_VERTEX, false>(pvt_dag *, const CountArgs &, int, cudaStream_t);
extern template pvt_status launch_class<4, MODE_EDGE, false>(pvt_dag *, const CountArgs &, int, cudaStream_t);
extern template pvt_status launch_class<8, MODE_GLOBAL, true>(pvt_dag *, const CountArgs &, int, cudaStream_t);
extern template pvt_status launch_class<8, MODE_VERTEX, false>(pvt_dag *, const CountArgs &, int, cudaStream_t);
extern template pvt_status launch_class<8, MODE_EDGE, false>(pvt_dag *, const CountArgs &, int, cudaStream_t);
extern template pvt_status launch_class<16, MODE_GLOBAL, true>(pvt_dag *, const CountArgs &, int, cudaStream_t);
extern template pvt_status launch_class<16, MODE_VERTEX, false>(pvt_dag *, const CountArgs &, int, cudaStream_t);
extern template pvt_status launch_class<16, MODE_EDGE, false>(pvt_dag *, const CountArgs &, int, cudaStream_t);
extern template pvt_status launch_class<32, MODE_GLOBAL, true>(pvt_dag *, const CountArgs &, int, cudaStream_t);
extern template pvt_status launch_class<32, MODE_VERTEX, false>(pvt_dag *, const CountArgs &, int, cudaStream_t);
extern template pvt_status launch_class<32, MODE_EDGE, false>(pvt_dag *, const CountArgs &, int, cudaStream_t);
extern template pvt_status launch_batch_class<1, MODE_GLOBAL>(const BatchGraph *, const uint64_t *, unsigned, unsigned *, const unsigned long long *, int, unsigned *, unsigned long long *, int, cudaStream_t);
extern template pvt_status launch_batch_class<1, MODE_VERTEX>(const BatchGraph *, const uint64_t *, unsigned, unsigned *, const unsigned long long *, int, unsigned *, unsigned long long *, int, cudaStream_t);
extern template pvt_status launch_batch_class<1, MODE_EDGE>(const BatchGraph *, const uint64_t *, unsigned, unsigned *, const unsigned long long *, int, unsigned *, unsigned long long *, int, cudaStream_t);
extern template pvt_status launch_batch_class<2, MODE_GLOBAL>(const BatchGraph *, const uint64_t *, unsigned, unsigned *, const unsigned long long *, int, unsigned *, unsigned long long *, int, cudaStream_t);
extern template pvt_status launch_batch_class<2, MODE_VERTEX>(const BatchGraph *, const uint64_t *, unsigned, unsigned *, const unsigned long long *, int, unsigned *, unsigned long long *, int, cudaStream_t);
extern template pvt_status launch_batch_class<2, MODE_EDGE>(const BatchGraph *, const uint64_t *, unsigned, unsigned *, const unsigned long long *, int, unsigned *, unsigned long long *, int, cudaStream_t);
extern template pvt_status launch_batch_class<4, MODE_GLOBAL>(const BatchGraph *, const uint64_t *, unsigned, unsigned *, const unsigned long long *, int, unsigned *, unsigned long long *, int, cudaStream_t);
extern template pvt_status launch_batch_class<4, MODE_VERTEX>(const BatchGraph *, const uint64_t *, unsigned, unsigned *, const unsigned long long *, int, unsigned *, unsigned long long *, int, cudaStream_t);
extern template pvt_status launch_batch_class<4, MODE_EDGE>(const BatchGraph *, const uint64_t *, unsigned, unsigned *, const unsigned long long *, int, unsigned *, unsigned long long *, int, cudaStream_t);
extern template pvt_status launch_batch_class<8, MODE_GLOBAL>(const BatchGraph *, const uint64_t *, unsigned, unsigned *, const unsigned long long *, int, unsigned *, unsigned long long *, int, cudaStream_t);
extern template pvt_status launch_batch_class<8, MODE_VERTEX>(const BatchGraph *, const uint64_t *, unsigned, unsigned *, const unsigned long long *, int, unsigned *, unsigned long long *, int, cudaStream_t);
extern template pvt_status launch_batch_class<8, MODE_EDGE>(const BatchGraph *, const uint64_t *, unsigned, unsigned *, const unsigned long long *, int, unsigned *, unsigned long long *, int, cudaStream_t);
extern template pvt_status launch_batch_class<16, MODE_GLOBAL>(const BatchGraph *, const uint64_t *, unsigned, unsigned *, const unsigned long long *, int, unsigned *, unsigned long long *, int, cudaStream_t);
extern template pvt_status launch_batch_class<16, MODE_VERTEX>(const BatchGraph *, const uint64_t *, unsigned, unsigned *, const unsigned long long *, int, unsigned *, unsigned long long *, int, cudaStream_t);
extern template pvt_status launch_batch_class<16, MODE_EDGE>(const BatchGraph *, const uint64_t *, unsigned, unsigned *, const unsigned long long *, int, unsigned *, unsigned long long *, int, cudaStream_t);

// The test-settable limit of the bounded device waits (policy.wait_limit_us).
static void apply_wait_limit(const pvt_dag *g, CountArgs &A)
{
    if (g->policy.wait_limit_us > 0) A.idle_ns = A.slot_ns = 1000ull * (unsigned long long)g->policy.wait_limit_us;
}

// ------------------------------------------------------ small kernels

// Roots with no out-neighbour: one path each with h = 1, p = 0.
__global__ void k_add_leaf(unsigned long long *cell, unsigned long long count)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) *cell += count;
}

// Sum of histogram row 1 (leaves with h = 1) into *out: taken before a
// range walk adds to a caller's histogram, as the base of k_check_paths.
__global__ void __launch_bounds__(256) k_row1_sum(const unsigned long long *__restrict__ hist, int hstride,
                                                  unsigned long long *out)
{
    __shared__ unsigned long long acc;
    if (threadIdx.x == 0) acc = 0;
    __syncthreads();
    unsigned long long a = 0;
    for (int p = threadIdx.x; p < hstride; p += blockDim.x) a += hist[hstride + p];
    atomicAdd(&acc, a);
    __syncthreads();
    if (threadIdx.x == 0) *out = acc;
}

// Consistency of a walk's (h, p) leaf histogram with the root paths of the
// SCT (Thm. scr).  Each walked root has exactly one all-pivot path, a leaf
// with h = 1, so row 1 gains one leaf per root (`roots`; minus *base, the
// row's sum before the walk, if base is set).  With orow set (a walk of every
// root, kmax >= 2), the 2-cliques read off the histogram,
// sum_p p * hist[1][p] + sum_p hist[2][p], are the edges of the DAG,
// orow[n] - orow[0].  A mismatch means walk work was lost or repeated:
// DERR_CHECK.
__global__ void __launch_bounds__(256) k_check_paths(const unsigned long long *__restrict__ hist, int hstride,
                                                     const unsigned long long *base, unsigned long long roots,
                                                     const int64_t *orow, int64_t n, unsigned *err)
{
    __shared__ unsigned long long s1, s2;
    if (threadIdx.x == 0) s1 = s2 = 0;
    __syncthreads();
    unsigned long long a = 0, b = 0;
    for (int p = threadIdx.x; p < hstride; p += blockDim.x) {
        const unsigned long long x = hist[hstride + p];
        a += x;
        b += x * (unsigned long long)p;
        if (2 < hstride) b += hist[2 * (size_t)hstride + p];
    }
    atomicAdd(&s1, a);
    atomicAdd(&s2, b);
    __syncthreads();
    if (threadIdx.x != 0) return;
    bool ok = s1 - (base ? *base : 0ull) == roots;
    if (orow) ok = ok && s2 == (unsigned long long)(orow[n] - orow[0]);
    if (!ok) atomicOr(err, DERR_CHECK);
}

// Local counts of roots with no out-neighbour: c_1(r) += 1.
__global__ void k_vertex_trivial(const uint32_t *__restrict__ roots, unsigned nroots,
                                 unsigned long long *cv, int K, int W)
{
    for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < nroots; i += gridDim.x * blockDim.x)
        cv[((size_t)roots[i] * K + 1) * W] += 1ull;
}

// Multi-word Pascal table C(a, b), 0 <= b <= a < rows, by Pascal's rule,
// one row at a time in a single block.
__global__ void k_binom(unsigned long long *B, int rows, int W, unsigned *err)
{
    for (int a = 0; a < rows; ++a) {
        for (int b = threadIdx.x; b <= a; b += blockDim.x) {
            unsigned long long *dst = B + ((size_t)a * (a + 1) / 2 + b) * W;
            if (b == 0 || b == a) {
                dst[0] = 1;
                for (int w = 1; w < W; ++w) dst[w] = 0;
            } else {
                const unsigned long long *x = B + ((size_t)(a - 1) * a / 2 + b - 1) * W;
                const unsigned long long *y = x + W;
                unsigned long long c = 0;
                for (int w = 0; w < W; ++w) {
                    unsigned long long s1 = x[w] + y[w];
                    unsigned long long c1 = s1 < x[w];
                    unsigned long long s2 = s1 + c;
                    c = c1 + (s2 < s1);
                    dst[w] = s2;
                }
                if (c) atomicOr(err, DERR_OVERFLOW);
            }
        }
        __syncthreads();
    }
}

// C_k = sum over (h, p) of hist[h][p] * C(p, k - h), one block per k, exact.
__global__ void __launch_bounds__(256) k_combine(const unsigned long long *__restrict__ hist,
                                                 int hstride, const unsigned long long *__restrict__ B,
                                                 int W, int kmax, unsigned long long *C, unsigned *err)
{
    __shared__ unsigned long long red[256][WMAX];
    const int k = blockIdx.x;
    unsigned long long acc[WMAX];
#pragma unroll
    for (int w = 0; w < WMAX; ++w) acc[w] = 0;
    bool ovf = false;
    const int pmax = hstride - 2;
    const int hmax = min(k, hstride - 1);
    const int total = hmax * (pmax + 1);  // pairs (h, p), h = 1..hmax
    for (int t = threadIdx.x; t < total; t += blockDim.x) {
        const int h = 1 + t / (pmax + 1), p = t % (pmax + 1);
        const int i = k - h;
        if (i < 0 || i > p) continue;
        const unsigned long long x = hist[(size_t)h * hstride + p];
        if (!x) continue;
        const unsigned long long *b = B + ((size_t)p * (p + 1) / 2 + i) * W;
        unsigned long long carry = 0;
#pragma unroll
        for (int w = 0; w < WMAX; ++w) {
            if (w >= W) break;
            unsigned long long lo = x * b[w], hi = __umul64hi(x, b[w]);
            unsigned long long s1 = acc[w] + lo;
            unsigned long long c1 = s1 < lo;
            unsigned long long s2 = s1 + carry;
            unsigned long long c2 = s2 < s1;
            acc[w] = s2;
            carry = hi + c1 + c2;
        }
        if (carry) ovf = true;
    }
#pragma unroll
    for (int w = 0; w < WMAX; ++w) red[threadIdx.x][w] = acc[w];
    __syncthreads();
    for (int stride = 128; stride > 0; stride >>= 1) {
        if (threadIdx.x < stride) {
            unsigned long long c = 0;
            for (int w = 0; w < W; ++w) {
                unsigned long long x = red[threadIdx.x][w], y = red[threadIdx.x + stride][w];
                unsigned long long s1 = x + y, c1 = s1 < x, s2 = s1 + c;
                c = c1 + (s2 < s1);
                red[threadIdx.x][w] = s2;
            }
            if (c) ovf = true;
        }
        __syncthreads();
    }
    if (threadIdx.x < W) C[(size_t)k * W + threadIdx.x] = red[0][threadIdx.x];
    if (ovf) atomicOr(err, DERR_OVERFLOW);
}

static pvt_status ensure_binom(pvt_dag *g, int W, cudaStream_t s)
{
    // a table with more rows holds this one as its prefix (entry (a, b) sits
    // at (a(a+1)/2 + b) W whatever the row count), so a pooled table is reused
    const int rows = g->alpha + 3;
    if (g->binom_rows >= rows && g->binom_W == W) return PVT_OK;
    pvt_status st = grow(g->binom, (size_t)rows * (rows + 1) / 2 * W, s);
    if (st != PVT_OK) return st;
    k_binom<<<1, 1024, 0, s>>>(g->binom.p, rows, W, g->d_err);
    PVT_CK(cudaGetLastError());
    g->stats.launches++;
    g->binom_rows = rows;
    g->binom_W = W;
    return PVT_OK;
}

// Second phase of a two-phase global count (k_walk_frames, or the lane walk)
// on stream s.
static pvt_status launch_frames(pvt_dag *g, const CountArgs &base, cudaStream_t s)
{
    if (g->policy.lanes) return launch_lanes_frames(g, base, s);
    CountArgs A = base;
    A.cls = FRAMES_SLOT;
    pvt_status st;
    if ((st = grow(g->qframes[0], (size_t)SPLIT_QCAP * FRAME_WORDS, s)) != PVT_OK) return st;
    if ((st = grow(g->qready[0], (size_t)SPLIT_QCAP * 2, s)) != PVT_OK) return st;
    PVT_CK(cudaMemsetAsync(g->qready[0].p, 0, (size_t)SPLIT_QCAP * 2 * sizeof(uint32_t), s));
    k_frames_init<<<1, 128, 0, s>>>(g->qctl, A.emit_count, A.emit_cap);
    PVT_CK(cudaGetLastError());
    A.qframes = g->qframes[0].p;
    A.qready = g->qready[0].p;
    A.qdone = g->qready[0].p + SPLIT_QCAP;
    A.qctl = g->qctl;
    A.qcap = SPLIT_QCAP;
    constexpr size_t smem = sizeof(WarpWork<1>) * FRAME_WPB + sizeof(unsigned long long) * HIST_H * HIST_P;
    auto kern = k_walk_frames<true>;
    PVT_CK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    PVT_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 32 * FRAME_WPB, smem));
    if (per_sm < 1) {
        set_error("frame walk kernel cannot be resident");
        return PVT_ECUDA;
    }
    phase_begin(g, PH_FRAMES, s);
    kern<<<g->num_sms * per_sm, 32 * FRAME_WPB, smem, s>>>(A);
    PVT_CK(cudaGetLastError());
    phase_end(g, PH_FRAMES, s);
    g->stats.launches += 2;
    return PVT_OK;
}

template <int MODE>
static pvt_status launch_all(pvt_dag *g, const CountArgs &A0, cudaStream_t s)
{
    // two-phase global counts: the classes above 32 emit their small labels
    // as frames into cframes (capacity from the number of heavy roots; a
    // full buffer only sends frames back to in-place walking)
    CountArgs A = A0;
    int64_t heavy = 0;
    for (int c = 2; c < NCLASS; ++c) heavy += g->wcnt[c];
    const bool frames = MODE == MODE_GLOBAL && g->policy.frames && g->policy.persistent && heavy > 0;
    if (frames) {
        const unsigned cap = (unsigned)std::min<int64_t>(std::max<int64_t>(64 * heavy, 1 << 16), 1 << 22);
        pvt_status st = grow(g->cframes, (size_t)cap * FRAME_WORDS, s);
        if (st != PVT_OK) return st;
        A.emit = g->cframes.p;
        A.emit_count = reinterpret_cast<unsigned long long *>(g->d_q + 8);  // words 8..9
        A.emit_cap = cap;
    }
    // heavy classes on side streams so that they overlap the light ones (or
    // all on s, one after another, when the autotuner times them)
    const bool serial = g->serial || g->policy.serial;
    if (!serial) PVT_CK(cudaEventRecord(g->ev_fork, s));
    pvt_status st = PVT_OK;
    for (int c = NCLASS - 1; c >= 1 && st == PVT_OK; --c) {
        cudaStream_t cs = serial ? s : g->side[c];
        if (!serial) PVT_CK(cudaStreamWaitEvent(cs, g->ev_fork, 0));
        switch (c) {
            case 1: st = launch_class<1, MODE, MODE == MODE_GLOBAL>(g, A0, c, cs); break;
            case 2: st = launch_class<2, MODE, MODE == MODE_GLOBAL>(g, A, c, cs); break;
            case 4:
            case 5:
            case 6:
                if (MODE == MODE_GLOBAL && g->policy.persistent && g->policy.cta[c]) {
                    st = launch_cta_class(g, A, c, cs);
                    break;
                }
                if (c == 4) st = launch_class<8, MODE, MODE == MODE_GLOBAL>(g, A, c, cs);
                else if (c == 5) st = launch_class<16, MODE, MODE == MODE_GLOBAL>(g, A, c, cs);
                else st = launch_class<32, MODE, MODE == MODE_GLOBAL>(g, A, c, cs);
                break;
            case 3: st = launch_class<4, MODE, MODE == MODE_GLOBAL>(g, A, c, cs); break;
        }
        if (!serial) PVT_CK(cudaEventRecord(g->ev_join[c], cs));
    }
    if (st != PVT_OK) return st;
    if (frames) {
        // the frame walk follows the heavy classes; the <= 32 class may
        // still be running beside it
        if (!serial)
            for (int c = NCLASS - 1; c >= 2; --c) PVT_CK(cudaStreamWaitEvent(s, g->ev_join[c], 0));
        if ((st = launch_frames(g, A, s)) != PVT_OK) return st;
    }
    if (!serial)
        for (int c = NCLASS - 1; c >= 1; --c) PVT_CK(cudaStreamWaitEvent(s, g->ev_join[c], 0));
    return st;
}

static void begin_call(pvt_dag *g)
{
    stats_reset(g);
    // walk every root unless a range call narrows the set
    g->wroots = g->roots;
    for (int c = 0; c < NCLASS; ++c) {
        g->wstart[c] = g->class_start[c];
        g->wcnt[c] = g->class_cnt[c];
    }
    for (int c = 0; c < NCLASS; ++c) g->stats.roots[c] = (uint64_t)g->class_cnt[c];
}

// Copy the walk statistics back, synchronise and check the device status.
// Roots with no out-neighbour are one node and one leaf each (h = 1, p = 0)
// when kmax >= 1; they are tallied without a walk, and counted here.
static pvt_status end_call(pvt_dag *g, cudaStream_t s, const char *fn, int32_t kmax)
{
    PVT_CK(cudaMemcpyAsync(g->h_stats, g->d_stats, (3 + NCLASS + 2) * sizeof(unsigned long long),
                           cudaMemcpyDeviceToHost, s));
    pvt_status st = check_device(g, s, fn);
    const uint64_t trivial = kmax >= 1 ? (uint64_t)g->wcnt[0] : 0;
    g->stats.sct_nodes = g->h_stats[0] + trivial;
    g->stats.sct_leaves = g->h_stats[1] + trivial;
    g->stats.pivot_words = g->h_stats[2];
    for (int c = 0; c < NCLASS; ++c) g->stats.class_words[c] = g->h_stats[3 + c];
    g->stats.frame_words = g->h_stats[3 + FRAMES_SLOT];
    g->stats.frames = g->h_stats[3 + FRAMES_SLOT + 1];
    return st;
}

static pvt_status check_args(pvt_dag *g, int32_t kmax, int32_t W, const void *out, int64_t rows,
                             const char *fn)
{
    if (!g || kmax < 0 || W < 1 || (!out && rows > 0)) {
        set_error(std::string(fn) + ": invalid argument");
        return PVT_EINVAL;
    }
    if (W < min_words(g->n, g->alpha)) {
        set_error(std::string(fn) + ": W=" + std::to_string(W) + " below the required " +
                  std::to_string(min_words(g->n, g->alpha)) + " words");
        return PVT_EOVERFLOW;
    }
    if (W > WMAX) {
        set_error(std::string(fn) + ": W above " + std::to_string(WMAX));
        return PVT_EINVAL;
    }
    return PVT_OK;
}

// Every device operation of a global count, in stream order on s (also the
// sequence recorded into a CUDA graph: no host synchronisation inside).
static pvt_status enqueue_global(pvt_dag *g, int32_t kmax, int32_t W, uint64_t *C, cudaStream_t s)
{
    pvt_status st;
    const int hstride = g->alpha + 2;
    if ((st = grow(g->hist, (size_t)hstride * hstride, s)) != PVT_OK) return st;
    if ((st = ensure_binom(g, W, s)) != PVT_OK) return st;
    PVT_CK(cudaMemsetAsync(g->d_err, 0, sizeof(unsigned), s));
    PVT_CK(cudaMemsetAsync(g->d_q, 0, 16 * sizeof(unsigned), s));
    PVT_CK(cudaMemsetAsync(g->hist.p, 0, (size_t)hstride * hstride * sizeof(unsigned long long), s));
    PVT_CK(cudaMemsetAsync(g->d_stats, 0, 16 * sizeof(unsigned long long), s));
    if (g->class_cnt[0] && kmax >= 1) {
        k_add_leaf<<<1, 32, 0, s>>>(g->hist.p + hstride, (unsigned long long)g->class_cnt[0]);
        PVT_CK(cudaGetLastError());
        g->stats.launches++;
    }
    CountArgs A{};
    A.orow = g->orow;
    A.ocol = g->ocol;
    A.hist = g->hist.p;
    A.hstride = hstride;
    A.B = g->binom.p;
    A.Bw = W;
    A.W = W;
    A.kmax = kmax;
    A.err = g->d_err;
    A.stats = g->d_stats;
    apply_wait_limit(g, A);
    if ((st = launch_all<MODE_GLOBAL>(g, A, s)) != PVT_OK) return st;
    phase_begin(g, PH_FINISH, s);
    if (kmax >= 1) {
        k_check_paths<<<1, 256, 0, s>>>(g->hist.p, hstride, nullptr, (unsigned long long)g->n,
                                        kmax >= 2 ? g->orow : nullptr, g->n, g->d_err);
        PVT_CK(cudaGetLastError());
        g->stats.launches++;
    }
    k_combine<<<kmax + 1, 256, 0, s>>>(g->hist.p, hstride, g->binom.p, W, kmax,
                                       reinterpret_cast<unsigned long long *>(C), g->d_err);
    PVT_CK(cudaGetLastError());
    phase_end(g, PH_FINISH, s);
    g->stats.launches++;
    return PVT_OK;
}

void drop_graph(pvt_dag *g)
{
    if (g->graph_exec) cudaGraphExecDestroy(g->graph_exec);
    g->graph_exec = nullptr;
    g->graph_kmax = -1;
    g->graph_W = 0;
    g->graph_out = nullptr;
    g->graph_launches = 0;
}

// Record the global count for (kmax, W, C) as a graph.  All scratch is sized
// by the direct call that precedes this, so the recorded sequence allocates
// nothing.  Recorded on the dag's own stream side[0] (the caller's stream
// may be the legacy default stream, which cannot be captured).
static pvt_status record_graph(pvt_dag *g, int32_t kmax, int32_t W, uint64_t *C)
{
    drop_graph(g);
    cudaStream_t cs = g->side[0];
    const pvt_stats keep = g->stats;
    g->stats.launches = 0;
    g->capturing = true;
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    pvt_status st = e == cudaSuccess ? enqueue_global(g, kmax, W, C, cs) : cuda_fail(e, "cudaStreamBeginCapture");
    cudaGraph_t graph = nullptr;
    if (e == cudaSuccess) {
        cudaError_t e2 = cudaStreamEndCapture(cs, &graph);
        if (st == PVT_OK && e2 != cudaSuccess) st = cuda_fail(e2, "cudaStreamEndCapture");
    }
    g->capturing = false;
    const uint64_t launches = g->stats.launches;
    g->stats = keep;
    if (st == PVT_OK) {
        e = cudaGraphInstantiate(&g->graph_exec, graph, 0);
        if (e != cudaSuccess) {
            g->graph_exec = nullptr;
            st = cuda_fail(e, "cudaGraphInstantiate");
        }
    }
    if (graph) cudaGraphDestroy(graph);
    if (st != PVT_OK) {
        drop_graph(g);
        return st;
    }
    g->graph_kmax = kmax;
    g->graph_W = W;
    g->graph_out = C;
    g->graph_launches = launches;
    return PVT_OK;
}

pvt_status count_global(pvt_dag *g, int32_t kmax, int32_t W, uint64_t *C, cudaStream_t s)
{
    pvt_status st = check_args(g, kmax, W, C, 1, "pvt_count_global");
    if (st != PVT_OK) return st;
    begin_call(g);
    const bool use_graph = g->policy.graph != 0 && !g->serial && !g->policy.serial;
    g->hist_valid = false;
    if (use_graph && g->graph_exec && g->graph_kmax == kmax && g->graph_W == W && g->graph_out == C) {
        PVT_CK(cudaGraphLaunch(g->graph_exec, s));
        g->stats.launches = g->graph_launches;
        st = end_call(g, s, "pvt_count_global", kmax);
        g->hist_valid = st == PVT_OK;
        return st;
    }
    if ((st = enqueue_global(g, kmax, W, C, s)) != PVT_OK) return st;
    if ((st = end_call(g, s, "pvt_count_global", kmax)) != PVT_OK) return st;
    g->hist_valid = true;
    return use_graph ? record_graph(g, kmax, W, C) : PVT_OK;
}

// Leaves by depth d = h + p (links on the root-to-leaf path) from the (h, p)
// histogram: out[d] = sum over h of hist[h][d - h], d = 0..H-1.  A leaf
// deeper than H-1 (impossible: a path's links form a clique of at most
// alpha + 1 vertices) is a range error.
__global__ void __launch_bounds__(256) k_leaf_depths(const unsigned long long *__restrict__ hist, int H,
                                                     unsigned long long *out, unsigned *err)
{
    for (int d = threadIdx.x; d <= 2 * (H - 1); d += blockDim.x) {
        unsigned long long a = 0;
        for (int h = max(0, d - (H - 1)); h <= min(d, H - 1); ++h) a += hist[(size_t)h * H + (d - h)];
        if (d < H) out[d] = a;
        else if (a) atomicOr(err, DERR_RANGE);
    }
}

pvt_status leaf_depths(pvt_dag *g, uint64_t *depth, cudaStream_t s)
{
    if (!g || !depth) {
        set_error("pvt_dag_leaf_depths: invalid argument");
        return PVT_EINVAL;
    }
    if (!g->hist_valid) {
        set_error("pvt_dag_leaf_depths: no completed pvt_count_global on this dag");
        return PVT_EINVAL;
    }
    const int H = g->alpha + 2;
    unsigned long long *d_out = nullptr;
    PVT_CK(cudaMallocAsync(&d_out, (size_t)H * sizeof(unsigned long long), s));
    PVT_CK(cudaMemsetAsync(g->d_err, 0, sizeof(unsigned), s));
    k_leaf_depths<<<1, 256, 0, s>>>(g->hist.p, H, d_out, g->d_err);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(depth, d_out, (size_t)H * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s);
    cudaFreeAsync(d_out, s);
    if (e != cudaSuccess) return cuda_fail(e, "pvt_dag_leaf_depths");
    return check_device(g, s, "pvt_dag_leaf_depths");
}

// ------------------------------------------- root ranges and checkpoints

struct ClassBounds {
    int64_t start[NCLASS], cnt[NCLASS];
};

__global__ void k_range_flags(const uint32_t *__restrict__ roots, int64_t n, int64_t begin, int64_t end,
                              uint32_t *flag)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        flag[i] = roots[i] >= (uint64_t)begin && roots[i] < (uint64_t)end;
}

__global__ void k_range_scatter(const uint32_t *__restrict__ roots, int64_t n, const uint32_t *__restrict__ flag,
                                const int64_t *__restrict__ pos, uint32_t *out)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        if (flag[i]) out[pos[i]] = roots[i];
}

// Start and length of each class inside the compacted range.
__global__ void k_range_bounds(const int64_t *__restrict__ pos, ClassBounds full, int64_t *out)
{
    const int c = threadIdx.x;
    if (c < NCLASS) {
        const int64_t a = pos[full.start[c]], b = pos[full.start[c] + full.cnt[c]];
        out[c] = a;
        out[NCLASS + c] = b - a;
    }
}

pvt_status count_hist(pvt_dag *g, int64_t begin, int64_t end, int32_t kmax, uint64_t *hist, cudaStream_t s)
{
    if (!g || !hist || kmax < 0 || begin < 0 || end < begin) {
        set_error("pvt_count_hist: invalid argument");
        return PVT_EINVAL;
    }
    begin_call(g);
    const int64_t n = g->n;
    end = std::min(end, n);
    begin = std::min(begin, end);
    pvt_status st;
    if (n > 0) {
        // the range's roots, class by class in the order of g->roots
        if ((st = grow(g->range_roots, (size_t)2 * n, s)) != PVT_OK) return st;
        if ((st = grow(g->range_pos, (size_t)n + 1, s)) != PVT_OK) return st;
        uint32_t *flag = g->range_roots.p, *out = g->range_roots.p + n;
        const int grid = g->num_sms * 4;
        k_range_flags<<<grid, 256, 0, s>>>(g->roots, n, begin, end, flag);
        PVT_CK(cudaGetLastError());
        if ((st = exclusive_scan_u32_i64(flag, g->range_pos.p, n, s)) != PVT_OK) return st;
        k_range_scatter<<<grid, 256, 0, s>>>(g->roots, n, flag, g->range_pos.p, out);
        ClassBounds full{};
        for (int c = 0; c < NCLASS; ++c) {
            full.start[c] = g->class_start[c];
            full.cnt[c] = g->class_cnt[c];
        }
        int64_t *d_b = reinterpret_cast<int64_t *>(flag);  // flags are spent; reuse their words
        k_range_bounds<<<1, 32, 0, s>>>(g->range_pos.p, full, d_b);
        PVT_CK(cudaGetLastError());
        int64_t hb[2 * NCLASS];
        PVT_CK(cudaMemcpyAsync(hb, d_b, sizeof(hb), cudaMemcpyDeviceToHost, s));
        PVT_CK(cudaStreamSynchronize(s));
        g->wroots = out;
        for (int c = 0; c < NCLASS; ++c) {
            g->wstart[c] = hb[c];
            g->wcnt[c] = hb[NCLASS + c];
            g->stats.roots[c] = (uint64_t)hb[NCLASS + c];
        }
        g->stats.launches += 7;
    }
    const int hstride = g->alpha + 2;
    PVT_CK(cudaMemsetAsync(g->d_err, 0, sizeof(unsigned), s));
    PVT_CK(cudaMemsetAsync(g->d_q, 0, 16 * sizeof(unsigned), s));
    PVT_CK(cudaMemsetAsync(g->d_stats, 0, 16 * sizeof(unsigned long long), s));
    // row 1 of the caller's histogram before this range adds to it
    unsigned long long *row1_base = g->d_stats + 14;
    if (kmax >= 1) {
        k_row1_sum<<<1, 256, 0, s>>>(reinterpret_cast<const unsigned long long *>(hist), hstride, row1_base);
        PVT_CK(cudaGetLastError());
        g->stats.launches++;
    }
    if (g->wcnt[0] && kmax >= 1) {
        k_add_leaf<<<1, 32, 0, s>>>(reinterpret_cast<unsigned long long *>(hist) + hstride,
                                    (unsigned long long)g->wcnt[0]);
        PVT_CK(cudaGetLastError());
        g->stats.launches++;
    }
    CountArgs A{};
    A.orow = g->orow;
    A.ocol = g->ocol;
    A.hist = reinterpret_cast<unsigned long long *>(hist);
    A.hstride = hstride;
    A.W = 1;
    A.Bw = 1;
    A.kmax = kmax;
    A.err = g->d_err;
    A.stats = g->d_stats;
    apply_wait_limit(g, A);
    if ((st = launch_all<MODE_GLOBAL>(g, A, s)) != PVT_OK) return st;
    if (kmax >= 1) {
        int64_t walked = 0;
        for (int c = 0; c < NCLASS; ++c) walked += g->wcnt[c];
        k_check_paths<<<1, 256, 0, s>>>(A.hist, hstride, row1_base, (unsigned long long)walked, nullptr, 0,
                                        g->d_err);
        PVT_CK(cudaGetLastError());
        g->stats.launches++;
    }
    return end_call(g, s, "pvt_count_hist", kmax);
}

pvt_status combine_hist(pvt_dag *g, const uint64_t *hist, int32_t kmax, int32_t W, uint64_t *C, cudaStream_t s)
{
    pvt_status st = check_args(g, kmax, W, C, 1, "pvt_combine_hist");
    if (st != PVT_OK) return st;
    if (!hist) {
        set_error("pvt_combine_hist: invalid argument");
        return PVT_EINVAL;
    }
    begin_call(g);
    if ((st = ensure_binom(g, W, s)) != PVT_OK) return st;
    PVT_CK(cudaMemsetAsync(g->d_err, 0, sizeof(unsigned), s));
    PVT_CK(cudaMemsetAsync(g->d_stats, 0, 16 * sizeof(unsigned long long), s));
    k_combine<<<kmax + 1, 256, 0, s>>>(reinterpret_cast<const unsigned long long *>(hist), g->alpha + 2, g->binom.p,
                                       W, kmax, reinterpret_cast<unsigned long long *>(C), g->d_err);
    PVT_CK(cudaGetLastError());
    g->stats.launches++;
    return end_call(g, s, "pvt_combine_hist", -1);
}

// Per-class minimum over three candidate policies, classes timed one at a time.
pvt_status autotune(pvt_dag *g, int32_t kmax, int32_t W, uint64_t *C, cudaStream_t s, pvt_policy *chosen,
                    float *ms)
{
    if (!g || !chosen) {
        set_error("pvt_dag_autotune: invalid argument");
        return PVT_EINVAL;
    }
    static const pvt_policy cand[3] = {
        {1, 4, {0, 0, 1, 1, 1, 1, 1}, 0, 1, 0, 1, {0, 0, 0, 0, 0, 0, 0}, 0},
        {1, 1, {0, 0, 0, 0, 0, 0, 0}, 0, 1, 0, 1, {0, 0, 0, 0, 1, 1, 1}, 0},
        {1, 16, {0, 0, 1, 1, 1, 1, 1}, 0, 1, 0, 1, {0, 0, 0, 0, 0, 0, 0}, 0},
    };
    const pvt_policy saved = g->policy;
    const bool saved_prof = g->profiling;
    float t[3][NCLASS] = {};
    pvt_status st = PVT_OK;
    drop_graph(g);
    g->serial = true;
    g->profiling = true;
    for (int pass = 0; pass < 2 && st == PVT_OK; ++pass)
        for (int c = 0; c < 3 && st == PVT_OK; ++c) {
            g->policy = cand[c];
            g->policy.wait_limit_us = saved.wait_limit_us;
            g->policy.lanes = saved.lanes;
            st = count_global(g, kmax, W, C, s);
            for (int cls = 1; st == PVT_OK && cls < NCLASS; ++cls) {
                float x = 0.f;
                if (g->phase_used[1 + cls] &&
                    cudaEventElapsedTime(&x, g->ev_t0[1 + cls], g->ev_t1[1 + cls]) == cudaSuccess)
                    t[c][cls] = x;
            }
        }
    g->serial = false;
    g->profiling = saved_prof;
    g->policy = saved;
    if (st != PVT_OK) return st;
    pvt_policy best = saved;
    int bc = 0;
    for (int c = 1; c < 3; ++c)
        if (t[c][1] < t[bc][1]) bc = c;
    best.chunk = cand[bc].chunk;
    for (int cls = 0; cls < NCLASS; ++cls) {
        best.cta[cls] = 0;
        if (cls < 2) { best.split[cls] = 0; continue; }
        // candidate 1 walks the classes above 128 a block per root, the
        // classes below a warp per root without splitting
        const float with = std::min(t[0][cls], t[2][cls]);
        if (t[1][cls] < with) {
            best.split[cls] = 0;
            best.cta[cls] = cls >= 4 ? 1 : 0;
        } else {
            best.split[cls] = 1;
        }
    }
    g->policy = best;
    *chosen = best;
    if (ms)
        for (int c = 0; c < 3; ++c)
            for (int cls = 0; cls < NCLASS; ++cls) ms[c * NCLASS + cls] = t[c][cls];
    return PVT_OK;
}

pvt_status count_local(pvt_dag *g, int32_t kmax, int32_t W, uint64_t *out, bool edge, cudaStream_t s)
{
    const char *fn = edge ? "pvt_count_local_edge" : "pvt_count_local_vertex";
    pvt_status st = check_args(g, kmax, W, out, g ? (edge ? g->m : g->n) : 0, fn);
    if (st != PVT_OK) return st;
    begin_call(g);
    if (edge && !g->oeid) {
        if ((st = ensure_edge_ids(g, s)) != PVT_OK) return st;
        g->stats.launches += 5;
    }
    if ((st = ensure_binom(g, W, s)) != PVT_OK) return st;
    const int64_t rows = edge ? g->m : g->n;
    PVT_CK(cudaMemsetAsync(g->d_err, 0, sizeof(unsigned), s));
    PVT_CK(cudaMemsetAsync(g->d_q, 0, 16 * sizeof(unsigned), s));
    if (rows > 0) PVT_CK(cudaMemsetAsync(out, 0, (size_t)rows * (kmax + 1) * W * sizeof(uint64_t), s));
    PVT_CK(cudaMemsetAsync(g->d_stats, 0, 16 * sizeof(unsigned long long), s));
    unsigned long long *o = reinterpret_cast<unsigned long long *>(out);
    if (!edge && g->class_cnt[0] && kmax >= 1) {
        k_vertex_trivial<<<g->num_sms * 4, 256, 0, s>>>(g->roots + g->class_start[0],
                                                       (unsigned)g->class_cnt[0], o, kmax + 1, W);
        g->stats.launches++;
    }
    CountArgs A{};
    A.orow = g->orow;
    A.ocol = g->ocol;
    A.oeid = g->oeid;
    A.out = o;
    A.B = g->binom.p;
    A.Bw = W;
    A.W = W;
    A.kmax = kmax;
    A.err = g->d_err;
    A.stats = g->d_stats;
    apply_wait_limit(g, A);
    st = edge ? launch_all<MODE_EDGE>(g, A, s) : launch_all<MODE_VERTEX>(g, A, s);
    if (st != PVT_OK) return st;
    return end_call(g, s, fn, kmax);
}


}  // namespace pvt

namespace pvt {
// Root entries of every graph of a batch, per (query kind, class):
// dst[mode][class][off[g][class] + i] = (g << 32) | roots[start + i].
__global__ void k_batch_entries(const BatchGraph *gs, uint64_t *const *dst, const unsigned *off)
{
    const int g = blockIdx.y;
    const BatchGraph &G = gs[g];
    const unsigned *start = G.info + BI_START, *cnt = G.info + BI_CNT;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < G.n; i += (int64_t)gridDim.x * blockDim.x) {
        int c = 0;
        while (c < NCLASS && !(i >= start[c] && i < start[c] + cnt[c])) ++c;
        if (c == NCLASS) continue;
        dst[G.mode * NCLASS + c][off[g * NCLASS + c] + (i - start[c])] = ((uint64_t)g << 32) | G.roots[i];
    }
}

// Global counts of the batch's global queries: one block per (graph, k).
__global__ void __launch_bounds__(256) k_combine_batch(const BatchGraph *gs, const int2 *work,
                                                       const unsigned long long *__restrict__ B, int Bw,
                                                       unsigned *err)
{
    __shared__ unsigned long long red[256][WMAX];
    const int2 wk = work[blockIdx.x];
    const BatchGraph &G = gs[wk.x];
    const int k = wk.y, W = G.W, hstride = G.hstride;
    const unsigned long long *hist = G.hist;
    unsigned long long acc[WMAX];
#pragma unroll
    for (int w = 0; w < WMAX; ++w) acc[w] = 0;
    bool ovf = false;
    const int pmax = hstride - 2;
    const int hmax = min(k, hstride - 1);
    const int total = hmax * (pmax + 1);
    for (int t = threadIdx.x; t < total; t += blockDim.x) {
        const int h = 1 + t / (pmax + 1), p = t % (pmax + 1);
        const int i = k - h;
        if (i < 0 || i > p) continue;
        const unsigned long long x = hist[(size_t)h * hstride + p];
        if (!x) continue;
        const unsigned long long *b = B + ((size_t)p * (p + 1) / 2 + i) * Bw;
        unsigned long long carry = 0;
#pragma unroll
        for (int w = 0; w < WMAX; ++w) {
            if (w >= W) break;
            unsigned long long lo = x * b[w], hi = __umul64hi(x, b[w]);
            unsigned long long s1 = acc[w] + lo;
            unsigned long long c1 = s1 < lo;
            unsigned long long s2 = s1 + carry;
            unsigned long long c2 = s2 < s1;
            acc[w] = s2;
            carry = hi + c1 + c2;
        }
        if (carry) ovf = true;
    }
#pragma unroll
    for (int w = 0; w < WMAX; ++w) red[threadIdx.x][w] = acc[w];
    __syncthreads();
    for (int stride = 128; stride > 0; stride >>= 1) {
        if (threadIdx.x < stride) {
            unsigned long long c = 0;
            for (int w = 0; w < W; ++w) {
                unsigned long long x = red[threadIdx.x][w], y = red[threadIdx.x + stride][w];
                unsigned long long s1 = x + y, c1 = s1 < x, s2 = s1 + c;
                c = c1 + (s2 < s1);
                red[threadIdx.x][w] = s2;
            }
            if (c) ovf = true;
        }
        __syncthreads();
    }
    if (threadIdx.x < W) G.out[(size_t)k * W + threadIdx.x] = red[0][threadIdx.x];
    if (ovf) atomicOr(err, DERR_OVERFLOW);
}

pvt_status batch_root_entries(BatchGraph *d_graphs, int count, uint64_t *const *d_entries,
                              const unsigned *d_class_offsets, cudaStream_t s)
{
    if (count <= 0) return PVT_OK;
    k_batch_entries<<<dim3(8, count), 256, 0, s>>>(d_graphs, d_entries, d_class_offsets);
    PVT_CK(cudaGetLastError());
    return PVT_OK;
}

template <int MODE>
static pvt_status launch_batch_mode(const BatchGraph *gs, const uint64_t *const *h_entries, const unsigned *n_entries,
                                    const unsigned long long *B, int Bw, unsigned *ctl, int num_sms, cudaStream_t s)
{
    pvt_status st = PVT_OK;
    for (int c = NCLASS - 1; c >= 0 && st == PVT_OK; --c) {
        const unsigned cnt = n_entries[MODE * NCLASS + c];
        if (!cnt) continue;
        const uint64_t *e = h_entries[MODE * NCLASS + c];
        unsigned *qhead = ctl + 1 + MODE * NCLASS + c;
        unsigned *err = ctl;
        unsigned long long *stats = reinterpret_cast<unsigned long long *>(ctl + 32);
        switch (c) {
            case 0:
            case 1: st = launch_batch_class<1, MODE>(gs, e, cnt, qhead, B, Bw, err, stats, num_sms, s); break;
            case 2: st = launch_batch_class<2, MODE>(gs, e, cnt, qhead, B, Bw, err, stats, num_sms, s); break;
            case 3: st = launch_batch_class<4, MODE>(gs, e, cnt, qhead, B, Bw, err, stats, num_sms, s); break;
            case 4: st = launch_batch_class<8, MODE>(gs, e, cnt, qhead, B, Bw, err, stats, num_sms, s); break;
            case 5: st = launch_batch_class<16, MODE>(gs, e, cnt, qhead, B, Bw, err, stats, num_sms, s); break;
            default: set_error("batched walk: out-degree above the batched limit"); st = PVT_EINVAL; break;
        }
    }
    return st;
}

// ctl (device): [0] status word, [1 + mode*NCLASS + class] queue heads,
// [32..] 64-bit walk statistics; zeroed by the caller.
pvt_status batch_count(BatchGraph *d_graphs, int count, const int2 *d_combine_work, int n_combine,
                       const uint64_t *const *h_entries, const unsigned *n_entries,
                       const unsigned long long *d_binom, int binom_stride, int num_sms, unsigned *d_ctl,
                       cudaStream_t s)
{
    if (count <= 0) return PVT_OK;
    pvt_status st;
    if ((st = launch_batch_mode<MODE_GLOBAL>(d_graphs, h_entries, n_entries, d_binom, binom_stride, d_ctl, num_sms, s)) != PVT_OK) return st;
    if ((st = launch_batch_mode<MODE_VERTEX>(d_graphs, h_entries, n_entries, d_binom, binom_stride, d_ctl, num_sms, s)) != PVT_OK) return st;
    if ((st = launch_batch_mode<MODE_EDGE>(d_graphs, h_entries, n_entries, d_binom, binom_stride, d_ctl, num_sms, s)) != PVT_OK) return st;
    if (n_combine > 0) {
        k_combine_batch<<<n_combine, 256, 0, s>>>(d_graphs, d_combine_work, d_binom, binom_stride, d_ctl);
        PVT_CK(cudaGetLastError());
    }
    return PVT_OK;
}

// Multi-word Pascal table into caller memory (rows x rows/2 entries of W words).
pvt_status build_binom(unsigned long long *B, int rows, int W, unsigned *err, cudaStream_t s)
{
    k_binom<<<1, 1024, 0, s>>>(B, rows, W, err);
    PVT_CK(cudaGetLastError());
    return PVT_OK;
}

// ------------------------------------------- allocation-free global count
//
// Some callers cannot allocate device memory when they count: code running
// inside a pre-sized memory arena or a framework whose allocator is not
// reachable from C, callers that forbid allocation on their latency path, or
// contexts in which a cudaMalloc could block on other work or fail under
// fragmentation.  pvt_count_global_noalloc serves them: the caller passes an
// already oriented graph and the output buffer, and every piece of scratch
// the walk needs (the (h, p) leaf histogram, the multi-word Pascal table,
// the work-queue head and the status word) lives in the fixed device array
// below, which the library holds on every GPU that loads it until the
// process exits.

constexpr int NOALLOC_MAX_ALPHA = 126;  // largest out-degree (bitsets of <= 4 words)
constexpr int NOALLOC_MAX_W = 4;        // largest W (64-bit words per count)
constexpr size_t NOALLOC_HIST = (size_t)(NOALLOC_MAX_ALPHA + 2) * (NOALLOC_MAX_ALPHA + 2);
constexpr size_t NOALLOC_BINOM = (size_t)(NOALLOC_MAX_ALPHA + 3) * (NOALLOC_MAX_ALPHA + 4) / 2 * NOALLOC_MAX_W;
constexpr size_t NOALLOC_CTL = 32;      // [0] queue head + status word, [1..] walk statistics
constexpr size_t NOALLOC_WORDS = NOALLOC_HIST + NOALLOC_BINOM + NOALLOC_CTL;  // 400 KB in all

static __device__ __align__(256) unsigned long long g_noalloc_scratch[NOALLOC_WORDS];

// Every vertex is a root; out-degrees above `alpha` are refused (they would
// index outside the histogram).  Same walk as k_count, global counts.
template <int NW>
__global__ void __launch_bounds__(32 * warps_per_block<NW>()) k_count_noalloc(CountArgs A, int alpha)
{
    constexpr int WPB = warps_per_block<NW>();
    extern __shared__ __align__(16) unsigned char smem[];
    WarpWork<NW> *ww = reinterpret_cast<WarpWork<NW> *>(smem);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    WalkCounters wc;
    for (;;) {
        unsigned qi = 0;
        if (lane == 0) qi = atomicAdd(A.qhead, 1u);
        qi = __shfl_sync(FULL, qi, 0);
        if (qi >= A.nroots) break;
        const int64_t d = A.orow[qi + 1] - A.orow[qi];
        if (d < 0 || d > alpha) {
            if (lane == 0) atomicOr(A.err, DERR_RANGE);
            break;
        }
        walk_root<NW, MODE_GLOBAL, false, false>(ww[wid], nullptr, A, lane, qi, wc);
        wc.fold();
        if (vload(A.err) & (DERR_STACK | DERR_RANGE)) break;
    }
    (void)WPB;
    wc.flush(A.stats, -1, lane);
}

template <int NW>
static pvt_status launch_noalloc(const CountArgs &A, int alpha, int num_sms, cudaStream_t s)
{
    constexpr size_t smem = sizeof(WarpWork<NW>) * warps_per_block<NW>();
    auto kern = k_count_noalloc<NW>;
    PVT_CK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    PVT_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 32 * warps_per_block<NW>(), smem));
    if (per_sm < 1) {
        set_error("pvt_count_global_noalloc: walk kernel cannot be resident");
        return PVT_ECUDA;
    }
    const unsigned need = (A.nroots + warps_per_block<NW>() - 1) / warps_per_block<NW>();
    const unsigned grid = std::max(1u, std::min<unsigned>((unsigned)(num_sms * per_sm), need));
    kern<<<grid, 32 * warps_per_block<NW>(), smem, s>>>(A, alpha);
    PVT_CK(cudaGetLastError());
    return PVT_OK;
}

}  // namespace pvt

extern "C" pvt_status pvt_count_global_noalloc(int64_t n, const int64_t *orow, const uint32_t *ocol,
                                               int32_t alpha, int32_t kmax, int32_t W, uint64_t *C,
                                               void *stream)
{
    const pvt::HostRange range("pvt_count_global_noalloc");
    using namespace pvt;
    if (n < 0 || n > 0xFFFFFFFEll || (n > 0 && (!orow || !ocol)) || !C || kmax < 0 || alpha < 0 || W < 1) {
        set_error("pvt_count_global_noalloc: invalid argument");
        return PVT_EINVAL;
    }
    if (alpha > NOALLOC_MAX_ALPHA || W > NOALLOC_MAX_W) {
        set_error("pvt_count_global_noalloc: alpha <= " + std::to_string(NOALLOC_MAX_ALPHA) + " and W <= " +
                  std::to_string(NOALLOC_MAX_W) + " required (fixed scratch)");
        return PVT_EINVAL;
    }
    if (W < min_words(n, alpha)) {
        set_error("pvt_count_global_noalloc: W below the required " + std::to_string(min_words(n, alpha)));
        return PVT_EOVERFLOW;
    }
    // once per device, with that device current: the device address of the
    // scratch array (its host-side name is only a stand-in)
    static std::mutex mu;
    static void *scratch_of[64] = {};
    static int sms_of[64] = {};
    int dev = 0;
    PVT_CK(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) {
        set_error("pvt_count_global_noalloc: device index above 63");
        return PVT_EINVAL;
    }
    void *base = nullptr;
    int num_sms = 0;
    {
        std::lock_guard<std::mutex> lock(mu);
        if (!scratch_of[dev]) {
            void *ptr = nullptr;
            PVT_CK(cudaGetSymbolAddress(&ptr, g_noalloc_scratch));
            int sms = 0;
            PVT_CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
            scratch_of[dev] = ptr;
            sms_of[dev] = sms;
        }
        base = scratch_of[dev];
        num_sms = sms_of[dev];
    }
    cudaStream_t s = (cudaStream_t)stream;
    unsigned long long *hist = static_cast<unsigned long long *>(base);
    unsigned long long *binom = hist + NOALLOC_HIST;
    unsigned long long *ctl = binom + NOALLOC_BINOM;
    unsigned *qhead = reinterpret_cast<unsigned *>(ctl);
    unsigned *err = qhead + 1;
    const int hstride = alpha + 2;
    // the array keeps the previous call's contents: clear what must start at zero
    PVT_CK(cudaMemsetAsync(hist, 0, (size_t)hstride * hstride * sizeof(unsigned long long), s));
    PVT_CK(cudaMemsetAsync(ctl, 0, NOALLOC_CTL * sizeof(unsigned long long), s));
    k_binom<<<1, 1024, 0, s>>>(binom, alpha + 3, W, err);
    PVT_CK(cudaGetLastError());
    if (n > 0) {
        CountArgs A{};
        A.orow = orow;
        A.ocol = ocol;
        A.nroots = (unsigned)n;
        A.qhead = qhead;
        A.hist = hist;
        A.hstride = hstride;
        A.B = binom;
        A.Bw = W;
        A.W = W;
        A.kmax = kmax;
        A.err = err;
        A.stats = ctl + 1;
        const int NWn = (alpha + 31) / 32;
        pvt_status st = NWn <= 1 ? launch_noalloc<1>(A, alpha, num_sms, s)
                        : NWn <= 2 ? launch_noalloc<2>(A, alpha, num_sms, s)
                                   : launch_noalloc<4>(A, alpha, num_sms, s);
        if (st != PVT_OK) return st;
        k_check_paths<<<1, 256, 0, s>>>(hist, hstride, nullptr, (unsigned long long)n, kmax >= 2 ? orow : nullptr, n,
                                        err);
        PVT_CK(cudaGetLastError());
    }
    k_combine<<<kmax + 1, 256, 0, s>>>(hist, hstride, binom, W, kmax, reinterpret_cast<unsigned long long *>(C), err);
    PVT_CK(cudaGetLastError());
    unsigned herr = 0;
    PVT_CK(cudaMemcpyAsync(&herr, err, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
    PVT_CK(cudaStreamSynchronize(s));
    if (herr & DERR_RANGE) {
        set_error("pvt_count_global_noalloc: an out-degree exceeds alpha");
        return PVT_EINVAL;
    }
    if (herr & DERR_OVERFLOW) {
        set_error("pvt_count_global_noalloc: multi-word overflow");
        return PVT_EOVERFLOW;
    }
    if (herr & DERR_CHECK) {
        set_error("pvt_count_global_noalloc: internal consistency check of the root paths failed");
        return PVT_EINTERNAL;
    }
    if (herr) {
        set_error("pvt_count_global_noalloc: device capacity check failed");
        return PVT_EINTERNAL;
    }
    return PVT_OK;
}
