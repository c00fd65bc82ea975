// Internal definitions shared by the CUDA translation units of libpivoter.
#pragma once

#include <nvtx3/nvToolsExt.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "pivoter.h"

namespace pvt {

constexpr unsigned FULL = 0xFFFFFFFFu;
constexpr uint32_t NOT_REMOVED = 0xFFFFFFFFu;

// Root classes by out-degree d = |N+(r)|: class 0 holds d = 0, class c >= 1
// holds 32 * 2^(c-2) < d <= 32 * 2^(c-1), i.e. bitsets of NW = 2^(c-1) words.
constexpr int NCLASS = 7;              // d = 0, <=32, <=64, <=128, <=256, <=512, <=1024
constexpr int MAX_ALPHA = 1024;        // largest degeneracy (out-degree) supported
constexpr int BATCH_MAX_ALPHA = 512;   // largest degeneracy of a served (batched) graph
constexpr int NPHASE = NCLASS + 3;     // peel, orient, one walk per class >= 1, finish, frame walk
constexpr int PH_FINISH = NCLASS + 1, PH_FRAMES = NCLASS + 2;
constexpr int WMAX = 20;               // largest W (64-bit words per count) supported

// Device-side error bits (one 32-bit status word per dag).
enum : unsigned {
    DERR_STACK = 1u,      // explicit DFS stack would overflow (capacity bug)
    DERR_TIMEOUT = 2u,    // bounded spin-wait gave up
    DERR_OVERFLOW = 4u,   // multi-word arithmetic carried out of the top word
    DERR_RANGE = 8u,      // an index fell outside its table (capacity bug)
    DERR_NOTSIMPLE = 16u,  // CSR validation failed
    DERR_CHECK = 32u       // a walk's leaf histogram disagrees with its root paths
};

// Per-call scratch that lives as long as the dag (grown on demand).
template <typename T>
struct DevBuf {
    T *p = nullptr;
    size_t n = 0;
};

}  // namespace pvt

struct pvt_dag {
    int device = 0;
    int num_sms = 0;
    int64_t n = 0, m = 0, nnz = 0;
    int32_t alpha = 0;
    const int64_t *row_ptr = nullptr;  // borrowed undirected CSR
    const uint32_t *col = nullptr;
    // owned device state
    uint32_t *rnd = nullptr;       // peel round of each vertex (orientation key high part)
    uint32_t *core = nullptr;      // peel level (core number) of each vertex
    int64_t *orow = nullptr;       // DAG CSR row pointers, int64[n+1]
    uint32_t *ocol = nullptr;      // DAG out-neighbours, sorted by id, uint32[m]
    uint32_t *oeid = nullptr;      // edge id of each out-edge (built on first use)
    uint32_t *roots = nullptr;     // roots grouped by class, descending out-degree
    int64_t class_start[pvt::NCLASS] = {0};  // first position of each class in roots
    int64_t class_cnt[pvt::NCLASS] = {0};
    // the roots a count walks: every root (wroots = roots) or a range of them
    // (pvt_count_hist), grouped by class the same way
    const uint32_t *wroots = nullptr;
    int64_t wstart[pvt::NCLASS] = {0}, wcnt[pvt::NCLASS] = {0};
    pvt::DevBuf<uint32_t> range_roots;  // roots of the last range, and its scan
    pvt::DevBuf<int64_t> range_pos;
    unsigned *d_err = nullptr;     // device status word
    unsigned *d_q = nullptr;       // work-queue heads [16]
    unsigned *h_err = nullptr;     // pinned host copy of the status word
    pvt::DevBuf<unsigned long long> hist;   // (h, p) leaf histogram
    // subtree splitting of heavy classes: published root adjacency, frame
    // queue, ready flags and queue counters, one set per class
    pvt::DevBuf<uint32_t> rootbuf[pvt::NCLASS], qframes[pvt::NCLASS], qready[pvt::NCLASS];
    uint32_t *qctl = nullptr;                 // [NCLASS][128] queue counters
    pvt::DevBuf<unsigned long long> binom;  // multi-word Pascal table
    int binom_rows = 0, binom_W = 0;
    cudaStream_t side[pvt::NCLASS] = {};    // per-class streams for concurrent launches
    cudaEvent_t ev_fork = nullptr, ev_join[pvt::NCLASS] = {};
    // statistics and phase timing of the last call
    unsigned long long *d_stats = nullptr;  // [0] nodes, [1] leaves, [2] pivot words
    unsigned long long *h_stats = nullptr;  // pinned host copy
    pvt_stats stats = {};
    bool profiling = false;
    pvt_policy policy = {1, 4, {0, 0, 1, 1, 1, 1, 1}, 0, 1, 0, 1, {0, 0, 0, 0, 0, 1, 1}, 0};
    pvt::DevBuf<uint32_t> cframes;  // compacted frames emitted by the wide walks
    bool serial = false;           // launch the classes one after another on the caller's stream
    bool capturing = false;        // recording a CUDA graph: no phase events
    cudaGraphExec_t graph_exec = nullptr;  // recorded global count (policy.graph)
    int graph_kmax = -1, graph_W = 0;
    void *graph_out = nullptr;
    uint64_t graph_launches = 0;
    cudaEvent_t ev_t0[pvt::NPHASE] = {}, ev_t1[pvt::NPHASE] = {};
    bool phase_used[pvt::NPHASE] = {};
    pvt::DevBuf<uint32_t> gstack[pvt::NCLASS];  // DFS stacks of the wide classes (global memory)
    pvt::DevBuf<uint32_t> etab[pvt::NCLASS];    // per-warp member-pair edge ids (per-edge counts)
    bool hist_valid = false;       // hist holds the leaves of the last completed global count
};

namespace pvt {

// One graph of a batched launch: a device-resident descriptor filled by the
// host, completed by the batched orient kernel (one block per graph).
enum BatchMode : int { BATCH_GLOBAL = 0, BATCH_VERTEX = 1, BATCH_EDGE = 2 };
enum BatchInfo : int { BI_ALPHA = 0, BI_ERR = 1, BI_CNT = 2, BI_START = 9 };  // info[] slots
struct BatchGraph {
    int64_t n = 0, nnz = 0;
    const int64_t *rp = nullptr;      // undirected CSR
    const uint32_t *col = nullptr;
    uint32_t *deg = nullptr, *rnd = nullptr, *lq = nullptr, *tmp = nullptr;  // scratch: n, n, n, 2n
    int64_t *orow = nullptr;          // DAG
    uint32_t *ocol = nullptr;
    uint32_t *oeid = nullptr;         // per-edge queries only
    int64_t *up = nullptr;            //   (n+1 scratch for edge ids)
    uint32_t *roots = nullptr;        // n, grouped by class, out-degree descending
    uint32_t info[16] = {};           // alpha, status, class counts [2..8], class starts [9..15]
    unsigned long long *hist = nullptr;  // global queries: (h, p) histogram
    int hstride = 0;
    unsigned long long *out = nullptr;   // result: C [K][W], or table [rows][K][W]
    int mode = BATCH_GLOBAL;
    int kmax = 0, W = 1;
};

// Batched orientation: one block per graph (peel, DAG CSR, edge ids for
// per-edge queries, root classes) for `count` device descriptors.
pvt_status batch_orient(BatchGraph *d_graphs, int count, cudaStream_t s);
// Batched walk of the root entries h_entries[mode * NCLASS + class] (device
// arrays of (graph << 32 | root), n_entries each) and the combine of the
// global queries (d_combine_work: (graph, k) per block).  d_ctl: zeroed
// status word, queue heads and statistics (see count.cu).
pvt_status batch_count(BatchGraph *d_graphs, int count, const int2 *d_combine_work, int n_combine,
                       const uint64_t *const *h_entries, const unsigned *n_entries,
                       const unsigned long long *d_binom, int binom_stride, int num_sms, unsigned *d_ctl,
                       cudaStream_t s);
// Fill the per-(mode, class) root entry lists of a batch from the descriptors.
pvt_status batch_root_entries(BatchGraph *d_graphs, int count, uint64_t *const *d_entries,
                              const unsigned *d_class_offsets /*[count][NCLASS]*/, cudaStream_t s);
// Multi-word Pascal table C(a, b), a < rows, W words per entry.
pvt_status build_binom(unsigned long long *B, int rows, int W, unsigned *err, cudaStream_t s);

// Thread-local error message used by pvt_last_error().
void set_error(const std::string &msg);

// Words needed so every count fits: each count is at most n * 2^alpha.
int32_t min_words(int64_t n, int32_t alpha);

// Map a CUDA error to a status (and record its message).
pvt_status cuda_fail(cudaError_t e, const char *what);

#define PVT_CK(call)                                          \
    do {                                                      \
        cudaError_t _e = (call);                              \
        if (_e != cudaSuccess) return pvt::cuda_fail(_e, #call); \
    } while (0)

// Orientation (orient.cu).
pvt_status orient_build(pvt_dag *g, uint32_t flags, cudaStream_t s);
pvt_status ensure_edge_ids(pvt_dag *g, cudaStream_t s);

// Counting (count.cu).
pvt_status count_global(pvt_dag *g, int32_t kmax, int32_t W, uint64_t *C, cudaStream_t s);
pvt_status count_local(pvt_dag *g, int32_t kmax, int32_t W, uint64_t *out, bool edge,
                       cudaStream_t s);
pvt_status autotune(pvt_dag *g, int32_t kmax, int32_t W, uint64_t *C, cudaStream_t s, pvt_policy *chosen,
                    float *ms);
pvt_status count_hist(pvt_dag *g, int64_t begin, int64_t end, int32_t kmax, uint64_t *hist, cudaStream_t s);
pvt_status combine_hist(pvt_dag *g, const uint64_t *hist, int32_t kmax, int32_t W, uint64_t *C, cudaStream_t s);
pvt_status leaf_depths(pvt_dag *g, uint64_t *depth, cudaStream_t s);
void drop_graph(pvt_dag *g);

// Exclusive prefix sum of uint32 counts into int64 offsets (out has n+1 entries).
pvt_status exclusive_scan_u32_i64(const uint32_t *in, int64_t *out, int64_t n, cudaStream_t s);

// Phase timing: record the start / end event of phase `ph` on stream s (no-op
// unless profiling is on).
void phase_begin(pvt_dag *g, int ph, cudaStream_t s);
void phase_end(pvt_dag *g, int ph, cudaStream_t s);
void stats_reset(pvt_dag *g);

// Read the device status word (synchronises s) and map it to a status.
pvt_status check_device(pvt_dag *g, cudaStream_t s, const char *what);

// A named host range around a library call, so that a profiler's timeline
// shows where each call begins and ends (NVTX; nothing happens without an
// attached tool).
struct HostRange {
    explicit HostRange(const char *name) { nvtxRangePushA(name); }
    ~HostRange() { nvtxRangePop(); }
    HostRange(const HostRange &) = delete;
    HostRange &operator=(const HostRange &) = delete;
};

// Nanosecond clock for bounded waits.
__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

}  // namespace pvt
