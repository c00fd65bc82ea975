/*
 * pivoter.h -- C ABI of libpivoter: exact k-clique counts for every k, on one
 * GPU, with the Succinct Clique Tree (SCT) of Jain & Seshadhri, "The Power of
 * Pivoting for Exact Clique Counting" (WSDM 2020).
 *
 * Conventions shared by every entry point
 *   - Graphs are given as CSR over vertices 0..n-1: row_ptr int64[n+1] and
 *     col uint32[nnz] with nnz = row_ptr[n] = 2m.  The graph must be simple
 *     and undirected (Sec. 3.1, "Problem Statement"; Sec. 3.2): every row is
 *     sorted strictly ascending, no self-loops, and v is in row u exactly
 *     when u is in row v.  Directed inputs must be symmetrised by the caller
 *     (the paper ignores edge directions, Sec. 5).
 *   - "device" pointers are CUDA global-memory pointers on the current
 *     device; "host" pointers are ordinary CPU memory.  The caller owns every
 *     buffer it passes in; the library owns the pvt_dag and its scratch.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Calls return once their results are complete and checked.
 *   - Counts are exact unsigned integers of W little-endian 64-bit words
 *     (word 0 least significant).  Arrays are indexed [.. ][k][word] with
 *     k = 0..kmax the clique size: entry 0 is 0, k = 1 counts vertices, k = 2
 *     edges, and entries with k above the clique number are 0.
 *   - Edge ids: edge {u, v} has the id of (min, max) in lexicographic order,
 *     i.e. its rank in the upper triangle of the CSR read row by row.
 *   - No C++ exception crosses the ABI.  On failure a call returns a status
 *     other than PVT_OK, leaves output buffers unspecified, and
 *     pvt_last_error() returns a message for the calling thread.
 */
#ifndef PIVOTER_H
#define PIVOTER_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum pvt_status {
    PVT_OK = 0,
    PVT_EINVAL = 1,      /* bad argument (sizes, NULL pointers, kmax) */
    PVT_ENOTSIMPLE = 2,  /* CSR not sorted / symmetric / loop-free (with PVT_VALIDATE) */
    PVT_ENOMEM = 3,      /* device allocation failed */
    PVT_EOVERFLOW = 4,   /* W words cannot hold every count of this graph */
    PVT_ECUDA = 5,       /* a CUDA call failed */
    PVT_ETIMEOUT = 6,    /* a bounded device-side wait expired */
    PVT_EINTERNAL = 7    /* a device-side capacity or consistency check failed (a library bug) */
} pvt_status;

/* Opaque, library-owned device state of one oriented graph. */
typedef struct pvt_dag pvt_dag;

/* pvt_orient flags: check that the CSR is a simple undirected graph first;
 * time every phase with CUDA events from the start (see pvt_dag_stats). */
#define PVT_VALIDATE 0x1u
#define PVT_PROFILE 0x2u

/*
 * Orient the graph along a degeneracy order (Lemma degen, Sec. 3.2; Alg. 1
 * step 1): k-core peeling on the device, then the out-neighbourhoods N+(v)
 * as a CSR over the DAG, every out-degree at most the degeneracy alpha.
 * alpha_out and pvt_dag_info report alpha = the degeneracy (the top core
 * level), which bounds every out-degree and does not depend on how removals
 * within a level are ordered.
 *   n, nnz       vertex count (< 2^32) and row_ptr[n] (= 2m), host values
 *   row_ptr,col  device CSR as above.  It is borrowed, not copied: it must
 *                stay valid and unchanged until pvt_dag_free (per-edge counts
 *                read it again).
 *   flags        0, PVT_VALIDATE (else the CSR is trusted), PVT_PROFILE
 *   dag_out      receives the new pvt_dag (host pointer to a pointer)
 *   alpha_out    receives the largest out-degree (host; may be NULL)
 * Errors: PVT_EINVAL, PVT_ENOTSIMPLE, PVT_ENOMEM, PVT_ECUDA, PVT_ETIMEOUT.
 */
pvt_status pvt_orient(int64_t n, int64_t nnz, const int64_t *row_ptr, const uint32_t *col,
                      uint32_t flags, void *stream, pvt_dag **dag_out, int32_t *alpha_out);

/*
 * Sizes of an oriented graph, all host outputs (any may be NULL): n, m,
 * alpha, and min_words = the smallest W every count call accepts,
 * ceil((bits(n) + alpha + 1) / 64) with a floor of 1: every clique lies in
 * {r} + N+(r) for its first vertex r, so each count is at most n * 2^alpha.
 */
pvt_status pvt_dag_info(const pvt_dag *dag, int64_t *n, int64_t *m, int32_t *alpha,
                        int32_t *min_words);

/*
 * Core numbers found by the peel (Sec. 3.2: the degeneracy order removes a
 * vertex of smallest residual degree; the core number of v is the largest k
 * such that v lies in a subgraph of minimum degree k).  Unlike the removal
 * order, core numbers do not depend on how ties are broken.
 *   core    device uint32[n] (caller-owned), written in full on `stream`
 * Errors: PVT_EINVAL (NULL dag, or NULL core with n > 0), PVT_ECUDA.
 */
pvt_status pvt_dag_cores(const pvt_dag *dag, uint32_t *core, void *stream);

/*
 * Global counts C_k for k = 0..kmax (Sec. 3.1; Alg. 2, the C_{|H|+i} update;
 * correctness: proof of Thm. main).  Each root vertex r explores the SCT
 * below its child N+(r) (Alg. 1) depth first; every root-to-leaf path T with
 * h = |H(T)| and p = |P(T)| adds C(p, i) to C_{h+i}.  kmax truncates (Sec. 4,
 * "Counting k-cliques for a specific k"): branches with more than kmax hold
 * links are cut and the counts for k <= kmax stay exact.
 *   kmax   >= 0; any value is accepted (entries above the clique number are 0)
 *   W      words per count, >= min_words (else PVT_EOVERFLOW before any launch)
 *   C      device uint64[kmax+1][W], written in full
 * Every root has exactly one all-pivot path (a leaf with h = 1), and the
 * 2-cliques read off the leaves are the edges; for kmax >= 1 the device
 * checks the first, for kmax >= 2 the second, before C is formed.
 * Errors: PVT_EINVAL, PVT_EOVERFLOW, PVT_ENOMEM, PVT_ECUDA, PVT_EINTERNAL
 * (a capacity check, or the path check above, failed).
 */
pvt_status pvt_count_global(pvt_dag *dag, int32_t kmax, int32_t W, uint64_t *C, void *stream);

/*
 * Per-vertex counts c_k(v) (Sec. 3.1; Alg. 2 steps ht and pt): for each path
 * T, every v in H(T) gains C(p, i) at k = h+i and every v in P(T) gains
 * C(p-1, i) at k = h+1+i.  The paper leaves parallel local counts as future
 * work (Sec. 4, "Parallel version"); here roots run in parallel and add into
 * one table with exact carry-propagating atomics.
 *   cv     device uint64[n][kmax+1][W], written in full
 * Other arguments and errors as pvt_count_global.
 */
pvt_status pvt_count_local_vertex(pvt_dag *dag, int32_t kmax, int32_t W, uint64_t *cv,
                                  void *stream);

/*
 * Per-edge counts c_k(e) (Sec. 3.1; Alg. 2 steps hht, pht, ppt): each pair
 * inside H(T) gains C(p, i) at k = h+i, each pair (P, H) gains C(p-1, i) at
 * k = h+1+i and each pair inside P(T) gains C(p-2, i) at k = h+2+i.
 *   ce     device uint64[m][kmax+1][W] indexed by edge id, written in full
 * Other arguments and errors as pvt_count_global.
 */
pvt_status pvt_count_local_edge(pvt_dag *dag, int32_t kmax, int32_t W, uint64_t *ce,
                                void *stream);

/*
 * Global counts in pieces, for checkpointing long counts.  Every clique is
 * counted once, at its first vertex in the orientation, and the roots are
 * independent (Sec. 4, "Parallel version"), so the (h, p) histogram of
 * root-to-leaf paths over a set of roots is the whole state of a count:
 * histograms of disjoint root sets add up, and C_k = sum over (h, p) of
 * hist[h][p] * C(p, k - h) (proof of Thm. main) turns the sum into counts.
 *   pvt_count_hist  walks the roots r with begin <= r < end (vertex ids;
 *                   end is clipped to n) and ADDS their path counts to
 *                   hist, device uint64[(alpha+2)][(alpha+2)] (row h,
 *                   column p; caller-owned, not cleared); branches with
 *                   more than kmax hold links are cut as in
 *                   pvt_count_global.  The call synchronises `stream` once
 *                   to size the range.
 *   pvt_combine_hist  C (device uint64[kmax+1][W]) from such a histogram;
 *                   kmax must not exceed the one the histogram was built
 *                   with; W as pvt_count_global.
 * Copying hist to the host after any range and back before the next is a
 * checkpoint; the histogram of disjoint ranges counted on different GPUs
 * (each with its own dag of the same graph) is their sum.
 * For kmax >= 1 the device checks that row h = 1 gained exactly one leaf
 * per root of the range (PVT_EINTERNAL otherwise).
 * Errors: PVT_EINVAL (NULL dag or hist, kmax < 0, begin < 0, end < begin),
 * others as pvt_count_global.
 */
pvt_status pvt_count_hist(pvt_dag *dag, int64_t begin, int64_t end, int32_t kmax, uint64_t *hist, void *stream);
pvt_status pvt_combine_hist(pvt_dag *dag, const uint64_t *hist, int32_t kmax, int32_t W, uint64_t *C,
                            void *stream);

/*
 * Frequency distribution of one column of a local count table (the
 * per-vertex clique distributions of the experiments, "Demonstrations of
 * Pivoter": f_k(b) = the number of vertices that take part in exactly b
 * k-cliques; over a per-edge table, the number of edges).
 *   table       device uint64[rows][K][W], as written by
 *               pvt_count_local_vertex / pvt_count_local_edge (read only)
 *   rows, K, W  its shape; rows <= 2^32 - 2, 1 <= W <= 20
 *   k           the column, 0 <= k < K
 *   values      device uint64[rows][W] (caller-owned): the distinct values b
 *               of column k, W words each, least significant first
 *   counts      device uint64[rows] (caller-owned): f_k(b) for each value
 *   n_distinct  host: the number of (value, count) pairs written
 * Pairs come in no particular order; the counts sum to rows.  The call
 * allocates stream-ordered scratch (12 bytes per hash slot, at least
 * 2 * rows slots) and returns once the pairs are written.
 * Errors: PVT_EINVAL (argument out of range), PVT_ENOMEM, PVT_ECUDA.
 */
pvt_status pvt_local_distribution(const uint64_t *table, int64_t rows, int32_t K, int32_t W, int32_t k,
                                  uint64_t *values, uint64_t *counts, int64_t *n_distinct, void *stream);

/*
 * Statistics of the last orient or count call on a dag (no counterpart in
 * the paper's algorithms; its Fig. treesize reports SCT sizes).  Tree
 * figures are of the walk the device performed: nodes visited (leaves and
 * roots with no out-neighbour included; a node whose label is a nonempty
 * clique is closed as one leaf, so the |S| nodes of its pivot chain are not
 * visited), root-to-leaf paths, and the pivot words: |S| * ceil(|S|/32) per
 * internal node, the AND + population-count word pairs of pivot selection
 * over rows restricted to the label's own members -- a property of the tree,
 * whichever row width a kernel walks it in.  ms[] holds device
 * time per phase when profiling is on (else zeros): [0] peel, [1] orient
 * (DAG CSR and root classes), [2..7] the walk kernels of out-degree classes
 * <=32, <=64, <=128, <=256, <=512, <=1024, [8] combine/finish, [9] the
 * frame walk (policy.frames).  Phases of different classes overlap in time.
 */
typedef struct pvt_stats {
    uint64_t sct_nodes;
    uint64_t sct_leaves;
    uint64_t pivot_words;
    uint64_t launches;      /* kernels launched by the call */
    uint64_t roots[7];      /* roots per out-degree class (0, <=32, ..., <=1024) */
    uint64_t class_words[7];/* pivot_words of the class kernels (walk of labels > 32
                               members only when frames are on) */
    uint64_t frame_words;   /* pivot_words of the frame walk (policy.frames) */
    uint64_t frames;        /* frames the wide walks emitted (above the buffer:
                               walked in place) */
    float ms[10];
    uint32_t peel_rounds;   /* orient: grid-wide barriers of the peel */
    uint32_t peel_levels;   /* orient: distinct core levels visited */
} pvt_stats;

/* Copy the statistics of the last call into *out (host). */
pvt_status pvt_dag_stats(const pvt_dag *dag, pvt_stats *out);

/*
 * Depth profile of the SCT (no counterpart in the paper's algorithms; its
 * Fig. treesize reports SCT sizes): the leaves walked by the last completed
 * pvt_count_global on this dag by depth d = h + p, the number of links on
 * the root-to-leaf path (= the size of the largest clique the path encodes,
 * H(T) with all of P(T)), for d = 0..alpha+1.
 *   depth   host uint64[alpha + 2]
 * Errors: PVT_EINVAL (NULL argument, or no completed global count since
 * pvt_orient), PVT_ECUDA.  The call synchronises `stream`.
 */
pvt_status pvt_dag_leaf_depths(pvt_dag *dag, uint64_t *depth, void *stream);

/*
 * The orientation itself (Lemma degen; Alg. 1 step 1): the DAG's out-lists
 * N+(v), v = 0..n-1, each sorted by vertex id -- the roots' children whose
 * subtrees the count calls walk.
 *   orow   device int64[n + 1] (caller-owned), CSR row offsets
 *   ocol   device uint32[m] (caller-owned; may be NULL when m = 0)
 * Errors: PVT_EINVAL (NULL argument), PVT_ECUDA.  The call synchronises
 * `stream`.
 */
pvt_status pvt_dag_out_lists(const pvt_dag *dag, int64_t *orow, uint32_t *ocol, void *stream);

/* Enable (1) or disable (0) per-phase device timing with CUDA events. */
pvt_status pvt_dag_set_profiling(pvt_dag *dag, int32_t enable);

/*
 * The measured integer ceiling of the walk kernels (no counterpart in the
 * paper): how many 32-bit AND + population count + add triples -- one pivot
 * word pair of the walk (Alg. 1 pivot step, |N(S,u)| word by word) -- the
 * current device sustains per second on independent register chains with
 * every SM busy (fastest of three timed launches after one warm-up, tens of
 * milliseconds each).  The roofline of the walk kernels divides by it.
 *   pairs_per_s  host: receives the rate
 *   stream       CUDA stream (NULL: the default stream); the call waits for it
 * Errors: PVT_EINVAL (NULL pairs_per_s), PVT_ECUDA.
 */
pvt_status pvt_measure_popc_rate(double *pairs_per_s, void *stream);

/*
 * Launch policy of the walk kernels (no counterpart in the paper, whose
 * parallel variant gives each thread whole roots, Sec. 4 "Parallel version").
 *   persistent  1 (default): per out-degree class, a grid sized to the GPU
 *               whose warps take roots from a device work queue (largest
 *               out-degree first); 0: the plain form, one warp per root and
 *               one launch per class.
 *   chunk       roots taken per queue access in the <=32 class (1..32,
 *               default 4); ignored by the plain form.
 *   split[c]    per out-degree class c (0, <=32, ..., <=1024): 1 lets the
 *               warps of a global count share the subtrees of heavy roots
 *               through a device frame queue (many warps on one root);
 *               0 keeps one warp per root.  Only classes with out-degree
 *               above 32 can split, and only in the persistent form; local
 *               counts never split.  Default {0, 0, 1, 1, 1, 1, 1}.
 *   frames      1 (default): global counts run in two phases -- the kernels
 *               of the classes above 32 walk only labels of more than 32
 *               members and emit every smaller label's subtree as a
 *               self-contained frame (its one-word adjacency rows), which a
 *               second kernel with small per-warp state, and so many more
 *               resident warps, walks for all classes; 0: each class walks
 *               its small labels itself.  Persistent form only.
 *   graph       1: pvt_count_global records its launch sequence as a CUDA
 *               graph at the first call with a given (kmax, W, C) and
 *               replays it at later calls with the same three (the dag's
 *               buffers are fixed after orientation); 0 (default): launch
 *               directly.  Replayed calls report no phase times.
 *   wait_limit_us  0 (default): the bounded device-side waits of the walk
 *               (an idle warp waiting for a donated frame, a donor waiting
 *               for a free ring slot) give up after 120 s without progress
 *               and 2 s respectively; > 0: after this many microseconds
 *               instead.  A wait that gives up ends the call with
 *               PVT_ETIMEOUT and leaves the library usable; the field
 *               exists to exercise that path (0 .. 10^9).
 *   lanes       1 (default): in global counts of the persistent form, the
 *               frames of the two-phase walk (labels of at most 32 members)
 *               are walked one subtree per lane, 32 subtrees per warp,
 *               instead of one per warp; 0: one per warp.  The walked tree
 *               is the same either way.
 *   cta[c]      per out-degree class c: 1 walks each root of the class with a
 *               whole thread block over one shared copy of its adjacency
 *               rows, the block's warps sharing its subtrees and walking its
 *               labels of at most 32 members one per lane; 0: a warp per
 *               root.  Global counts of the persistent form, classes above
 *               128 (c >= 4) only.  Default {0, 0, 0, 0, 0, 1, 1}.
 *   serial      0 (default): the classes' kernels run on streams of their own
 *               and overlap; 1: one after another on the caller's stream, so
 *               that the phase times of pvt_dag_stats are each kernel's own
 *               (a measurement setting; results are the same).
 * Each field is checked: PVT_EINVAL for a value out of range.
 */
typedef struct pvt_policy {
    int32_t persistent;
    int32_t chunk;
    int32_t split[7];
    int32_t graph;
    int32_t frames;
    int32_t wait_limit_us;
    int32_t lanes;
    int32_t cta[7];
    int32_t serial;
} pvt_policy;

/* Set the launch policy for later count calls on this dag (drops a recorded
 * graph). */
pvt_status pvt_dag_set_policy(pvt_dag *dag, const pvt_policy *policy);

/* Copy the dag's current launch policy into *out (host). */
pvt_status pvt_dag_get_policy(const pvt_dag *dag, pvt_policy *out);

/*
 * Autotuner of the launch policy (no counterpart in the paper).  Runs
 * pvt_count_global(dag, kmax, W, C, stream) under three candidate policies
 * -- {chunk 4, split}, {chunk 1, no split}, {chunk 16, split} -- twice each,
 * with the out-degree classes launched one after another and timed with CUDA
 * events, then keeps per class the fastest: the chunk of the <=32 class and,
 * for every wider class, whether its heavy roots split across warps.  The
 * chosen policy (persistent, graph flag unchanged) is set on the dag and
 * copied to *chosen; ms (host float[3][7], may be NULL) receives the second
 * timing of each class under each candidate.  C holds the counts on return;
 * errors as pvt_count_global.
 */
pvt_status pvt_dag_autotune(pvt_dag *dag, int32_t kmax, int32_t W, uint64_t *C, void *stream,
                            pvt_policy *chosen, float *ms);

/*
 * Global counts without any device allocation.  The paper has no
 * counterpart: this entry point exists for callers that cannot call
 * cudaMalloc while they count -- code that runs inside a pre-sized memory
 * arena or a framework whose allocator it cannot reach, latency paths that
 * forbid allocation, or contexts where an allocation could block or fail.
 * The caller passes an oriented graph and the output; all scratch (leaf
 * histogram, Pascal table, work-queue head, status word) lives in one fixed
 * device array of about 400 KB that the library holds on every GPU that
 * loads it, until the process exits.
 *   n            vertex count (host value)
 *   orow, ocol   device CSR of an acyclic orientation: the out-neighbours of
 *                v are ocol[orow[v] .. orow[v+1]), sorted ascending, no
 *                self-loops; every edge of the graph in exactly one list
 *                (any acyclic orientation gives the same counts, e.g. "keep
 *                the neighbours with a larger id")
 *   alpha        the largest out-degree, at most 126 (else PVT_EINVAL; a
 *                list longer than alpha is refused with PVT_EINVAL)
 *   kmax, W, C   as pvt_count_global; W at most 4 (else PVT_EINVAL)
 * The first call on a device looks up the array's device address with that
 * device current.  Every call on a device shares the one array and clears
 * what must start at zero; calls whose work overlaps on the GPU (other
 * streams, other host threads) race on it and must be serialised by the
 * caller.  The call reads its status word back and synchronises `stream`
 * before it returns, so it cannot be called while `stream` is being
 * captured into a CUDA graph.  It returns once C is complete and checked
 * (the root-path checks of pvt_count_global, every vertex being a root;
 * PVT_EINTERNAL if they fail).
 * Errors: PVT_EINVAL (NULL orow or ocol with n > 0, NULL C, alpha or W
 * beyond the limits above, an out-list longer than alpha), PVT_EOVERFLOW,
 * PVT_ECUDA, PVT_EINTERNAL.
 */
pvt_status pvt_count_global_noalloc(int64_t n, const int64_t *orow, const uint32_t *ocol, int32_t alpha,
                                    int32_t kmax, int32_t W, uint64_t *C, void *stream);

/*
 * Serving: a query server with continuous batching (no counterpart in the
 * paper; its parallel variant gives whole roots to threads, Sec. 4, and the
 * root subproblems of many graphs are just as independent).  Queries arrive
 * with host CSRs; a worker admits them while device memory (mem_budget
 * bytes, estimated from the CSR and the bound alpha <= sqrt(2m)) and slots
 * (max_inflight) allow, orients every newly admitted group in one batched
 * launch (one block per graph), and walks the roots of the whole group in
 * shared persistent launches; a later group is admitted and oriented while
 * earlier groups still run, and groups run on separate streams so their work
 * overlaps.  Queries of at least direct_edges edges bypass the batches: a
 * second worker runs them one at a time through pvt_orient and the count
 * entry points on a stream of its own, whole-GPU kernels beside the batches.
 * Results are exact and equal to the single-graph entry points.
 */
typedef struct pvt_server pvt_server;

typedef struct pvt_server_config {
    size_t mem_budget;     /* device bytes for requests in flight (0: 8 GiB) */
    int32_t max_inflight;  /* requests admitted at once (0: 1024) */
    int32_t max_batch;     /* graphs per batched launch (0: 256) */
    int32_t streams;       /* concurrent batches (0: 4) */
    int64_t direct_edges;  /* queries with at least this many edges run alone on
                              the whole GPU (the single-graph entry points, in
                              a worker of their own) instead of in a batch;
                              0: 65536, < 0: never */
} pvt_server_config;

enum { PVT_QUERY_GLOBAL = 0, PVT_QUERY_VERTEX = 1, PVT_QUERY_EDGE = 2 };

/* Start a server on the current device. */
pvt_status pvt_server_create(const pvt_server_config *cfg, pvt_server **out);

/*
 * Submit one query: host CSR (as for pvt_orient; copied before return, so the
 * caller may reuse its buffers), kind PVT_QUERY_*, kmax < 0 for every k
 * (alpha + 1).  n must be below 2^32 and the degeneracy at most 512 (1024 for
 * queries on the direct path).
 * ticket receives the query's handle.  Errors: PVT_EINVAL, PVT_ENOMEM (the
 * query can never fit in mem_budget).
 */
pvt_status pvt_server_submit(pvt_server *sv, int64_t n, int64_t nnz, const int64_t *row_ptr,
                             const uint32_t *col, int32_t kind, int32_t kmax, uint64_t *ticket);

/* Wait up to timeout_ms (< 0: no limit) for a query; *done = 1 when its
 * result is ready (or it failed: pvt_server_result reports the status). */
pvt_status pvt_server_wait(pvt_server *sv, uint64_t ticket, int32_t timeout_ms, int32_t *done);

/*
 * Result of a finished query: rows (1 global, n per-vertex, m per-edge), K
 * (= kmax + 1) and W as in pvt_count_*; with out != NULL and out_words >=
 * rows*K*W the words are copied to out (host, layout as pvt_count_*), the
 * query is released and *latency_s (may be NULL) receives submit-to-done
 * seconds.  With out == NULL only the sizes are reported.
 */
pvt_status pvt_server_result(pvt_server *sv, uint64_t ticket, int64_t *rows, int32_t *K, int32_t *W,
                             uint64_t *out, size_t out_words, double *latency_s);

/* Stop the server after the queries in flight finish; frees everything. */
void pvt_server_destroy(pvt_server *sv);

/* Release a pvt_dag and all its device memory (NULL is ignored). */
void pvt_dag_free(pvt_dag *dag);

/* Message for the last failed call on this thread ("" if none). */
const char *pvt_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* PIVOTER_H */
