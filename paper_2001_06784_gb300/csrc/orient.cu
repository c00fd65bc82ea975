// Degeneracy orientation on the device (Lemma degen, Sec. 3.2; Alg. 1 step 1).
//
// 1. Optional CSR validation (simple undirected graph, Sec. 3.1).
// 2. k-core peeling in one cooperative kernel, exact by level (core numbers
//    are exact), asynchronous within a level (see k_peel): each vertex gets a
//    unique removal time rnd[v].
// 3. The orientation u -> v iff rnd[u] < rnd[v]: a vertex's later
//    neighbours number at most its level k <= alpha, so every out-degree is
//    at most the degeneracy.  Out-lists keep the CSR's ascending-id order.
// 4. Roots grouped by out-degree class (bitset width), largest first.
#include <cooperative_groups.h>

#include <algorithm>
#include <vector>

#include "pvt_internal.cuh"

namespace pvt {

// ------------------------------------------------------------ validation

__global__ void k_validate(int64_t n, int64_t nnz, const int64_t *__restrict__ rp,
                           const uint32_t *__restrict__ col, unsigned *err)
{
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t v = warp; v < n; v += nwarps) {
        int64_t b = rp[v], e = rp[v + 1];
        if (b < 0 || e < b || e > nnz) {
            if (lane == 0) atomicOr(err, DERR_NOTSIMPLE);
            continue;
        }
        for (int64_t j = b + lane; j < e; j += 32) {
            uint32_t u = col[j];
            bool bad = (u >= (uint64_t)n) || (u == (uint64_t)v) || (j + 1 < e && col[j + 1] <= u);
            if (!bad) {
                // symmetry: v must be in row u
                int64_t lo = rp[u], hi = rp[u + 1];
                if (lo < 0 || hi < lo || hi > nnz) {
                    bad = true;
                } else {
                    while (lo < hi) {
                        int64_t mid = lo + ((hi - lo) >> 1);
                        if (col[mid] < (uint32_t)v) lo = mid + 1; else hi = mid;
                    }
                    bad = !(lo < rp[u + 1] && col[lo] == (uint32_t)v);
                }
            }
            if (bad) atomicOr(err, DERR_NOTSIMPLE);
        }
    }
}

// --------------------------------------------------------------- peeling

// Shared state of the peel.  Counters that many warps touch sit on their own
// 128-byte lines.
struct PeelState {
    unsigned head;        // next claim on the removal queue
    unsigned pad0[31];
    unsigned tail;        // vertices pushed onto the removal queue so far
    unsigned pad1[31];
    unsigned done;        // queue entries fully processed so far
    unsigned pad2[31];
    unsigned min_next[2]; // lower bound of the next level's smallest residual degree (by level parity)
    unsigned scan_end[2]; // end of the queue positions the scan pushed (by level parity)
    unsigned alive_cnt[2];// length of the alive list being built (by level parity)
    unsigned bar_count;   // grid barrier arrivals
    unsigned bar_gen;     // grid barrier generation
    unsigned rounds;      // grid barriers passed (diagnostic)
    unsigned levels;      // levels visited (diagnostic)
    unsigned top_level;   // degeneracy: the last level k at which a vertex was removed
    // hand-over to the one-block finish (k_peel_tail)
    unsigned stop;        // 1: the grid peel stopped with few vertices left
    unsigned stop_k;      // k of the first level left to the finish
    unsigned stop_q;      // parity of that level (which alive list)
    unsigned stop_all;    // 1: stopped at level 0 (every vertex is alive, no list)
    unsigned stop_cnt;    // entries of that alive list
    unsigned res_n;       // vertices left (local ids 0..res_n-1)
    unsigned long long res_edges;  // entries of their residual adjacency
};

// The grid peel hands the levels over to one block once at most this many
// vertices are alive: their degrees, removal queue and row offsets then fit
// in shared memory, and a level costs block barriers instead of grid ones.
constexpr unsigned TAIL_MAX = 16384;
constexpr int TAIL_THREADS = 1024;
// residual-row entries a lane loads before it uses the first
constexpr int TAIL_UNROLL = 8;

constexpr unsigned long long BARRIER_LIMIT_NS = 4000000000ull;  // 4 s
constexpr unsigned long long CASCADE_LIMIT_NS = 4000000000ull;  // 4 s without progress
constexpr uint32_t EMPTY = 0xFFFFFFFFu;
// a removal-queue entry whose vertex the pushing warp processes itself
// (vertex ids stop at 0xFFFFFFFD)
constexpr uint32_t TAKEN = 0xFFFFFFFEu;
// bulk processing of a level's scan pushes: from this many pushes on, one
// thread per pushed vertex, for out-lists up to BULK_LANE_MAX entries
constexpr unsigned BULK_MIN = 4096, BULK_LANE_MAX = 64;

// Rows are read PEEL_UNROLL entries per lane at a time: every load, then
// every degree decrement, is in flight before the first result is used.
constexpr int PEEL_UNROLL = 4;
// A warp adds its processed entries to done at least every DONE_REPORT
// entries (and before every claim).
constexpr unsigned DONE_REPORT = 64;

// One removal found by a decrement (bulk phase: single pushes, no warp
// aggregation).
__device__ __forceinline__ void peel_push_one(PeelState *st, uint32_t *rnd, uint32_t *core, uint32_t *lq,
                                              uint32_t u, unsigned k)
{
    const unsigned pos = atomicAdd(&st->tail, 1u);
    rnd[u] = pos;
    core[u] = k;
    *(volatile uint32_t *)(lq + pos) = u;
}

// Grid-wide barrier for a cooperative launch, with a bounded wait: on
// timeout it sets DERR_TIMEOUT and every block leaves the kernel.
__device__ bool grid_barrier(PeelState *st, unsigned *err)
{
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned *vgen = &st->bar_gen;
        unsigned gen = *vgen;
        int ok = 1;
        __threadfence();
        unsigned arrived = atomicAdd(&st->bar_count, 1u) + 1u;
        if (arrived == gridDim.x) {
            st->bar_count = 0;
            st->rounds++;
            __threadfence();
            atomicAdd(&st->bar_gen, 1u);
        } else {
            // poll tightly first (a barrier usually completes within a few
            // microseconds), then back off; give up after BARRIER_LIMIT_NS
            unsigned long long t0 = global_ns();
            unsigned spins = 0;
            while (*vgen == gen) {
                if (++spins < 4096) continue;
                if (*(volatile unsigned *)err & DERR_TIMEOUT) { ok = 0; break; }
                if (global_ns() - t0 > BARRIER_LIMIT_NS) {
                    atomicOr(err, DERR_TIMEOUT);
                    ok = 0;
                    break;
                }
                __nanosleep(32);
            }
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// k-core peeling, exact by level, asynchronous within a level.
//
// Level k removes every remaining vertex whose residual degree is (or falls
// to) at most k; k runs upward from the smallest degree.  A level has two
// phases, each closed by a grid barrier:
//   scan     every vertex of the alive list (all vertices at level 0) that
//            is still present is pushed onto one global removal queue if its
//            degree is <= k, else appended to the next alive list;
//   cascade  warps take queue entries one at a time and lower the residual
//            degree of every neighbour of the entry; the one decrement that
//            takes a neighbour from k+1 to k pushes it at once.  A warp
//            processes the first vertex its own decrements push (its queue
//            entry is marked taken) before it claims another entry: a chain
//            of pushes then skips the queue's publish/claim round trip.  The
//            level ends when every pushed entry has been processed
//            (done == tail).
// Every vertex is pushed exactly once, so its queue position is a unique
// removal time: rnd[v].  Neighbours already removed are decremented too: a
// removed vertex's degree is <= k and only falls, so it can never be pushed
// again, and skipping the presence test saves a dependent load per hop.
// The next level's k is the smallest degree seen above k -- at the scan and
// at every decrement -- which never exceeds the true smallest residual
// degree, so no level with removals is skipped (a level can be empty).
// Out-degree bound: a neighbour pushed after v never lowered deg[v] (v was
// already removed when it was processed), so at v's push deg[v] <= k counts
// all of v's later neighbours.
__global__ void __launch_bounds__(1024, 1) k_peel(int64_t n, const int64_t *__restrict__ rp,
                                               const uint32_t *__restrict__ col, uint32_t *deg,
                                               uint32_t *rnd, uint32_t *core, uint32_t *lq, uint32_t *alive,
                                               PeelState *st, unsigned tail_max, unsigned *err)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
    volatile PeelState *vst = st;

    if (tid == 0) {
        st->min_next[0] = st->min_next[1] = NOT_REMOVED;
        st->alive_cnt[0] = st->alive_cnt[1] = 0;
    }
    if (!grid_barrier(st, err)) return;
    {
        unsigned mine = NOT_REMOVED;
        for (int64_t v = tid; v < n; v += nthreads) {
            const uint32_t dv = (uint32_t)(rp[v + 1] - rp[v]);
            deg[v] = dv;
            rnd[v] = NOT_REMOVED;
            lq[v] = EMPTY;
            mine = min(mine, dv);
        }
        mine = __reduce_min_sync(FULL, mine);
        if (lane == 0 && mine != NOT_REMOVED) atomicMin(&st->min_next[0], mine);
    }
    if (!grid_barrier(st, err)) return;

    unsigned top = 0;
    for (unsigned level = 0;; ++level) {
        const unsigned q = level & 1u;
        // done only moves during a cascade: every thread reads the same value
        // here, and it equals tail (the last cascade ended with done == tail)
        const unsigned t_start = vst->done;
        if ((int64_t)t_start >= n) break;  // every vertex removed
        const unsigned k = vst->min_next[q];
        const int64_t cnt = level == 0 ? n : (int64_t)vst->alive_cnt[q];
        if (cnt <= (int64_t)tail_max) {  // the rest in one block (k_peel_tail)
            if (tid == 0) {
                st->stop = 1;
                st->stop_k = k;
                st->stop_q = q;
                st->stop_all = level == 0;
                st->stop_cnt = (unsigned)cnt;
            }
            break;
        }
        // ---- scan: push present vertices of degree <= k, keep the others
        unsigned mnext = NOT_REMOVED;
        for (int64_t base = tid - lane; base < cnt; base += nthreads) {
            const int64_t i = base + lane;
            uint32_t v = 0;
            bool present = false;
            uint32_t dv = 0;
            if (i < cnt) {
                v = level == 0 ? (uint32_t)i : alive[(q ? n : 0) + i];
                present = rnd[v] == NOT_REMOVED;
                if (present) dv = deg[v];
            }
            const bool take = present && dv <= k, keep = present && dv > k;
            const unsigned bt = __ballot_sync(FULL, take), bk = __ballot_sync(FULL, keep);
            const unsigned below = (1u << lane) - 1u;
            if (bt) {
                unsigned at = 0;
                if (lane == 0) {
                    at = atomicAdd(&st->tail, (unsigned)__popc(bt));
                    atomicMax(&st->scan_end[q], at + (unsigned)__popc(bt));
                }
                at = __shfl_sync(FULL, at, 0);
                if (take) {
                    const unsigned pos = at + __popc(bt & below);
                    rnd[v] = pos;
                    core[v] = k;
                    lq[pos] = v;
                }
            }
            if (bk) {
                unsigned at = 0;
                if (lane == 0) at = atomicAdd(&st->alive_cnt[q ^ 1u], (unsigned)__popc(bk));
                at = __shfl_sync(FULL, at, 0);
                if (keep) {
                    alive[(q ? 0 : n) + at + __popc(bk & below)] = v;
                    mnext = min(mnext, dv);
                }
            }
        }
        if (!grid_barrier(st, err)) return;
        // every scan push happened before the barrier and nothing moves
        // scan_end during the cascade, so every thread reads the same end
        const unsigned se = max(vst->scan_end[q], t_start);
        if (tid == 0) {
            st->levels++;
            st->min_next[q] = NOT_REMOVED;  // read by every thread above; next written at level + 1
            st->alive_cnt[q] = 0;
            st->scan_end[q ^ 1u] = 0;       // last read at level - 1; next written at level + 1
        }
        // ---- bulk: when the scan pushed many vertices, one thread per pushed
        // vertex lowers its neighbours' degrees (lists longer than
        // BULK_LANE_MAX by the whole warp); the claims below then start at se
        const bool bulk = se - t_start >= BULK_MIN;
        if (bulk) {
            unsigned ndone = 0;
            for (int64_t base = (int64_t)t_start + tid - lane; base < (int64_t)se; base += nthreads) {
                const int64_t i = base + lane;
                uint32_t v = 0;
                int64_t b = 0, e = 0;
                if (i < (int64_t)se) {
                    v = lq[i];
                    b = rp[v];
                    e = rp[v + 1];
                    ++ndone;
                }
                const bool mine = e - b <= (int64_t)BULK_LANE_MAX;
                if (mine) {
                    for (int64_t j = b; j < e; j += PEEL_UNROLL) {
                        uint32_t u[PEEL_UNROLL];
                        unsigned old[PEEL_UNROLL];
#pragma unroll
                        for (int t = 0; t < PEEL_UNROLL; ++t) u[t] = j + t < e ? col[j + t] : EMPTY;
#pragma unroll
                        for (int t = 0; t < PEEL_UNROLL; ++t) old[t] = u[t] != EMPTY ? atomicSub(&deg[u[t]], 1u) : 0u;
#pragma unroll
                        for (int t = 0; t < PEEL_UNROLL; ++t) {
                            if (u[t] == EMPTY) continue;
                            if (old[t] == k + 1) peel_push_one(st, rnd, core, lq, u[t], k);
                            else if (old[t] > k + 1) mnext = min(mnext, old[t] - 1);
                        }
                    }
                }
                for (unsigned big = __ballot_sync(FULL, !mine); big; big &= big - 1) {
                    const int src = __ffs(big) - 1;
                    const int64_t bb = __shfl_sync(FULL, b, src), ee = __shfl_sync(FULL, e, src);
                    for (int64_t j0 = bb + lane; j0 < ee; j0 += 32 * PEEL_UNROLL) {
                        uint32_t u[PEEL_UNROLL];
                        unsigned old[PEEL_UNROLL];
#pragma unroll
                        for (int t = 0; t < PEEL_UNROLL; ++t) u[t] = j0 + 32 * t < ee ? col[j0 + 32 * t] : EMPTY;
#pragma unroll
                        for (int t = 0; t < PEEL_UNROLL; ++t) old[t] = u[t] != EMPTY ? atomicSub(&deg[u[t]], 1u) : 0u;
#pragma unroll
                        for (int t = 0; t < PEEL_UNROLL; ++t) {
                            if (u[t] == EMPTY) continue;
                            if (old[t] == k + 1) peel_push_one(st, rnd, core, lq, u[t], k);
                            else if (old[t] > k + 1) mnext = min(mnext, old[t] - 1);
                        }
                    }
                }
            }
            __threadfence();  // these entries' pushes are counted before they are done
            ndone = __reduce_add_sync(FULL, ndone);
            if (lane == 0 && ndone) atomicAdd(&st->done, ndone);
        }
        // ---- cascade, on as many warps per block as the waiting entries need
        // (at least two per block; warps that read the counters late may see
        // a different count, which changes only how many warps take part)
        const unsigned waiting = vst->tail - vst->done;
        const unsigned want = min(max(waiting > (1u << 28) ? (1u << 30) : 4u * waiting, 256u), (unsigned)(nthreads >> 5));
        const unsigned per_block = (want + gridDim.x - 1) / gridDim.x;
        if ((unsigned)wid < per_block) {
            const unsigned below = (1u << lane) - 1u;
            unsigned claim = EMPTY;  // lane 0: this warp's queue position
            unsigned ndone = 0;      // lane 0: entries processed and not yet counted in done
            // a vertex this warp pushed and processes itself (warp-uniform),
            // with its row bounds already loaded
            uint32_t keep = EMPTY;
            int64_t kb = 0, ke = 0;
            for (;;) {
                int64_t b = kb, e = ke;
                if (keep == EMPTY) {
                    int got = 0;  // 1: vertex in `v`, 2: level done, 3: error
                    uint32_t v = 0;
                    if (lane == 0) {
                        // report the finished entries before waiting: the level
                        // cannot end while they are uncounted
                        if (ndone) {
                            __threadfence();  // their pushes are counted before they are done
                            atomicAdd(&st->done, ndone);
                            ndone = 0;
                        }
                        unsigned spins = 0, last = 0xFFFFFFFFu;
                        unsigned long long t0 = 0;
                        for (;;) {
                            if (claim == EMPTY) claim = atomicAdd(&st->head, 1u) + (bulk ? se - t_start : 0u);
                            if (claim < (uint64_t)n) {
                                const uint32_t x = *(volatile uint32_t *)(lq + claim);
                                if (x == TAKEN) { claim = EMPTY; continue; }  // its pusher processes it
                                if (x != EMPTY) { v = x; got = 1; break; }
                            }
                            if ((++spins & 7u) == 0) {
                                // quiescent once every pushed entry is processed; read
                                // done before tail (done <= tail at all times)
                                const unsigned dn = vst->done;
                                __threadfence();
                                if (vst->tail == dn) { got = 2; break; }
                                if (*(volatile unsigned *)err & DERR_TIMEOUT) { got = 3; break; }
                                if (dn != last) { last = dn; t0 = global_ns(); }
                                else if (global_ns() - t0 > CASCADE_LIMIT_NS) { atomicOr(err, DERR_TIMEOUT); got = 3; break; }
                            }
                            __nanosleep(spins < 64 ? 20 : 200);
                        }
                        if (got == 1) claim = EMPTY;
                    }
                    got = __shfl_sync(FULL, got, 0);
                    if (got == 3) return;
                    if (got == 2) break;
                    v = __shfl_sync(FULL, v, 0);
                    b = rp[v];
                    e = rp[v + 1];
                }
                keep = EMPTY;
                // lower the neighbours' degrees; the pushes of one
                // 32 * PEEL_UNROLL-entry stretch take consecutive queue
                // positions (one atomic), and the warp keeps the first of them
                // when it holds none
                for (int64_t j0 = b + lane; __any_sync(FULL, j0 < e); j0 += 32 * PEEL_UNROLL) {
                    uint32_t u[PEEL_UNROLL];
                    unsigned old[PEEL_UNROLL], bp[PEEL_UNROLL];
#pragma unroll
                    for (int t = 0; t < PEEL_UNROLL; ++t) u[t] = j0 + 32 * t < e ? col[j0 + 32 * t] : EMPTY;
#pragma unroll
                    for (int t = 0; t < PEEL_UNROLL; ++t) old[t] = u[t] != EMPTY ? atomicSub(&deg[u[t]], 1u) : 0u;
                    unsigned tot = 0;
                    uint32_t kv = EMPTY;
#pragma unroll
                    for (int t = 0; t < PEEL_UNROLL; ++t) {
                        if (u[t] != EMPTY && old[t] > k + 1) mnext = min(mnext, old[t] - 1);
                        bp[t] = __ballot_sync(FULL, u[t] != EMPTY && old[t] == k + 1);
                        tot += __popc(bp[t]);
                        if (kv == EMPTY && bp[t]) kv = __shfl_sync(FULL, u[t], __ffs(bp[t]) - 1);
                    }
                    if (!tot) continue;
                    const bool take = keep == EMPTY;
                    if (take) {
                        keep = kv;
                        kb = rp[keep];  // in flight during the atomic below
                        ke = rp[keep + 1];
                    }
                    unsigned pos = 0;
                    if (lane == 0) pos = atomicAdd(&st->tail, tot);
                    pos = __shfl_sync(FULL, pos, 0);
#pragma unroll
                    for (int t = 0; t < PEEL_UNROLL; ++t) {
                        if (bp[t] >> lane & 1u) {
                            const unsigned p = pos + __popc(bp[t] & below);
                            rnd[u[t]] = p;
                            core[u[t]] = k;
                            *(volatile uint32_t *)(lq + p) = take && u[t] == kv ? TAKEN : u[t];
                        }
                        pos += __popc(bp[t]);
                    }
                }
                if (lane == 0 && ++ndone >= DONE_REPORT) {
                    // a long chain of kept vertices (a path graph's level is
                    // one chain) reports its progress as it goes: waiting
                    // warps give up after CASCADE_LIMIT_NS without any
                    __threadfence();  // their pushes are counted before they are done
                    atomicAdd(&st->done, ndone);
                    ndone = 0;
                }
            }
        }
        mnext = __reduce_min_sync(FULL, mnext);
        if (lane == 0 && mnext != NOT_REMOVED) atomicMin(&st->min_next[q ^ 1u], mnext);
        if (!grid_barrier(st, err)) return;
        const unsigned t_end = vst->done;
        if (t_end > t_start) top = k;
        if (tid == 0) st->head = t_end;  // drop claims past the end of the queue
    }
    if (tid == 0) st->top_level = top;
}

// ------------------------------------------------ one-block finish of the peel

__device__ void block_scan_u32_i64(const uint32_t *in, int64_t *out, int64_t n);

// Vertices still present where the grid peel stopped get local ids
// 0..res_n-1 (tv: local -> global, loc: global -> local) and their residual
// degrees: deg[v] counts exactly the present neighbours, since every removed
// vertex has been processed.
__global__ void k_tail_compact(int64_t n, const uint32_t *__restrict__ alive, const uint32_t *__restrict__ rnd,
                               const uint32_t *__restrict__ deg, uint32_t *loc, uint32_t *tv, uint32_t *rdeg,
                               PeelState *st)
{
    if (!st->stop) return;
    const int64_t cnt = st->stop_cnt;
    const bool all = st->stop_all != 0;
    if (!all && st->stop_q) alive += n;
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = blockIdx.x * (int64_t)blockDim.x + threadIdx.x - lane; base < cnt; base += stride) {
        const int64_t i = base + lane;
        uint32_t v = 0;
        bool present = false;
        if (i < cnt) {
            v = all ? (uint32_t)i : alive[i];
            present = rnd[v] == NOT_REMOVED;
        }
        const unsigned b = __ballot_sync(FULL, present);
        if (!b) continue;
        unsigned at = 0;
        if (lane == 0) at = atomicAdd(&st->res_n, (unsigned)__popc(b));
        at = __shfl_sync(FULL, at, 0);
        if (present) {
            const unsigned id = at + __popc(b & ((1u << lane) - 1u));
            loc[v] = id;
            tv[id] = v;
            rdeg[id] = deg[v];
        }
    }
}

// Row offsets of the residual adjacency (one block).
__global__ void k_tail_scan(const uint32_t *rdeg, int64_t *roff, PeelState *st)
{
    if (!st->stop) return;
    const unsigned R = st->res_n;
    block_scan_u32_i64(rdeg, roff, R);
    if (threadIdx.x == 0) st->res_edges = (unsigned long long)roff[R];
}

// Residual adjacency: local ids of the present neighbours (warp per vertex).
__global__ void k_tail_fill(const int64_t *__restrict__ rp, const uint32_t *__restrict__ col,
                            const uint32_t *__restrict__ rnd, const uint32_t *__restrict__ loc,
                            const uint32_t *__restrict__ tv, const int64_t *__restrict__ roff, uint32_t *rcol,
                            const PeelState *st, unsigned *err)
{
    if (!st->stop) return;
    const int lane = threadIdx.x & 31;
    const unsigned R = st->res_n;
    const int64_t w0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = w0; i < (int64_t)R; i += nw) {
        const uint32_t v = tv[i];
        const int64_t beg = rp[v], end = rp[v + 1], out = roff[i], cap = roff[i + 1] - out;
        int64_t pos = 0;
        for (int64_t j0 = beg; j0 < end; j0 += 32) {
            const int64_t j = j0 + lane;
            uint32_t u = 0;
            bool keep = false;
            if (j < end) {
                u = col[j];
                keep = rnd[u] == NOT_REMOVED;
            }
            const unsigned b = __ballot_sync(FULL, keep);
            if (keep) {
                const int64_t at = pos + __popc(b & ((1u << lane) - 1u));
                if (at < cap) rcol[out + at] = loc[u];
            }
            pos += __popc(b);
        }
        if (lane == 0 && pos != cap) atomicOr(err, DERR_RANGE);
    }
}

// The remaining levels in one block, same rules as k_peel (scan, then a
// cascade that ends when done == tail) on block-shared state: residual
// degrees, the removal queue and the row offsets live in shared memory,
// the residual adjacency (local ids) in global memory.  Removal times
// continue the grid peel's numbering.
__global__ void __launch_bounds__(TAIL_THREADS, 1) k_peel_tail(const int64_t *__restrict__ roff,
                                                            const uint32_t *__restrict__ rcol,
                                                            const uint32_t *__restrict__ rdeg,
                                                            const uint32_t *__restrict__ tv, uint32_t *rnd,
                                                            uint32_t *core, PeelState *st, unsigned *err)
{
    extern __shared__ __align__(16) uint32_t tsm[];
    uint32_t *sdeg = tsm, *sq = tsm + TAIL_MAX, *soff = tsm + 2 * TAIL_MAX, *sgone = tsm + 3 * TAIL_MAX + 1;
    __shared__ unsigned s_head, s_tail, s_done, s_min[2], s_bad;
    volatile unsigned *vq = sq;
    const int lane = threadIdx.x & 31;
    if (!st->stop) return;
    const unsigned R = st->res_n;
    if (R > TAIL_MAX) {
        if (threadIdx.x == 0) atomicOr(err, DERR_RANGE);
        return;
    }
    const unsigned base = st->done;  // removals so far (grid peel)
    for (unsigned i = threadIdx.x; i < R; i += blockDim.x) {
        sdeg[i] = rdeg[i];
        sq[i] = EMPTY;
        soff[i] = (uint32_t)roff[i];
    }
    for (unsigned i = threadIdx.x; i < (R + 31) / 32; i += blockDim.x) sgone[i] = 0;
    if (threadIdx.x == 0) {
        soff[R] = (uint32_t)roff[R];
        s_head = s_tail = s_done = 0;
        s_min[0] = st->stop_k;
        s_min[1] = NOT_REMOVED;
        s_bad = 0;
    }
    __syncthreads();
    unsigned top = st->top_level, levels = 0;
    // a push touches shared memory only: the removal times and core numbers
    // of a level go out to global memory once the level is over
    auto push = [&](unsigned i) {
        atomicOr(&sgone[i >> 5], 1u << (i & 31));
        const unsigned pos = atomicAdd(&s_tail, 1u);
        vq[pos] = i;
        // the warp that takes this entry runs on this SM: bring the start of
        // the vertex's residual row into L1 for it
        asm volatile("prefetch.global.L1 [%0];" ::"l"(rcol + soff[i]));
    };
    for (unsigned level = 0;; ++level) {
        const unsigned q = level & 1u;
        const unsigned t_start = *(volatile unsigned *)&s_done;
        if (t_start >= R) break;
        const unsigned k = s_min[q];
        ++levels;
        unsigned mnext = NOT_REMOVED;
        // ---- scan of the vertices still present, 16 per thread from the
        // removed bitmap (only the owner of a chunk pushes from it, so the
        // bits it read do not change under it)
        for (unsigned c = threadIdx.x; c < (R + 15) / 16; c += blockDim.x) {
            const unsigned base = c * 16;
            uint32_t live = (~sgone[c >> 1] >> (16 * (c & 1))) & 0xFFFFu;
            if (base + 16 > R) live &= (1u << (R - base)) - 1u;
            for (; live; live &= live - 1) {
                const unsigned i = base + __ffs(live) - 1;
                const unsigned d = sdeg[i];
                if (d <= k) push(i);
                else mnext = min(mnext, d);
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) s_min[q] = NOT_REMOVED;  // read above by every thread
        // ---- cascade (every warp); none when the scan took every vertex
        // left: decrements could then only reach removed vertices
        if (*(volatile unsigned *)&s_tail == R) {
            if (threadIdx.x == 0) s_done = R;
        } else {
            unsigned claim = EMPTY;
            for (;;) {
                int got = 0;  // 1: entry in i, 2: level done, 3: error
                unsigned i = 0;
                if (lane == 0) {
                    if (claim == EMPTY) claim = atomicAdd(&s_head, 1u);
                    unsigned spins = 0, last = EMPTY;
                    unsigned long long t0 = 0;
                    for (;;) {
                        if (claim < R) {
                            const unsigned x = vq[claim];
                            if (x != EMPTY) { i = x; got = 1; break; }
                        }
                        const unsigned dn = *(volatile unsigned *)&s_done;
                        __threadfence_block();
                        if (*(volatile unsigned *)&s_tail == dn) { got = 2; break; }
                        if ((++spins & 63u) == 0) {
                            if (*(volatile unsigned *)&s_bad) { got = 3; break; }
                            if (dn != last) { last = dn; t0 = global_ns(); }
                            else if (global_ns() - t0 > CASCADE_LIMIT_NS) {
                                atomicOr(err, DERR_TIMEOUT);
                                s_bad = 1;
                                got = 3;
                                break;
                            }
                        }
                        if (spins > 16) __nanosleep(32);
                    }
                    if (got == 1) claim = EMPTY;
                }
                got = __shfl_sync(FULL, got, 0);
                if (got != 1) break;
                i = __shfl_sync(FULL, i, 0);
                const unsigned e = soff[i + 1];
                for (unsigned j0 = soff[i] + lane; j0 < e; j0 += 32 * TAIL_UNROLL) {
                    uint32_t u[TAIL_UNROLL];
#pragma unroll
                    for (int t = 0; t < TAIL_UNROLL; ++t) u[t] = j0 + 32 * t < e ? rcol[j0 + 32 * t] : EMPTY;
#pragma unroll
                    for (int t = 0; t < TAIL_UNROLL; ++t) {
                        if (u[t] == EMPTY) continue;
                        const unsigned old = atomicSub(&sdeg[u[t]], 1u);
                        if (old == k + 1) push(u[t]);
                        else if (old > k + 1) mnext = min(mnext, old - 1);
                    }
                }
                __syncwarp();
                if (lane == 0) {
                    __threadfence_block();  // this entry's pushes are counted before it is done
                    atomicAdd(&s_done, 1u);
                }
            }
        }
        mnext = __reduce_min_sync(FULL, mnext);
        if (lane == 0 && mnext != NOT_REMOVED) atomicMin(&s_min[q ^ 1u], mnext);
        __syncthreads();
        if (s_bad) return;
        const unsigned t_end = s_done;
        if (t_end > t_start) top = k;
        for (unsigned p = t_start + threadIdx.x; p < t_end; p += blockDim.x) {
            const uint32_t v = tv[sq[p]];
            rnd[v] = base + p;
            core[v] = k;
        }
        __syncthreads();  // every thread has read s_done before the claims are reset
        if (threadIdx.x == 0) s_head = s_tail;
    }
    if (threadIdx.x == 0) {
        st->top_level = top;
        st->levels += levels;
    }
}

// ------------------------------------------------------------ orientation

__device__ __forceinline__ bool key_less(uint32_t ra, uint32_t a, uint32_t rb, uint32_t b)
{
    return ra < rb || (ra == rb && a < b);
}

// Out-degree of every vertex (warp per vertex) and the largest one.
__global__ void k_outdeg(int64_t n, const int64_t *__restrict__ rp, const uint32_t *__restrict__ col,
                         const uint32_t *__restrict__ rnd, uint32_t *odeg, unsigned *alpha)
{
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    unsigned most = 0;  // largest out-degree this warp has seen
    for (int64_t v = warp; v < n; v += nwarps) {
        uint32_t rv = rnd[v];
        unsigned c = 0;
        for (int64_t j = rp[v] + lane; j < rp[v + 1]; j += 32) {
            uint32_t u = col[j];
            c += key_less(rv, (uint32_t)v, rnd[u], u);
        }
        c = __reduce_add_sync(FULL, c);
        if (lane == 0) odeg[v] = c;
        most = max(most, c);
    }
    if (lane == 0 && most) atomicMax(alpha, most);
}

// Out-lists in CSR order (ascending id), compacted with a warp ballot.
__global__ void k_fill(int64_t n, const int64_t *__restrict__ rp, const uint32_t *__restrict__ col,
                       const uint32_t *__restrict__ rnd, const int64_t *__restrict__ orow,
                       uint32_t *ocol)
{
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t v = warp; v < n; v += nwarps) {
        uint32_t rv = rnd[v];
        int64_t out = orow[v];
        for (int64_t j0 = rp[v]; j0 < rp[v + 1]; j0 += 32) {
            int64_t j = j0 + lane;
            uint32_t u = 0;
            bool keep = false;
            if (j < rp[v + 1]) {
                u = col[j];
                keep = key_less(rv, (uint32_t)v, rnd[u], u);
            }
            unsigned b = __ballot_sync(FULL, keep);
            if (keep) ocol[out + __popc(b & ((1u << lane) - 1u))] = u;
            out += __popc(b);
        }
    }
}

// Class of an out-degree: 0 for d = 0, else 1 + ceil(log2(ceil(d / 32))).
__host__ __device__ inline int degree_class(uint32_t d)
{
    if (d == 0) return 0;
    int c = 1;
    uint32_t cap = 32;
    while (d > cap) { cap <<= 1; ++c; }
    return c;
}

// (a block-shared histogram first: out-degrees crowd into a few small values)
__global__ void k_deg_hist(int64_t n, const uint32_t *__restrict__ odeg, unsigned *hist, int nd)
{
    extern __shared__ unsigned sh[];
    for (int i = threadIdx.x; i < nd; i += blockDim.x) sh[i] = 0;
    __syncthreads();
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(&sh[min(odeg[v], (uint32_t)(nd - 1))], 1u);
    __syncthreads();
    for (int i = threadIdx.x; i < nd; i += blockDim.x)
        if (sh[i]) atomicAdd(&hist[i], sh[i]);
}

// Scatter roots so that out-degrees descend within the array (slot[d] holds
// the next free position for out-degree d); lanes with equal out-degrees
// share one atomic.
__global__ void k_deg_scatter(int64_t n, const uint32_t *__restrict__ odeg, unsigned *slot,
                              uint32_t *roots)
{
    const int lane = threadIdx.x & 31;
    for (int64_t base = blockIdx.x * (int64_t)blockDim.x + threadIdx.x - lane; base < n;
         base += (int64_t)gridDim.x * blockDim.x) {
        const int64_t v = base + lane;
        const bool valid = v < n;
        const unsigned act = __ballot_sync(FULL, valid);
        if (!valid) continue;
        const uint32_t d = odeg[v];
        const unsigned peers = __match_any_sync(act, d);
        const int leader = __ffs(peers) - 1;
        unsigned at = 0;
        if (lane == leader) at = atomicAdd(&slot[d], (unsigned)__popc(peers));
        at = __shfl_sync(peers, at, leader);
        roots[at + __popc(peers & ((1u << lane) - 1u))] = (uint32_t)v;
    }
}

// ------------------------------------------------------------------ scan

__global__ void k_scan_blocks(const uint32_t *__restrict__ in, int64_t *out, int64_t n,
                              unsigned long long *bsum)
{
    // exclusive scan of one 1024-element tile per block; tile total to bsum
    __shared__ unsigned long long ws[32];
    int64_t i = blockIdx.x * 1024ll + threadIdx.x;
    unsigned long long x = i < n ? in[i] : 0;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    unsigned long long inc = x;
    for (int o = 1; o < 32; o <<= 1) {
        unsigned long long t = __shfl_up_sync(FULL, inc, o);
        if (lane >= o) inc += t;
    }
    if (lane == 31) ws[wid] = inc;
    __syncthreads();
    if (wid == 0) {
        unsigned long long w = ws[lane], wi = w;
        for (int o = 1; o < 32; o <<= 1) {
            unsigned long long t = __shfl_up_sync(FULL, wi, o);
            if (lane >= o) wi += t;
        }
        ws[lane] = wi - w;
        if (lane == 31) bsum[blockIdx.x] = wi;
    }
    __syncthreads();
    if (i < n) out[i] = (int64_t)(inc - x + ws[wid]);
}

__global__ void k_scan_sums(unsigned long long *bsum, int64_t nb, int64_t *total_out)
{
    // single block: exclusive scan of the tile totals in place
    __shared__ unsigned long long carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __shared__ unsigned long long ws[32];
    for (int64_t base = 0; base < nb; base += 1024) {
        int64_t i = base + threadIdx.x;
        unsigned long long x = i < nb ? bsum[i] : 0, inc = x;
        for (int o = 1; o < 32; o <<= 1) {
            unsigned long long t = __shfl_up_sync(FULL, inc, o);
            if (lane >= o) inc += t;
        }
        if (lane == 31) ws[wid] = inc;
        __syncthreads();
        if (wid == 0) {
            unsigned long long w = ws[lane], wi = w;
            for (int o = 1; o < 32; o <<= 1) {
                unsigned long long t = __shfl_up_sync(FULL, wi, o);
                if (lane >= o) wi += t;
            }
            ws[lane] = wi - w;
        }
        __syncthreads();
        unsigned long long c = carry;
        if (i < nb) bsum[i] = c + inc - x + ws[wid];
        __syncthreads();
        if (threadIdx.x == 1023) carry = c + inc + ws[wid];
        __syncthreads();
    }
    if (threadIdx.x == 0) *total_out = (int64_t)carry;
}

__global__ void k_scan_add(int64_t *out, int64_t n, const unsigned long long *__restrict__ bsum)
{
    int64_t i = blockIdx.x * 1024ll + threadIdx.x;
    if (i < n) out[i] += (int64_t)bsum[blockIdx.x];
}

pvt_status exclusive_scan_u32_i64(const uint32_t *in, int64_t *out, int64_t n, cudaStream_t s)
{
    int64_t nb = (n + 1023) / 1024;
    unsigned long long *bsum = nullptr;
    PVT_CK(cudaMallocAsync(&bsum, (size_t)std::max<int64_t>(nb, 1) * sizeof(unsigned long long), s));
    if (nb > 0) k_scan_blocks<<<(unsigned)nb, 1024, 0, s>>>(in, out, n, bsum);
    k_scan_sums<<<1, 1024, 0, s>>>(bsum, nb, out + n);
    if (nb > 0) k_scan_add<<<(unsigned)nb, 1024, 0, s>>>(out, n, bsum);
    PVT_CK(cudaGetLastError());
    PVT_CK(cudaFreeAsync(bsum, s));
    return PVT_OK;
}

// ------------------------------------------------------------- edge ids

// Edge id of every out-edge r -> u: rank of (min, max) in lexicographic
// order = up[a] + (position of b in row a) - (position of the first entry
// > a in row a), with a = min, b = max and up[a] = edges (x, y), x < y, x < a.
__global__ void k_upper_count(int64_t n, const int64_t *__restrict__ rp,
                              const uint32_t *__restrict__ col, uint32_t *cnt)
{
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x) {
        int64_t lo = rp[v], hi = rp[v + 1], e = hi;
        while (lo < hi) {
            int64_t mid = lo + ((hi - lo) >> 1);
            if (col[mid] <= (uint32_t)v) lo = mid + 1; else hi = mid;
        }
        cnt[v] = (uint32_t)(e - lo);
    }
}

__device__ __forceinline__ int64_t lower_bound_row(const uint32_t *__restrict__ col, int64_t lo,
                                                   int64_t hi, uint32_t x)
{
    while (lo < hi) {
        int64_t mid = lo + ((hi - lo) >> 1);
        if (col[mid] < x) lo = mid + 1; else hi = mid;
    }
    return lo;
}

__global__ void k_edge_ids(int64_t n, const int64_t *__restrict__ rp, const uint32_t *__restrict__ col,
                           const int64_t *__restrict__ up, const int64_t *__restrict__ orow,
                           const uint32_t *__restrict__ ocol, uint32_t *oeid)
{
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t r = warp; r < n; r += nwarps) {
        for (int64_t j = orow[r] + lane; j < orow[r + 1]; j += 32) {
            uint32_t u = ocol[j];
            uint32_t a = min((uint32_t)r, u), b = max((uint32_t)r, u);
            int64_t pos = lower_bound_row(col, rp[a], rp[a + 1], b);
            int64_t first = lower_bound_row(col, rp[a], rp[a + 1], a + 1);
            oeid[j] = (uint32_t)(up[a] + (pos - first));
        }
    }
}

pvt_status ensure_edge_ids(pvt_dag *g, cudaStream_t s)
{
    if (g->oeid || g->m == 0) return PVT_OK;
    if (g->m > 0xFFFFFFFFll) {
        set_error("pvt_count_local_edge: more than 2^32 edges");
        return PVT_EINVAL;
    }
    uint32_t *cnt = nullptr;
    int64_t *up = nullptr;
    PVT_CK(cudaMallocAsync(&cnt, (size_t)g->n * sizeof(uint32_t) + 4, s));
    PVT_CK(cudaMallocAsync(&up, (size_t)(g->n + 1) * sizeof(int64_t), s));
    PVT_CK(cudaMallocAsync(&g->oeid, (size_t)g->m * sizeof(uint32_t), s));
    int grid = g->num_sms * 8;
    k_upper_count<<<grid, 256, 0, s>>>(g->n, g->row_ptr, g->col, cnt);
    pvt_status st = exclusive_scan_u32_i64(cnt, up, g->n, s);
    if (st != PVT_OK) return st;
    k_edge_ids<<<grid, 256, 0, s>>>(g->n, g->row_ptr, g->col, up, g->orow, g->ocol, g->oeid);
    PVT_CK(cudaGetLastError());
    PVT_CK(cudaFreeAsync(cnt, s));
    PVT_CK(cudaFreeAsync(up, s));
    return PVT_OK;
}

// ---------------------------------------------------------------- driver

pvt_status orient_build(pvt_dag *g, uint32_t flags, cudaStream_t s)
{
    const int64_t n = g->n;
    const int grid = g->num_sms * 8;
    PVT_CK(cudaMemsetAsync(g->d_err, 0, sizeof(unsigned), s));
    if (flags & PVT_VALIDATE) {
        k_validate<<<grid, 256, 0, s>>>(n, g->nnz, g->row_ptr, g->col, g->d_err);
        PVT_CK(cudaGetLastError());
        g->stats.launches++;
        pvt_status st = check_device(g, s, "pvt_orient: CSR validation");
        if (st != PVT_OK) return st;
    }

    uint32_t *deg = nullptr, *lq = nullptr, *odeg = nullptr, *alive = nullptr;
    uint32_t *tv = nullptr, *rdeg = nullptr, *rcol = nullptr;
    int64_t *roff = nullptr;
    unsigned *dhist = nullptr;
    PeelState *pst = nullptr;
    const size_t nb = (size_t)std::max<int64_t>(n, 1) * sizeof(uint32_t);
    PVT_CK(cudaMallocAsync(&deg, nb, s));
    PVT_CK(cudaMallocAsync(&lq, nb, s));
    PVT_CK(cudaMallocAsync(&alive, 2 * nb, s));
    PVT_CK(cudaMallocAsync(&pst, sizeof(PeelState) + sizeof(unsigned), s));
    PVT_CK(cudaMallocAsync(&g->rnd, nb, s));
    PVT_CK(cudaMallocAsync(&g->core, nb, s));
    PVT_CK(cudaMemsetAsync(pst, 0, sizeof(PeelState) + sizeof(unsigned), s));

    // one cooperative launch: every block must be resident at once
    int per_sm = 0;
    PVT_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_peel, 1024, 0));
    per_sm = std::min(per_sm, 1);
    if (per_sm < 1) {
        set_error("pvt_orient: peel kernel cannot be resident");
        return PVT_ECUDA;
    }
    {
        int64_t nn = n;
        const int64_t *rp = g->row_ptr;
        const uint32_t *col = g->col;
        uint32_t *rnd = g->rnd, *core = g->core;
        unsigned *err = g->d_err;
        unsigned tail_max = TAIL_MAX;
        void *args[] = {&nn, &rp, &col, &deg, &rnd, &core, &lq, &alive, &pst, &tail_max, &err};
        phase_begin(g, 0, s);
        PVT_CK(cudaLaunchCooperativeKernel((void *)k_peel, dim3(g->num_sms * per_sm), dim3(1024), args,
                                           0, s));
        // the levels left once at most TAIL_MAX vertices are alive: one block
        // on the compacted residual graph (each kernel returns at once if the
        // grid peel finished by itself); lq is free by now and holds local ids
        PVT_CK(cudaMallocAsync(&tv, (size_t)TAIL_MAX * sizeof(uint32_t), s));
        PVT_CK(cudaMallocAsync(&rdeg, (size_t)TAIL_MAX * sizeof(uint32_t), s));
        PVT_CK(cudaMallocAsync(&roff, (size_t)(TAIL_MAX + 1) * sizeof(int64_t), s));
        PVT_CK(cudaMallocAsync(&rcol, (size_t)std::max<int64_t>(g->nnz, 1) * sizeof(uint32_t), s));
        k_tail_compact<<<(TAIL_MAX + 255) / 256, 256, 0, s>>>(n, alive, g->rnd, deg, lq, tv, rdeg, pst);
        k_tail_scan<<<1, 1024, 0, s>>>(rdeg, roff, pst);
        k_tail_fill<<<g->num_sms * 8, 256, 0, s>>>(g->row_ptr, g->col, g->rnd, lq, tv, roff, rcol, pst, g->d_err);
        constexpr size_t tail_smem = (3 * (size_t)TAIL_MAX + 1 + TAIL_MAX / 32) * sizeof(uint32_t);
        PVT_CK(cudaFuncSetAttribute(k_peel_tail, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tail_smem));
        k_peel_tail<<<1, TAIL_THREADS, tail_smem, s>>>(roff, rcol, rdeg, tv, g->rnd, g->core, pst, g->d_err);
        PVT_CK(cudaGetLastError());
        phase_end(g, 0, s);
        g->stats.launches += 5;
    }
    phase_begin(g, 1, s);

    // orientation
    unsigned *d_alpha = (unsigned *)(pst + 1);
    PVT_CK(cudaMallocAsync(&odeg, nb + sizeof(uint32_t), s));
    PVT_CK(cudaMallocAsync(&g->orow, (size_t)(n + 1) * sizeof(int64_t), s));
    k_outdeg<<<grid, 256, 0, s>>>(n, g->row_ptr, g->col, g->rnd, odeg, d_alpha);
    PVT_CK(cudaGetLastError());
    pvt_status st = exclusive_scan_u32_i64(odeg, g->orow, n, s);
    g->stats.launches += 4;
    if (st != PVT_OK) return st;
    unsigned alpha = 0;
    PeelState hst{};
    PVT_CK(cudaMemcpyAsync(&hst, pst, sizeof(PeelState), cudaMemcpyDeviceToHost, s));
    PVT_CK(cudaMemcpyAsync(&alpha, d_alpha, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
    PVT_CK(cudaStreamSynchronize(s));
    st = check_device(g, s, "pvt_orient: peeling");
    if (st != PVT_OK) return st;
    // alpha = the degeneracy (top core level): it bounds every out-degree and,
    // unlike the largest out-degree, does not depend on the removal order
    // within a level
    if (alpha > hst.top_level) {
        set_error("pvt_orient: an out-degree exceeds the degeneracy");
        return PVT_EINTERNAL;
    }
    alpha = hst.top_level;
    g->alpha = (int32_t)alpha;
    g->stats.peel_rounds = hst.rounds;
    g->stats.peel_levels = hst.levels;
    if (g->alpha > MAX_ALPHA) {
        set_error("pvt_orient: degeneracy " + std::to_string(alpha) + " above the supported " +
                  std::to_string(MAX_ALPHA));
        return PVT_EINVAL;
    }
    PVT_CK(cudaMallocAsync(&g->ocol, (size_t)std::max<int64_t>(g->m, 1) * sizeof(uint32_t), s));
    k_fill<<<grid, 256, 0, s>>>(n, g->row_ptr, g->col, g->rnd, g->orow, g->ocol);
    PVT_CK(cudaGetLastError());
    g->stats.launches++;

    // roots by descending out-degree (counting sort), grouped into classes
    const int nd = g->alpha + 1;
    PVT_CK(cudaMallocAsync(&dhist, (size_t)nd * sizeof(unsigned), s));
    PVT_CK(cudaMemsetAsync(dhist, 0, (size_t)nd * sizeof(unsigned), s));
    k_deg_hist<<<grid, 256, (size_t)nd * sizeof(unsigned), s>>>(n, odeg, dhist, nd);
    g->stats.launches++;
    std::vector<unsigned> hh(nd), slot(nd);
    PVT_CK(cudaMemcpyAsync(hh.data(), dhist, (size_t)nd * sizeof(unsigned), cudaMemcpyDeviceToHost, s));
    PVT_CK(cudaStreamSynchronize(s));
    // positions: larger out-degrees first; class c (degree range) is then a
    // contiguous slice, higher classes first
    unsigned pos = 0;
    for (int d = nd - 1; d >= 0; --d) { slot[d] = pos; pos += hh[d]; }
    for (int c = 0; c < NCLASS; ++c) g->class_cnt[c] = 0;
    for (int d = 0; d < nd; ++d) g->class_cnt[degree_class((uint32_t)d)] += hh[d];
    {
        int64_t off = 0;
        for (int c = NCLASS - 1; c >= 0; --c) { g->class_start[c] = off; off += g->class_cnt[c]; }
    }
    PVT_CK(cudaMemcpyAsync(dhist, slot.data(), (size_t)nd * sizeof(unsigned), cudaMemcpyHostToDevice, s));
    PVT_CK(cudaMallocAsync(&g->roots, nb, s));
    k_deg_scatter<<<grid, 256, 0, s>>>(n, odeg, dhist, g->roots);
    PVT_CK(cudaGetLastError());
    phase_end(g, 1, s);
    g->stats.launches++;
    for (int c = 0; c < NCLASS; ++c) g->stats.roots[c] = (uint64_t)g->class_cnt[c];

    PVT_CK(cudaFreeAsync(deg, s));
    PVT_CK(cudaFreeAsync(lq, s));
    PVT_CK(cudaFreeAsync(alive, s));
    PVT_CK(cudaFreeAsync(tv, s));
    PVT_CK(cudaFreeAsync(rdeg, s));
    PVT_CK(cudaFreeAsync(roff, s));
    PVT_CK(cudaFreeAsync(rcol, s));
    PVT_CK(cudaFreeAsync(pst, s));
    PVT_CK(cudaFreeAsync(odeg, s));
    PVT_CK(cudaFreeAsync(dhist, s));
    PVT_CK(cudaStreamSynchronize(s));
    return check_device(g, s, "pvt_orient");
}


// ----------------------------------------------------- batched orientation
//
// Small graphs of a served batch are oriented one block per graph, in a
// single launch: the same exact-by-level peel with a removal cascade (here on
// shared-memory counters), the DAG CSR, per-edge ids when the query needs
// them, and the roots grouped by class.  Block-level waits are bounded.

// Exclusive prefix sum of in[0..n) into out[0..n] (out[n] = total) by one block.
__device__ void block_scan_u32_i64(const uint32_t *in, int64_t *out, int64_t n)
{
    __shared__ long long s_warp[32];
    __shared__ long long s_carry;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (threadIdx.x == 0) s_carry = 0;
    __syncthreads();
    for (int64_t base = 0; base < n; base += blockDim.x) {
        const int64_t i = base + threadIdx.x;
        const long long x = i < n ? (long long)in[i] : 0;
        long long inc = x;
        for (int o = 1; o < 32; o <<= 1) {
            long long t = __shfl_up_sync(FULL, inc, o);
            if (lane >= o) inc += t;
        }
        if (lane == 31) s_warp[wid] = inc;
        __syncthreads();
        if (wid == 0) {
            long long w = lane < nw ? s_warp[lane] : 0, wi = w;
            for (int o = 1; o < 32; o <<= 1) {
                long long t = __shfl_up_sync(FULL, wi, o);
                if (lane >= o) wi += t;
            }
            if (lane < nw) s_warp[lane] = wi - w;
        }
        __syncthreads();
        const long long excl = s_carry + s_warp[wid] + inc - x;
        if (i < n) out[i] = excl;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) s_carry = excl + x;
        __syncthreads();
    }
    if (threadIdx.x == 0) out[n] = s_carry;
    __syncthreads();
}

constexpr unsigned long long BLOCK_WAIT_LIMIT_NS = 2000000000ull;  // 2 s without progress

__global__ void __launch_bounds__(1024) k_orient_batch(BatchGraph *gs)
{
    BatchGraph &G = gs[blockIdx.x];
    const int64_t n = G.n;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int64_t *rp = G.rp;
    const uint32_t *col = G.col;
    uint32_t *deg = G.deg, *rnd = G.rnd, *lq = G.lq;
    __shared__ unsigned s_len, s_min, s_head, s_tail, s_pending, s_err, s_alpha;
    __shared__ unsigned s_hist[BATCH_MAX_ALPHA + 2];
    __shared__ unsigned s_cls[NCLASS];
    if (threadIdx.x == 0) { s_head = 0; s_tail = 0; s_pending = 0; s_err = 0; s_alpha = 0; }
    for (int64_t v = threadIdx.x; v < n; v += blockDim.x) {
        deg[v] = (uint32_t)(rp[v + 1] - rp[v]);
        rnd[v] = NOT_REMOVED;
        lq[v] = 0xFFFFFFFFu;
        G.tmp[v] = (uint32_t)v;
    }
    __syncthreads();

    // ---- 1. peel: exact levels, removal cascade within a level
    uint32_t *L = G.tmp, *L2 = G.tmp + n;
    unsigned len = (unsigned)n, k = 0, claim = 0xFFFFFFFFu;
    for (;;) {
        if (threadIdx.x == 0) { s_len = 0; s_min = NOT_REMOVED; }
        __syncthreads();
        for (unsigned i = threadIdx.x; i < len; i += blockDim.x) {
            const uint32_t v = L[i];
            if (rnd[v] == NOT_REMOVED) {
                L2[atomicAdd(&s_len, 1u)] = v;
                atomicMin(&s_min, deg[v]);
            }
        }
        __syncthreads();
        len = s_len;
        { uint32_t *t = L; L = L2; L2 = t; }
        if (len == 0) break;
        k = max(k, s_min);
        for (unsigned i = threadIdx.x; i < len; i += blockDim.x) {
            const uint32_t v = L[i];
            if (deg[v] <= k) {
                const unsigned t = atomicAdd(&s_tail, 1u);
                atomicAdd(&s_pending, 1u);
                rnd[v] = t;
                lq[t] = v;
            }
        }
        __syncthreads();
        for (;;) {
            int got = 0;  // 1 vertex, 2 level done, 3 error
            uint32_t v = 0;
            if (lane == 0) {
                if (claim == 0xFFFFFFFFu) claim = atomicAdd(&s_head, 1u);
                unsigned last = 0xFFFFFFFFu;
                unsigned long long t0 = global_ns();
                for (;;) {
                    if (claim < (uint64_t)n) {
                        const uint32_t x = *(volatile uint32_t *)(lq + claim);
                        if (x != 0xFFFFFFFFu) { v = x; got = 1; break; }
                    }
                    const unsigned pend = *(volatile unsigned *)&s_pending;
                    if (pend == 0) { got = 2; break; }
                    if (*(volatile unsigned *)&s_err) { got = 3; break; }
                    if (pend != last) { last = pend; t0 = global_ns(); }
                    else if (global_ns() - t0 > BLOCK_WAIT_LIMIT_NS) { atomicOr(&s_err, DERR_TIMEOUT); got = 3; break; }
                    __nanosleep(32);
                }
                if (got == 1) claim = 0xFFFFFFFFu;
            }
            got = __shfl_sync(FULL, got, 0);
            if (got != 1) break;
            v = __shfl_sync(FULL, v, 0);
            for (int64_t j = rp[v] + lane; j < rp[v + 1]; j += 32) {
                const uint32_t u = col[j];
                if (rnd[u] == NOT_REMOVED) {
                    const unsigned old = atomicSub(&deg[u], 1u);
                    if (old == k + 1) {
                        atomicAdd(&s_pending, 1u);
                        const unsigned t = atomicAdd(&s_tail, 1u);
                        rnd[u] = t;
                        __threadfence_block();
                        *(volatile uint32_t *)(lq + t) = u;
                    }
                }
            }
            __syncwarp();
            if (lane == 0) {
                __threadfence_block();
                atomicSub(&s_pending, 1u);
            }
        }
        __syncthreads();
        if (s_err) break;
    }
    __syncthreads();
    if (s_err) {
        if (threadIdx.x == 0) G.info[BI_ERR] = s_err;
        return;
    }
    const unsigned top_level = k;  // degeneracy

    // ---- 2. DAG: out-degrees (into deg), offsets, out-lists in id order
    for (int64_t v = wid; v < n; v += nwarps) {
        const uint32_t rv = rnd[v];
        unsigned c = 0;
        for (int64_t j = rp[v] + lane; j < rp[v + 1]; j += 32) c += rnd[col[j]] > rv;
        for (int o = 16; o; o >>= 1) c += __shfl_xor_sync(FULL, c, o);
        if (lane == 0) {
            deg[v] = c;
            atomicMax(&s_alpha, c);
        }
    }
    __syncthreads();
    block_scan_u32_i64(deg, G.orow, n);
    for (int64_t v = wid; v < n; v += nwarps) {
        const uint32_t rv = rnd[v];
        int64_t out = G.orow[v];
        for (int64_t j0 = rp[v]; j0 < rp[v + 1]; j0 += 32) {
            const int64_t j = j0 + lane;
            uint32_t u = 0;
            bool keep = false;
            if (j < rp[v + 1]) {
                u = col[j];
                keep = rnd[u] > rv;
            }
            const unsigned b = __ballot_sync(FULL, keep);
            if (keep) G.ocol[out + __popc(b & ((1u << lane) - 1u))] = u;
            out += __popc(b);
        }
    }
    __syncthreads();

    // ---- 3. edge ids (rank of (min, max) in lexicographic order)
    if (G.oeid) {
        for (int64_t v = threadIdx.x; v < n; v += blockDim.x) {
            int64_t lo = rp[v], hi = rp[v + 1], e = hi;
            while (lo < hi) {
                int64_t mid = lo + ((hi - lo) >> 1);
                if (col[mid] <= (uint32_t)v) lo = mid + 1; else hi = mid;
            }
            L[v] = (uint32_t)(e - lo);  // neighbours above v (tmp is free now)
        }
        __syncthreads();
        block_scan_u32_i64(L, G.up, n);
        for (int64_t r = wid; r < n; r += nwarps) {
            for (int64_t j = G.orow[r] + lane; j < G.orow[r + 1]; j += 32) {
                const uint32_t u = G.ocol[j];
                const uint32_t a = min((uint32_t)r, u), b = max((uint32_t)r, u);
                int64_t lo = rp[a], hi = rp[a + 1];
                while (lo < hi) {
                    int64_t mid = lo + ((hi - lo) >> 1);
                    if (col[mid] < b) lo = mid + 1; else hi = mid;
                }
                const int64_t pos = lo;
                lo = rp[a];
                hi = rp[a + 1];
                while (lo < hi) {
                    int64_t mid = lo + ((hi - lo) >> 1);
                    if (col[mid] <= a) lo = mid + 1; else hi = mid;
                }
                G.oeid[j] = (uint32_t)(G.up[a] + (pos - lo));
            }
        }
        __syncthreads();
    }

    // ---- 4. roots by class, out-degree descending (counting sort)
    const unsigned alpha = top_level;  // bounds every out-degree (s_alpha)
    if (s_alpha > top_level || alpha > BATCH_MAX_ALPHA) {
        if (threadIdx.x == 0) { G.info[BI_ALPHA] = alpha; G.info[BI_ERR] = DERR_RANGE; }
        return;
    }
    for (unsigned d = threadIdx.x; d <= alpha; d += blockDim.x) s_hist[d] = 0;
    __syncthreads();
    for (int64_t v = threadIdx.x; v < n; v += blockDim.x) atomicAdd(&s_hist[deg[v]], 1u);
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned pos = 0;
        for (int c = 0; c < NCLASS; ++c) s_cls[c] = 0;
        for (int d = (int)alpha; d >= 0; --d) {
            const unsigned c = s_hist[d];
            s_hist[d] = pos;
            pos += c;
            s_cls[degree_class((uint32_t)d)] += c;
        }
        unsigned off = 0;
        for (int c = NCLASS - 1; c >= 0; --c) {
            G.info[BI_START + c] = off;
            G.info[BI_CNT + c] = s_cls[c];
            off += s_cls[c];
        }
        G.info[BI_ALPHA] = alpha;
        G.info[BI_ERR] = 0;
    }
    __syncthreads();
    for (int64_t v = threadIdx.x; v < n; v += blockDim.x) G.roots[atomicAdd(&s_hist[deg[v]], 1u)] = (uint32_t)v;
}

pvt_status batch_orient(BatchGraph *d_graphs, int count, cudaStream_t s)
{
    if (count <= 0) return PVT_OK;
    k_orient_batch<<<count, 1024, 0, s>>>(d_graphs);
    PVT_CK(cudaGetLastError());
    return PVT_OK;
}

}  // namespace pvt
