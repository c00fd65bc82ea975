// One-word SCT walk with one subtree per lane (global counts).
//
// Labels of at most 32 members -- the compacted subtrees that the wide
// walks emit as frames, and the small labels below a dense root (cta.cuh) --
// hold almost all nodes of the SCT, and each of their nodes is a handful of
// word operations: pivot selection is |S| ANDs and population counts on
// one-word rows (Alg. 1 pivot step), each child one AND (Alg. 1 hold step).
// A warp that walks one such subtree spends tens of instructions of
// reductions, shuffles and stack bookkeeping per node.  Here each lane of a
// warp walks its own subtree instead: the 32 one-word rows of lane j's label
// sit in shared memory column j (rows[v][j]), its depth-first stack in
// column j of the warp's stack arrays, so that every shared-memory access of
// the warp touches 32 distinct banks whatever depth or row each lane is at.
// Per node a lane runs the same steps as the warp walk -- pivot = most
// neighbours inside S, ties to the lowest index; a clique label closes as
// one leaf with p + |S|; children of at most two members close at once (the
// closed forms of walk.cuh) -- so the tree, its statistics and the (h, p)
// leaf histogram are exactly those of the warp walk.
//
// Work moves at three levels: a free lane takes the next frame of the
// launch's source; a
// free lane with the source exhausted takes the oldest pending stack entry
// of a busy lane of its warp (with that lane's rows); and, through the ring
// queue of walk.cuh, a busy warp donates the oldest pending entry of its
// most loaded lane, as a compacted frame, to a warp that has run dry.
#pragma once

#include "walk.cuh"

namespace pvt {

constexpr int LANE_WPB = 8;     // warps per block
constexpr int LSTK = 32;        // per-lane stack slots (a label of s <= 32 keeps at most 31 pending)
constexpr unsigned LANE_DONATE_EVERY = 16;  // node steps between looks at the ring queue
constexpr unsigned LANE_DONATE_MAX = 4;     // entries one look may donate

struct LaneWork {
    uint32_t rows[32][32];      // rows[v][lane]: row v of the lane's current subtree
    uint32_t stkS[LSTK][32];    // pending labels, circular per lane
    uint32_t stkHP[LSTK][32];   // their (h << 16) | p
};

// Per-lane walk statistics (each lane its own subtrees; summed at the end).
struct LaneCounters {
    unsigned long long nodes = 0, leaves = 0, words = 0;
    __device__ __forceinline__ void flush(unsigned long long *stats, int slot, int lane)
    {
        const unsigned long long n = warp_sum64(nodes), l = warp_sum64(leaves), w = warp_sum64(words);
        if (lane == 0 && n) {
            atomicAdd(&stats[0], n);
            atomicAdd(&stats[1], l);
            atomicAdd(&stats[2], w);
            if (slot >= 0) atomicAdd(&stats[3 + slot], w);
        }
    }
    __device__ __forceinline__ static unsigned long long warp_sum64(unsigned long long x)
    {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(FULL, x, o);
        return x;
    }
};

// Leaf tally of one lane.  Leaves with h < HIST_H and p < HIST_P go to the
// block's 32-bit histogram in shared memory (native 32-bit shared atomics,
// which 32 lanes tallying at once need); an increment that wraps a counter
// adds 2^32 to the 64-bit histogram in global memory, so the sum of the two
// is exact at any count.  lane_hist_flush adds what is left at the end.
__device__ __forceinline__ void lane_tally(unsigned *sh32, const CountArgs &A, int h, int p)
{
    if (h < HIST_H && p < HIST_P) {
        const unsigned old = atomicAdd(&sh32[h * HIST_P + p], 1u);
        if (old == 0xFFFFFFFFu) atomicAdd(&A.hist[(size_t)h * A.hstride + p], 1ull << 32);
    } else {
        atomicAdd(&A.hist[(size_t)h * A.hstride + p], 1ull);
    }
}

// The block's 32-bit histogram into the global one (all threads of the block,
// after the last tally).
__device__ __forceinline__ void lane_hist_flush(unsigned *sh32, const CountArgs &A)
{
    __syncthreads();
    for (int i = threadIdx.x; i < HIST_H * HIST_P; i += blockDim.x) {
        const unsigned x = sh32[i];
        if (x) atomicAdd(&A.hist[(size_t)(i / HIST_P) * A.hstride + (i % HIST_P)], (unsigned long long)x);
    }
}

// Subtree of a label of at most two members in closed form, by one lane
// (the cases of close_small in walk.cuh).
__device__ __forceinline__ void lane_close_small(unsigned *sh32, const CountArgs &A, int cs, bool adjacent, int h,
                                                 int p, LaneCounters &lc)
{
    const bool split = cs == 2 && !adjacent;
    const bool hold = split && h + 1 <= A.kmax;
    lc.nodes += 1 + split + hold;
    lc.leaves += 1 + hold;
    lc.words += (unsigned)cs;
    if (!split) {
        lane_tally(sh32, A, h, p + cs);
        return;
    }
    lane_tally(sh32, A, h, p + 1);  // the pivot leaf below the pair
    if (hold) lane_tally(sh32, A, h + 1, p);
}

// One node of the lane's current subtree: label S reached with (h, p).
// Leaves and closed forms clear `has`; otherwise hold children of three or
// more members are pushed and the lane moves to the pivot child.
__device__ __forceinline__ void lane_node(LaneWork &L, unsigned *sh32, const CountArgs &A, int lane,
                                          uint32_t &S, int &h, int &p, bool &has, unsigned &top, unsigned bot,
                                          LaneCounters &lc)
{
    const int s = __popc(S);
    ++lc.nodes;
    if (s == 0) {
        ++lc.leaves;
        lane_tally(sh32, A, h, p);
        has = false;
        return;
    }
    // pivot: most neighbours inside S, ties -> lowest index; the degree sum
    // tells whether S is a clique.  Two members per round for two
    // independent load-AND-POPC chains.
    uint32_t best = 0, dsum = 0, x = S;
    while (x) {
        const int v = __ffs(x) - 1;
        x &= x - 1;
        const uint32_t c = __popc(L.rows[v][lane] & S);
        best = max(best, (c << 5) | (31u - (uint32_t)v));
        dsum += c;
        if (x) {
            const int u = __ffs(x) - 1;
            x &= x - 1;
            const uint32_t c2 = __popc(L.rows[u][lane] & S);
            best = max(best, (c2 << 5) | (31u - (uint32_t)u));
            dsum += c2;
        }
    }
    lc.words += (unsigned)s;
    if (dsum == (uint32_t)s * (uint32_t)(s - 1)) {
        ++lc.leaves;
        lane_tally(sh32, A, h, p + s);
        has = false;
        return;
    }
    const int piv = 31 - (int)(best & 31u);
    const uint32_t rp = L.rows[piv][lane];
    if (h + 1 <= A.kmax) {
        // hold children N(S, v_i) minus the earlier non-neighbours, ascending
        uint32_t y = S & ~rp & ~(1u << piv), below = 0;
        while (y) {
            const int v = __ffs(y) - 1;
            y &= y - 1;
            const uint32_t child = L.rows[v][lane] & S & ~below;
            below |= 1u << v;
            const int cs = __popc(child);
            if (cs <= 2) {
                const bool adj = cs == 2 && ((L.rows[__ffs(child) - 1][lane] >> (31 - __clz(child))) & 1u);
                lane_close_small(sh32, A, cs, adj, h + 1, p, lc);
            } else {
                L.stkS[top & (LSTK - 1)][lane] = child;
                L.stkHP[top & (LSTK - 1)][lane] = ((uint32_t)(h + 1) << 16) | (uint32_t)p;
                ++top;
            }
        }
        if (top - bot > (unsigned)LSTK) atomicOr(A.err, DERR_STACK);  // cannot happen (at most 31 pending)
    }
    // the pivot child N(S, piv), closed at once if it has at most two members
    const uint32_t P = rp & S;
    const int ps = __popc(P);
    if (ps <= 2) {
        const bool adj = ps == 2 && ((L.rows[__ffs(P) - 1][lane] >> (31 - __clz(P))) & 1u);
        lane_close_small(sh32, A, ps, adj, h, p + 1, lc);
        has = false;
    } else {
        S = P;
        p += 1;
    }
}

// Lanes of `freeM` without a source item take the oldest pending entry of a
// busy lane (one that keeps work), with that lane's rows.  Returns the
// lanes that received one.
__device__ __forceinline__ unsigned lane_steal(LaneWork &L, int lane, unsigned freeM, uint32_t &S, int &h, int &p,
                                               bool &has, unsigned top, unsigned &bot)
{
    const unsigned pend = top - bot;
    const unsigned donors = __ballot_sync(FULL, pend >= 2 || (pend == 1 && has));
    const int np = min(__popc(freeM), __popc(donors));
    if (np == 0) return 0u;
    const unsigned lt = (1u << lane) - 1u;
    int src = lane;  // the donor this lane receives from
    bool recv = false;
    if ((freeM >> lane) & 1u) {
        const int rank = __popc(freeM & lt);
        if (rank < np) {
            unsigned m = donors;  // the rank-th donor, counting from bit 0
            for (int k = 0; k < rank; ++k) m &= m - 1;
            src = __ffs(m) - 1;
            recv = true;
        }
    }
    const unsigned sbot = __shfl_sync(FULL, bot, src);
    if (recv) {
        S = L.stkS[sbot & (LSTK - 1)][src];
        const uint32_t hp = L.stkHP[sbot & (LSTK - 1)][src];
        h = (int)(hp >> 16);
        p = (int)(hp & 0xFFFFu);
        for (int v = 0; v < 32; ++v) L.rows[v][lane] = L.rows[v][src];
        has = true;
    }
    if ((donors >> lane) & 1u) {
        if (__popc(donors & lt) < np) ++bot;
    }
    __syncwarp();
    return __ballot_sync(FULL, recv);
}

// Lane j takes frame `item` of the emitted buffer: its 32 rows into column j
// with eight 16-byte loads (every lane its own frame, so the warp's stores
// hit 32 distinct banks), its label and (h, p).
__device__ __forceinline__ void lane_load_frame(LaneWork &L, const uint32_t *fr, int lane, uint32_t &S, int &h,
                                                int &p)
{
    const uint4 *v = reinterpret_cast<const uint4 *>(fr + 4);
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const uint4 x = __ldcs(v + q);
        L.rows[4 * q + 0][lane] = x.x;
        L.rows[4 * q + 1][lane] = x.y;
        L.rows[4 * q + 2][lane] = x.z;
        L.rows[4 * q + 3][lane] = x.w;
    }
    const uint4 head = __ldcs(reinterpret_cast<const uint4 *>(fr));
    S = head.z;
    h = (int)(head.y >> 16);
    p = (int)(head.y & 0xFFFFu);
}

constexpr unsigned LANE_CLAIM = 32;  // source items a warp claims at once

// The lane walk over the first `nitems` emitted frames (A.emit).  A warp
// claims LANE_CLAIM frames at a time through qctl[Q_ROOT] and hands them to
// its free lanes; qctl[Q_OUT] counts items not yet finished (a warp
// returns its items once every lane is idle), and warps that run dry wait on
// the ring queue for donated frames until it drops to zero (walk.cuh:
// queue_take).
__device__ inline void lane_walk(LaneWork &L, unsigned *sh32, const CountArgs &A, int lane, unsigned nitems, int slot)
{
    LaneCounters lc;
    uint32_t S = 0;
    int h = 0, p = 0;
    bool has = false;
    unsigned top = 0, bot = 0;
    unsigned held = 0;           // items this warp took and has not returned (uniform)
    unsigned cur = 0, end = 0;   // claimed, not yet started items [cur, end) (uniform)
    bool src_done = false;       // uniform
    unsigned steps = 0;
    for (;;) {
        unsigned freeM = __ballot_sync(FULL, !has && top == bot);
        if (freeM && !src_done) {
            if (cur == end) {
                unsigned base = nitems;
                if (lane == 0 && vload(A.qctl + Q_ROOT) < nitems) base = atomicAdd(A.qctl + Q_ROOT, LANE_CLAIM);
                base = __shfl_sync(FULL, base, 0);
                if (base >= nitems) {
                    src_done = true;
                } else {
                    cur = base;
                    end = min(base + LANE_CLAIM, nitems);
                    if (lane < (int)(end - cur)) {
                        // the claimed frames into L2 ahead of their lanes
                        const char *a = reinterpret_cast<const char *>(A.emit + (size_t)(cur + lane) * FRAME_WORDS);
                        asm volatile("prefetch.global.L2 [%0];" ::"l"(a));
                        asm volatile("prefetch.global.L2 [%0];" ::"l"(a + 128));
                    }
                }
            }
            if (cur < end) {
                // the first free lanes take items cur, cur+1, ...
                const unsigned got = min((unsigned)__popc(freeM), end - cur);
                const unsigned rank = (unsigned)__popc(freeM & ((1u << lane) - 1u));
                if (((freeM >> lane) & 1u) && rank < got) {
                    lane_load_frame(L, A.emit + (size_t)(cur + rank) * FRAME_WORDS, lane, S, h, p);
                    has = true;
                }
                cur += got;
                held += got;
                __syncwarp();
                freeM = __ballot_sync(FULL, !has && top == bot);
            }
        }
        if (freeM && src_done) {
            lane_steal(L, lane, freeM, S, h, p, has, top, bot);
            freeM = __ballot_sync(FULL, !has && top == bot);
            if (freeM == FULL) {
                // every lane idle: return this warp's items, then wait for a
                // donated frame (or the end of the launch)
                if (lane == 0 && held) atomicSub(A.qctl + Q_OUT, held);
                held = 0;
                unsigned v = 0;
                int kind = lane == 0 ? queue_take(A, 0u, v) : 0;
                kind = __shfl_sync(FULL, kind, 0);
                v = __shfl_sync(FULL, v, 0);
                if (kind != 1) break;
                const uint32_t *fr = A.qframes + (size_t)(v & (A.qcap - 1u)) * FRAME_WORDS;
                if (lane == 0) {
                    const uint32_t hp = __ldcg(fr + 1);
                    S = __ldcg(fr + 2);
                    h = (int)(hp >> 16);
                    p = (int)(hp & 0xFFFFu);
                    for (int v2 = 0; v2 < 32; ++v2) L.rows[v2][0] = __ldcg(fr + 4 + v2);
                    __threadfence();
                    atomicExch(A.qdone + (v & (A.qcap - 1u)), v + 1u);
                    has = true;
                }
                held = 1;
                __syncwarp();
                continue;
            }
        }
        // one node per lane that has work
        if (!has && top != bot) {
            --top;
            S = L.stkS[top & (LSTK - 1)][lane];
            const uint32_t hp = L.stkHP[top & (LSTK - 1)][lane];
            h = (int)(hp >> 16);
            p = (int)(hp & 0xFFFFu);
            has = true;
        }
        if (has) lane_node(L, sh32, A, lane, S, h, p, has, top, bot, lc);
        __syncwarp();
        if (++steps % LANE_DONATE_EVERY == 0) {
            // warps wait on the ring: donate, for up to LANE_DONATE_MAX of
            // them, the oldest pending entry of the lane with the most pending
            // entries, with that lane's rows
            unsigned waiters = lane == 0 ? queue_waiters(A, LANE_DONATE_MAX) : 0u;
            waiters = __shfl_sync(FULL, waiters, 0);
            for (unsigned d = 0; d < waiters; ++d) {
                const unsigned pend = top - bot;
                const unsigned key =
                    pend >= 2 && __popc(L.stkS[bot & (LSTK - 1)][lane]) >= DONATE_MIN_COMPACT ? (pend << 5) | (unsigned)lane : 0u;
                const unsigned best = __reduce_max_sync(FULL, key);
                if (!best) break;
                const int dl = (int)(best & 31u);
                unsigned t = 0;
                uint32_t *fr = frame_reserve(A, lane, t);
                if (!fr) break;
                fr[4 + lane] = L.rows[lane][dl];
                if (lane == dl) {
                    fr[0] = FRAME_COMPACT;
                    fr[1] = L.stkHP[bot & (LSTK - 1)][lane];
                    fr[2] = L.stkS[bot & (LSTK - 1)][lane];
                    fr[3] = (uint32_t)A.cls;
                    ++bot;
                }
                frame_publish(A, lane, t);
            }
        }
    }
    lc.flush(A.stats, slot, lane);
}

constexpr size_t lane_smem_bytes() { return sizeof(LaneWork) * LANE_WPB + sizeof(unsigned) * HIST_H * HIST_P; }

}  // namespace pvt
