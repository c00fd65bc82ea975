// CTA-per-root walk of the heaviest roots (global counts).
//
// A root of out-degree d keeps the adjacency induced on N+(r) as d rows of
// ceil(d/32) words (step 1 of walk.cuh).  For d in the hundreds these rows
// fill most of an SM's shared memory, so a kernel that gives each warp its
// own root keeps a single warp per SM.  Here a thread block owns one root at
// a time: its threads gather the rows together once, and all of its warps
// walk that root's SCT (Alg. 1) over the one shared copy.  The warps share
// the root's subtrees through a small queue in shared memory: a warp whose
// subtree is done takes the next pending one, and busy warps hand over
// their oldest pending subtree (the largest) while a warp of the block has
// none.  Labels of at most 32 members leave the wide walk: they are
// relabelled to one-word rows (the ballots of compact_rows in walk.cuh) into
// a free lane of the warp's lane batch and walked one subtree per lane
// (lanes.cuh), so the many small subtrees below a dense root never leave the
// SM.  A warp runs its lanes whenever it has no wide work or no free lane.
// The tree, its statistics and the (h, p) histogram are those of walk.cuh.
#pragma once

#include "lanes.cuh"

namespace pvt {

constexpr int CTA_QCAP = 32;                 // pending wide subtrees a block's queue holds
constexpr int CTA_CQCAP = 64;                // relabelled small subtrees it holds
constexpr int CTA_MAXW = 16;                 // warps per block at most
constexpr unsigned CTA_DONATE_EVERY = 2;     // wide nodes between looks at the block's queue
constexpr unsigned CTA_LANE_SLICE = 64;      // lane steps between looks while waiting
constexpr unsigned long long CTA_LOCK_LIMIT_NS = 2000000000ull;  // 2 s for the block's queue lock
// Labels of 33..128 members below a wider root are relabelled to rows of
// MID_NW words (in the warp's shared memory) and walked there: a pivot word
// pair then costs a 4-word row instead of the root's NW words.
constexpr int MID_NW = 4, MID_RS = 5, MID_D = 32 * MID_NW;
// ... when at least this many hold levels may still follow (kmax - h): the
// relabelling costs up to |S| * MID_NW ballots, which a subtree cut a level
// or two further down does not pay back
constexpr int CTA_MID_DEPTH = 3;

// Per-warp shared state of the CTA walk beside its lane batch: the rows of a
// relabelled mid-size label and the member list of a label being relabelled.
struct alignas(16) CtaWarp {
    uint32_t mid[MID_D * MID_RS];
    uint16_t mem[MID_D];
};

// Shared state of a block, before the per-warp lane batches.
template <int NW>
struct alignas(16) CtaQueue {
    int lock;
    int head, tail;       // pending wide subtrees q[head .. tail)
    int busy;             // warps walking a wide subtree of the current root
    unsigned progress;    // bumped by every take and every finish (bounded waits)
    unsigned root;        // index of the current root in the class list (~0: stop)
    int d;                // its out-degree
    int chead, ctail;     // relabelled small subtrees taken / reserved
    uint32_t S[CTA_QCAP][NW];
    uint32_t hp[CTA_QCAP];
    // relabelled small subtrees: one-word rows, label, (h, p); an entry t is
    // published when cseq[t % CTA_CQCAP] == t + 1
    uint32_t crow[CTA_CQCAP][33];  // odd stride: takers of different entries hit distinct banks
    uint32_t cS[CTA_CQCAP], chp[CTA_CQCAP], cseq[CTA_CQCAP];
    // each warp's current label S and non-neighbour set R, for reads of word
    // j by a loop index (registers hold them for the unrolled word loops)
    uint32_t wS[CTA_MAXW][NW], wR[CTA_MAXW][NW];
    uint32_t wM[CTA_MAXW][32];  // the members of a small label being relabelled
};

template <int NW>
struct CtaLayout {
    static constexpr int RS = (NW & 1) ? NW : NW + 1;  // odd row stride: no bank conflicts
    // dynamic shared memory: queue, per-warp lane batches, block histogram,
    // then the root's rows (dmax rows of RS words)
    __host__ __device__ static size_t bytes(int warps, int dmax)
    {
        return sizeof(CtaQueue<NW>) + (sizeof(LaneWork) + sizeof(CtaWarp)) * warps +
               sizeof(unsigned) * HIST_H * HIST_P + (size_t)dmax * RS * sizeof(uint32_t);
    }
    // per warp in global memory: the DFS stack of the root's level, then
    // that of the mid level
    __host__ __device__ static size_t stack_words(int dmax)
    {
        return (size_t)(dmax + 1) * (NW + 1) + (size_t)(MID_D + 1) * (MID_NW + 1);
    }
    // global scratch of a block's gather: member ids, prefix offsets (dmax + 2
    // words) and out-list starts (dmax 8-byte words)
    __host__ __device__ static size_t gather_words(int dmax) { return (size_t)(2 * dmax + 2) + 2 * (size_t)dmax; }
};

// The lane state of one lane (registers): its current subtree node and stack.
struct LaneState {
    uint32_t S = 0;
    int h = 0, p = 0;
    bool has = false;
    unsigned top = 0, bot = 0;
    __device__ __forceinline__ bool free_() const { return !has && top == bot; }
};

// The subtree of a label of at most two members in closed form (the cases
// of close_small in walk.cuh), tallied in the block's 32-bit histogram.
// UNIFORM: every lane calls with the same arguments, lane 0 tallies.
template <bool UNIFORM>
__device__ __forceinline__ void cta_close_small(unsigned *sh32, const CountArgs &A, int lane, int cs, bool adjacent,
                                                int h, int p, unsigned wpm, WalkCounters &wc)
{
    const bool split = cs == 2 && !adjacent;
    const bool hold = split && h + 1 <= A.kmax;
    if (UNIFORM) {
        wc.nodes += 1 + split + hold;
        wc.leaves += 1 + hold;
        wc.words += (unsigned long long)cs * wpm;
    } else {
        wc.xnodes += 1u + split + hold;
        wc.xleaves += 1u + hold;
        wc.xwords += (unsigned)cs * wpm;
    }
    if (UNIFORM && lane != 0) return;
    if (!split) {
        lane_tally(sh32, A, h, p + cs);
        return;
    }
    lane_tally(sh32, A, h, p + 1);  // the pivot leaf below the pair
    if (hold) lane_tally(sh32, A, h + 1, p);
}

// Run the warp's lane batch: at most `budget` node steps, stopping early
// once `stop_free` lanes are free (0: only when every lane is idle).
__device__ inline void lane_run(LaneWork &L, unsigned *sh32, const CountArgs &A, int lane, LaneState &ls,
                         LaneCounters &lc, unsigned budget, int stop_free)
{
    for (unsigned step = 0; step < budget; ++step) {
        const unsigned freeM = __ballot_sync(FULL, ls.free_());
        if (freeM == FULL) return;
        if (stop_free && __popc(freeM) >= stop_free) return;
        if (freeM) lane_steal(L, lane, freeM, ls.S, ls.h, ls.p, ls.has, ls.top, ls.bot);
        if (!ls.has && ls.top != ls.bot) {
            --ls.top;
            ls.S = L.stkS[ls.top & (LSTK - 1)][lane];
            const uint32_t hp = L.stkHP[ls.top & (LSTK - 1)][lane];
            ls.h = (int)(hp >> 16);
            ls.p = (int)(hp & 0xFFFFu);
            ls.has = true;
        }
        if (ls.has) lane_node(L, sh32, A, lane, ls.S, ls.h, ls.p, ls.has, ls.top, ls.bot, lc);
        __syncwarp();
    }
}

// Relabel the warp's current label (wS: NW-word bitset over the root's
// members, s <= 32 of them): member k of the label = its k-th member in
// ascending order; lane k returns row k of the one-word adjacency (the
// ballot over lanes j of "member k is adjacent to member j").
template <int NW, int RS>
__device__ __forceinline__ uint32_t relabel_small(const uint32_t *adj, const uint32_t *wS, uint32_t *wM, int lane,
                                                  int s)
{
    int before = 0;
    for (int w = 0; w < NW; ++w) {
        const uint32_t sw = wS[w];
        if ((sw >> lane) & 1u) wM[before + __popc(sw & ((1u << lane) - 1u))] = (uint32_t)(w * 32 + lane);
        before += __popc(sw);
    }
    __syncwarp();
    const uint32_t mj = lane < s ? wM[lane] : 0u;
    uint32_t mine = 0;
    for (int k = 0; k < s; ++k) {
        const uint32_t mk = __shfl_sync(FULL, mj, k);
        const bool bit = lane < s && ((adj[mj * RS + (mk >> 5)] >> (mk & 31)) & 1u);
        const uint32_t row = __ballot_sync(FULL, bit);
        if (lane == k) mine = row;
    }
    __syncwarp();
    return mine;
}

// A relabelled small label into a free lane of the warp's own batch (run
// the batch until a lane is free first).
__device__ __forceinline__ void lane_add(LaneWork &L, unsigned *sh32, const CountArgs &A, int lane, LaneState &ls,
                                         LaneCounters &lc, uint32_t row, int s, int h, int p)
{
    unsigned freeM = __ballot_sync(FULL, ls.free_());
    if (!freeM) {
        lane_run(L, sh32, A, lane, ls, lc, 0xFFFFFFFFu, 1);
        freeM = __ballot_sync(FULL, ls.free_());
    }
    const int slot = __ffs(freeM) - 1;
    L.rows[lane][slot] = row;
    __syncwarp();
    if (lane == slot) {
        ls.S = s >= 32 ? FULL : ((1u << s) - 1u);
        ls.h = h;
        ls.p = p;
        ls.has = true;
        ls.top = ls.bot = 0;
    }
    __syncwarp();
}

// Block-wide lock of the queue (lane 0 of a warp), bounded.
__device__ __forceinline__ bool cta_lock(int *lk, unsigned *err)
{
    const unsigned long long t0 = global_ns();
    while (atomicCAS(lk, 0, 1) != 0) {
        if (global_ns() - t0 > CTA_LOCK_LIMIT_NS) {
            atomicOr(err, DERR_TIMEOUT);
            return false;
        }
        __nanosleep(32);
    }
    __threadfence_block();
    return true;
}
__device__ __forceinline__ void cta_unlock(int *lk)
{
    __threadfence_block();
    atomicExch(lk, 0);
}

// A small label (s <= 32 members) found by a wide walk: relabelled into the
// block's ring, from which any warp with free lanes takes it; into the
// warp's own batch when the ring is full.
template <int NW, int LNW, int RS>
__device__ __forceinline__ void cta_push_small(CtaQueue<NW> &Q, LaneWork &L, unsigned *sh32, const CountArgs &A,
                                               int lane, int wid, LaneState &ls, LaneCounters &lc,
                                               const uint32_t *adj, int s, int h, int p)
{
    const uint32_t row = relabel_small<LNW, RS>(adj, Q.wS[wid], Q.wM[wid], lane, s);
    int t = -1;
    if (lane == 0 && *(volatile int *)&Q.ctail - *(volatile int *)&Q.chead < CTA_CQCAP && cta_lock(&Q.lock, A.err)) {
        if (Q.ctail - Q.chead < CTA_CQCAP) t = Q.ctail++;
        cta_unlock(&Q.lock);
    }
    t = __shfl_sync(FULL, t, 0);
    if (t < 0) {
        lane_add(L, sh32, A, lane, ls, lc, row, s, h, p);
        return;
    }
    const int e = t % CTA_CQCAP;
    Q.crow[e][lane] = row;
    if (lane == 0) {
        Q.cS[e] = s >= 32 ? FULL : ((1u << s) - 1u);
        Q.chp[e] = ((uint32_t)h << 16) | (uint32_t)p;
    }
    __syncwarp();
    if (lane == 0) {
        __threadfence_block();
        *(volatile uint32_t *)&Q.cseq[e] = (uint32_t)t + 1u;
    }
}

// Free lanes of the warp take published small labels from the block's ring
// (copied out under the lock, so a slot is reused only once copied).
// Returns how many were taken.
template <int NW>
__device__ __forceinline__ int cta_take_small(CtaQueue<NW> &Q, LaneWork &L, int lane, LaneState &ls, unsigned *err)
{
    const unsigned freeM = __ballot_sync(FULL, ls.free_());
    if (!freeM) return 0;
    int base = 0, n = 0;
    if (lane == 0 && *(volatile int *)&Q.ctail > *(volatile int *)&Q.chead && cta_lock(&Q.lock, err)) {
        base = Q.chead;
        const int lim = min(__popc(freeM), Q.ctail - Q.chead);
        while (n < lim && *(volatile uint32_t *)&Q.cseq[(base + n) % CTA_CQCAP] == (uint32_t)(base + n) + 1u) ++n;
        if (n == 0) cta_unlock(&Q.lock);
    }
    n = __shfl_sync(FULL, n, 0);
    if (n == 0) return 0;
    base = __shfl_sync(FULL, base, 0);
    __threadfence_block();
    const int rank = __popc(freeM & ((1u << lane) - 1u));
    if (((freeM >> lane) & 1u) && rank < n) {
        const int e = (base + rank) % CTA_CQCAP;
        for (int v = 0; v < 32; ++v) L.rows[v][lane] = Q.crow[e][v];
        ls.S = Q.cS[e];
        const uint32_t hp = Q.chp[e];
        ls.h = (int)(hp >> 16);
        ls.p = (int)(hp & 0xFFFFu);
        ls.has = true;
        ls.top = ls.bot = 0;
    }
    __syncwarp();
    if (lane == 0) {
        Q.chead = base + n;
        Q.progress += 1;
        cta_unlock(&Q.lock);
    }
    __syncwarp();
    return n;
}

// One level of the walk: the subtree of label S (LNW-word bitset over the
// rows `rows`, stride RS: the root's rows at the top level, a relabelled
// mid-size label's at the mid level) reached with (h, p), depth first, its
// pending children on the warp's stack `stk` in global memory (at most
// cap + 1 frames of LNW + 1 words).  Labels of at most 32 members go to the
// lanes (the block's ring, else the warp's own batch); at the top level a
// label of 33..MID_D members over wider rows is relabelled to MID_NW-word
// rows in the warp's shared memory and walked there first (unless kmax
// truncates its subtree within CTA_MID_DEPTH hold levels), and pending
// subtrees are handed to idle warps of the block.  The current label lives
// in registers S[w] (word loops are unrolled) and in the warp's wS copy
// (reads of word j by loop index).
template <int NW, int LNW, int RS, bool TOP>
__device__ __forceinline__ void cta_level(CtaQueue<NW> &Q, CtaWarp &CW, LaneWork &L, unsigned *sh32,
                                          const CountArgs &A, int lane, int wid, LaneState &ls, LaneCounters &lc,
                                          WalkCounters &wc, const uint32_t *rows, uint32_t *stk, uint32_t *mstk,
                                          uint32_t (&S)[LNW], int h, int p, int cap)
{
    constexpr int FW = LNW + 1;  // stack frame words: S, then (h << 16) | p
    uint32_t *wS = Q.wS[wid], *wR = Q.wR[wid];
    int top = 0, bot = 0;
    unsigned clock = 0;
    const uint32_t low = (1u << lane) - 1u;
    const int warps = (int)(blockDim.x >> 5);
    for (;;) {
        int s = 0;
#pragma unroll
        for (int w = 0; w < LNW; ++w) s += __popc(S[w]);
#pragma unroll
        for (int w = 0; w < LNW; ++w)
            if (lane == w) wS[w] = S[w];
        __syncwarp();
        bool closed = true;
        if (s <= 32) {
            cta_push_small<NW, LNW, RS>(Q, L, sh32, A, lane, wid, ls, lc, rows, s, h, p);
        } else if (TOP && LNW > MID_NW && s <= MID_D && A.kmax - h >= CTA_MID_DEPTH) {
            // relabel the members to 0..s-1 and walk the label over MID_NW-word rows
            int before = 0;
#pragma unroll
            for (int w = 0; w < LNW; ++w) {
                if ((S[w] >> lane) & 1u) CW.mem[before + __popc(S[w] & low)] = (uint16_t)(w * 32 + lane);
                before += __popc(S[w]);
            }
            __syncwarp();
            uint32_t mj[MID_NW];
#pragma unroll
            for (int q = 0; q < MID_NW; ++q) mj[q] = q * 32 + lane < s ? CW.mem[q * 32 + lane] : 0u;
            for (int k = 0; k < s; ++k) {
                const uint32_t mk = CW.mem[k];
                uint32_t word = 0;
#pragma unroll
                for (int q = 0; q < MID_NW; ++q) {
                    const bool bit = q * 32 + lane < s && ((rows[mj[q] * RS + (mk >> 5)] >> (mk & 31)) & 1u);
                    const uint32_t b = __ballot_sync(FULL, bit);
                    if (lane == q) word = b;
                }
                if (lane < MID_NW) CW.mid[k * MID_RS + lane] = word;
            }
            __syncwarp();
            uint32_t M[MID_NW];
#pragma unroll
            for (int q = 0; q < MID_NW; ++q) {
                const int bits = s - 32 * q;
                M[q] = bits >= 32 ? FULL : (bits <= 0 ? 0u : ((1u << bits) - 1u));
            }
            cta_level<NW, MID_NW, MID_RS, false>(Q, CW, L, sh32, A, lane, wid, ls, lc, wc, CW.mid, mstk, nullptr, M,
                                                 h, p, MID_D);
        } else {
            wc.nodes++;
            ++clock;
            // pivot: most neighbours inside S, ties -> lowest member index
            uint32_t best = 0, dsum = 0;
            for (int j = 0; j < LNW; ++j) {
                if ((wS[j] >> lane) & 1u) {
                    const uint32_t *row = rows + (j * 32 + lane) * RS;
                    uint32_t c = 0;
#pragma unroll
                    for (int w = 0; w < LNW; ++w) c += __popc(row[w] & S[w]);
                    best = max(best, ((c + 1u) << 10) | (1023u - (uint32_t)(j * 32 + lane)));
                    dsum += c;
                }
            }
            best = __reduce_max_sync(FULL, best);
            dsum = __reduce_add_sync(FULL, dsum);
            wc.words += (unsigned long long)s * (unsigned)((s + 31) >> 5);
            const int piv = 1023 - (int)(best & 1023u);
            if (dsum == (uint32_t)s * (uint32_t)(s - 1)) {
                wc.leaves++;
                if (lane == 0) lane_tally(sh32, A, h, p + s);
            } else {
                const uint32_t *prow = rows + piv * RS;
                uint32_t R[LNW];
                int nR = 0;
#pragma unroll
                for (int w = 0; w < LNW; ++w) {
                    R[w] = S[w] & ~prow[w];
                    if (w == (piv >> 5)) R[w] &= ~(1u << (piv & 31));
                    nR += __popc(R[w]);
                }
#pragma unroll
                for (int w = 0; w < LNW; ++w)
                    if (lane == w) wR[w] = R[w];
                __syncwarp();
                if (nR > 0 && h + 1 <= A.kmax) {
                    if (top + nR > cap + 1) {
                        if (bot > 0) {
                            // donated frames left room at the base: move the live ones down
                            for (int t = lane; t < (top - bot) * FW; t += 32) stk[t] = stk[bot * FW + t];
                            top -= bot;
                            bot = 0;
                            __syncwarp();
                        }
                        if (top + nR > cap + 1) {
                            if (lane == 0) atomicOr(A.err, DERR_STACK);
                            return;
                        }
                    }
                    // hold child of member j*32+lane: N(S, v) minus the earlier
                    // members of R; labels of at most two members close here
                    int before = 0;
                    for (int j = 0; j < LNW; ++j) {
                        const uint32_t Rj = wR[j];
                        const bool inR = (Rj >> lane) & 1u;
                        bool push = inR;
                        const uint32_t *row = rows + (j * 32 + lane) * RS;
                        if (inR) {
                            int cs = 0, a = 0, b = 0;
#pragma unroll
                            for (int w = 0; w < LNW; ++w) {
                                const uint32_t bl = w < j ? R[w] : (w == j ? (Rj & low) : 0u);
                                const uint32_t cw = row[w] & S[w] & ~bl;
                                if (cw) {
                                    if (cs == 0) a = w * 32 + __ffs(cw) - 1;
                                    b = w * 32 + 31 - __clz(cw);
                                }
                                cs += __popc(cw);
                            }
                            if (cs <= 2) {
                                const bool adjp = cs == 2 && ((rows[a * RS + (b >> 5)] >> (b & 31)) & 1u);
                                cta_close_small<false>(sh32, A, lane, cs, adjp, h + 1, p, 1u, wc);
                                push = false;
                            }
                        }
                        const uint32_t pushed = __ballot_sync(FULL, push);
                        if (push) {
                            uint32_t *fr = stk + (size_t)(top + before + __popc(pushed & low)) * FW;
#pragma unroll
                            for (int w = 0; w < LNW; ++w) {
                                const uint32_t bl = w < j ? R[w] : (w == j ? (Rj & low) : 0u);
                                fr[w] = row[w] & S[w] & ~bl;
                            }
                            fr[LNW] = ((uint32_t)(h + 1) << 16) | (uint32_t)p;
                        }
                        before += __popc(pushed);
                    }
                    top += before;
                    __syncwarp();
                    if (TOP && clock >= CTA_DONATE_EVERY) {
                        clock = 0;
                        // a warp of the block is not walking a wide subtree: hand
                        // it our oldest pending one (the largest), if there is room
                        int give = 0;
                        if (lane == 0 && top - bot >= 2 && *(volatile int *)&Q.busy < warps &&
                            *(volatile int *)&Q.tail - *(volatile int *)&Q.head < CTA_QCAP) {
                            int sz = 0;
                            for (int w = 0; w < LNW; ++w) sz += __popc(stk[bot * FW + w]);
                            if (sz >= DONATE_MIN_WIDE && cta_lock(&Q.lock, A.err)) {
                                give = 1;
                                if (Q.tail - Q.head >= CTA_QCAP) {
                                    cta_unlock(&Q.lock);
                                    give = 0;
                                }
                            }
                        }
                        give = __shfl_sync(FULL, give, 0);
                        if (give) {
                            const int slot = Q.tail % CTA_QCAP;
                            if (lane < LNW) Q.S[slot][lane] = stk[bot * FW + lane];
                            if (lane == 0) Q.hp[slot] = stk[bot * FW + LNW];
                            __syncwarp();
                            if (lane == 0) {
                                Q.tail += 1;
                                Q.progress += 1;
                                cta_unlock(&Q.lock);
                            }
                            ++bot;
                        }
                    }
                }
                // continue into the pivot child N(S, piv), or close it at once
                int ps = 0, a = 0, b = 0;
                uint32_t P[LNW];
#pragma unroll
                for (int w = 0; w < LNW; ++w) {
                    P[w] = prow[w] & S[w];
                    if (P[w]) {
                        if (ps == 0) a = w * 32 + __ffs(P[w]) - 1;
                        b = w * 32 + 31 - __clz(P[w]);
                    }
                    ps += __popc(P[w]);
                }
                if (ps <= 2) {
                    const bool adjp = ps == 2 && ((rows[a * RS + (b >> 5)] >> (b & 31)) & 1u);
                    cta_close_small<true>(sh32, A, lane, ps, adjp, h, p + 1, 1u, wc);
                } else {
                    closed = false;
#pragma unroll
                    for (int w = 0; w < LNW; ++w) S[w] = P[w];
                    p += 1;
                }
            }
        }
        __syncwarp();
        if (!closed) continue;
        if (top == bot) break;
        --top;
#pragma unroll
        for (int w = 0; w < LNW; ++w) S[w] = stk[top * FW + w];
        const uint32_t hp = stk[top * FW + LNW];
        h = (int)(hp >> 16);
        p = (int)(hp & 0xFFFFu);
    }
    __syncwarp();
}

// Walk the wide subtree of the label in queue slot `qs` (NW words over the
// root's rows): copied out under the caller's lock, which is then released.
template <int NW>
__device__ __forceinline__ void cta_dfs(CtaQueue<NW> &Q, CtaWarp &CW, LaneWork &L, unsigned *sh32,
                                        const CountArgs &A, int lane, int wid, LaneState &ls, LaneCounters &lc,
                                        WalkCounters &wc, const uint32_t *adj, uint32_t *gstk, int qs, int d)
{
    uint32_t S[NW];
#pragma unroll
    for (int w = 0; w < NW; ++w) S[w] = Q.S[qs][w];
    const uint32_t hp0 = Q.hp[qs];
    __syncwarp();
    if (lane == 0) {
        Q.progress += 1;
        cta_unlock(&Q.lock);
    }
    uint32_t *mstk = gstk + (size_t)(d + 1) * (NW + 1);
    cta_level<NW, NW, CtaLayout<NW>::RS, true>(Q, CW, L, sh32, A, lane, wid, ls, lc, wc, adj, gstk, mstk, S,
                                               (int)(hp0 >> 16), (int)(hp0 & 0xFFFFu), d);
}

// The block's rows for root r (all threads): member ids, their out-list
// starts and the prefix offsets of their lengths in the block's global
// scratch (gather_words), then every entry of the members' out-lists looked
// up among the members by binary search.  Q.d receives the out-degree (0
// after a range error).
template <int NW>
__device__ void cta_gather(CtaQueue<NW> &Q, uint32_t *scratch, uint32_t *adj, const CountArgs &A, uint32_t r,
                           int dmax)
{
    constexpr int RS = CtaLayout<NW>::RS;
    const int64_t rbeg = A.orow[r];
    const int d = (int)(A.orow[r + 1] - rbeg);
    uint32_t *ids = scratch;
    uint32_t *off = ids + dmax;                                  // d + 1 prefix offsets
    int64_t *rs = reinterpret_cast<int64_t *>(off + dmax + 2);   // 8-byte aligned: 2 dmax + 2 words before
    const int tid = threadIdx.x, nt = blockDim.x;
    __shared__ uint32_t wsum[32];
    if (d > 32 * NW || d > dmax) {
        if (tid == 0) {
            atomicOr(A.err, DERR_RANGE);
            Q.d = 0;
        }
        __syncthreads();
        return;
    }
    for (int t = tid; t < d * RS; t += nt) adj[t] = 0;
    // member i: id, out-list start, length; block scan of the lengths
    const int lane = tid & 31, wid = tid >> 5, nw = nt >> 5;
    uint32_t carry = 0;
    for (int i0 = 0; i0 < d; i0 += nt) {
        const int i = i0 + tid;
        uint32_t od = 0;
        if (i < d) {
            const uint32_t id = A.ocol[rbeg + i];
            const int64_t b = A.orow[id];
            od = (uint32_t)(A.orow[id + 1] - b);
            ids[i] = id;
            rs[i] = b;
        }
        uint32_t inc = od;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(FULL, inc, o);
            if (lane >= o) inc += t;
        }
        if (lane == 31) wsum[wid] = inc;
        __syncthreads();
        if (wid == 0) {
            uint32_t x = lane < nw ? wsum[lane] : 0u;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t t = __shfl_up_sync(FULL, x, o);
                if (lane >= o) x += t;
            }
            if (lane < nw) wsum[lane] = x;
        }
        __syncthreads();
        const uint32_t wbase = wid ? wsum[wid - 1] : 0u;
        if (i < d) off[i + 1] = carry + wbase + inc;
        carry += wsum[nw - 1];
        __syncthreads();
    }
    if (tid == 0) {
        off[0] = 0;
        Q.d = d;
    }
    __threadfence_block();
    __syncthreads();
    const uint32_t T = off[d];
    for (uint32_t t = tid; t < T; t += nt) {
        // member u owning entry t: the largest u with off[u] <= t
        int lo = 0, hi = d;
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (off[mid] <= t) lo = mid; else hi = mid;
        }
        const uint32_t x = A.ocol[rs[lo] + (t - off[lo])];
        int a = 0, b = d;
        while (a < b) {
            const int mid = (a + b) >> 1;
            if (ids[mid] < x) a = mid + 1; else b = mid;
        }
        if (a < d && ids[a] == x) {
            atomicOr(&adj[lo * RS + (a >> 5)], 1u << (a & 31));
            atomicOr(&adj[a * RS + (lo >> 5)], 1u << (lo & 31));
        }
    }
    __syncthreads();
}

// Persistent blocks over the roots A.roots[0..A.nroots) of one class: each
// block takes a root, gathers it, and its warps walk the root's subtrees.
// dmax: the largest out-degree of the class (rows and stacks are sized by
// it).  A.gstack: per warp a DFS stack of (dmax + 1) * (NW + 1) words, then
// per block the gather's scratch.  The lane batches and the ring of small
// labels carry over from one root to the next: their rows are their own.
template <int NW>
__global__ void __launch_bounds__(32 * CTA_MAXW, 1) k_cta(CountArgs A, int dmax)
{
    extern __shared__ __align__(16) unsigned char smem[];
    CtaQueue<NW> &Q = *reinterpret_cast<CtaQueue<NW> *>(smem);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, warps = blockDim.x >> 5;
    LaneWork *lw = reinterpret_cast<LaneWork *>(smem + sizeof(CtaQueue<NW>));
    CtaWarp *cw = reinterpret_cast<CtaWarp *>(lw + warps);
    unsigned *sh32 = reinterpret_cast<unsigned *>(cw + warps);
    uint32_t *adj = sh32 + HIST_H * HIST_P;
    LaneWork &L = lw[wid];
    const size_t stack_words = CtaLayout<NW>::stack_words(dmax);
    uint32_t *gstk = A.gstack + (size_t)(blockIdx.x * warps + wid) * stack_words;
    uint32_t *gscratch = A.gstack + (size_t)gridDim.x * warps * stack_words +
                         (size_t)blockIdx.x * CtaLayout<NW>::gather_words(dmax);
    LaneState ls;
    LaneCounters lc;
    WalkCounters wc;
    for (int i = threadIdx.x; i < HIST_H * HIST_P; i += blockDim.x) sh32[i] = 0;
    for (int i = threadIdx.x; i < CTA_CQCAP; i += blockDim.x) Q.cseq[i] = 0;
    if (threadIdx.x == 0) {
        Q.lock = 0;
        Q.chead = Q.ctail = 0;
    }
    __syncthreads();
    bool more = true;
    while (more) {
        // ---- next root (one decision for the whole block)
        if (threadIdx.x == 0) {
            Q.root = (vload(A.err) & (DERR_STACK | DERR_RANGE | DERR_TIMEOUT)) ? 0xFFFFFFFFu : atomicAdd(A.qhead, 1u);
            Q.head = Q.tail = 0;
            Q.busy = 0;
            Q.progress = 0;
        }
        __syncthreads();
        const unsigned qi = Q.root;
        int d = 0;
        if (qi < A.nroots) {
            cta_gather<NW>(Q, gscratch, adj, A, A.roots[qi], dmax);
            d = Q.d;
            if (threadIdx.x == 0 && d > 0) {
#pragma unroll
                for (int w = 0; w < NW; ++w) {
                    const int bits = d - 32 * w;
                    Q.S[0][w] = bits >= 32 ? FULL : (bits <= 0 ? 0u : ((1u << bits) - 1u));
                }
                Q.hp[0] = 1u << 16;  // h = 1 (the root's hold link), p = 0
                Q.tail = 1;
            }
            __syncthreads();
        } else {
            more = false;  // no root left: finish the ring and the lane batches
        }
        // ---- walk: wide subtrees of the root first, small labels of the
        // ring into free lanes, then the warp's own lanes; the root is done
        // when no wide subtree is pending or walked (the ring and the lanes
        // carry over); the last round ends when the ring is empty too
        unsigned last = 0xFFFFFFFFu;
        unsigned long long t0 = global_ns();
        for (;;) {
            int took = 0;
            if (lane == 0 && more && *(volatile int *)&Q.tail > *(volatile int *)&Q.head) {
                if (cta_lock(&Q.lock, A.err)) {
                    if (Q.tail > Q.head) {
                        took = 1 + (Q.head % CTA_QCAP);
                        Q.head += 1;
                        atomicAdd(&Q.busy, 1);  // the lock is released by cta_dfs once the slot is copied
                    } else {
                        cta_unlock(&Q.lock);
                    }
                } else {
                    took = -1;  // timed out (status set)
                }
            }
            took = __shfl_sync(FULL, took, 0);
            if (took < 0) break;
            if (took > 0) {
                cta_dfs<NW>(Q, cw[wid], L, sh32, A, lane, wid, ls, lc, wc, adj, gstk, took - 1, d);
                wc.fold();
                __syncwarp();
                if (lane == 0) {
                    atomicSub(&Q.busy, 1);
                    atomicAdd(&Q.progress, 1u);
                }
                t0 = global_ns();
                continue;
            }
            if (cta_take_small<NW>(Q, L, lane, ls, A.err) > 0) {
                t0 = global_ns();
                continue;
            }
            if (__ballot_sync(FULL, ls.free_()) != FULL) {
                lane_run(L, sh32, A, lane, ls, lc, CTA_LANE_SLICE, 0);
                t0 = global_ns();
                continue;
            }
            // this warp is idle: is the round over, or has the wait run out?
            // Lane 0 decides for the warp (every lane must leave the loop
            // together: the block barrier below waits for all of them)
            int act = 0;  // 1: the round is over, 2: the wait gave up
            if (lane == 0) {
                const bool wide_done = *(volatile int *)&Q.tail == *(volatile int *)&Q.head &&
                                       *(volatile int *)&Q.busy == 0;
                if (more ? wide_done : wide_done && *(volatile int *)&Q.ctail == *(volatile int *)&Q.chead) {
                    act = 1;
                } else {
                    const unsigned pr = *(volatile unsigned *)&Q.progress;
                    if (pr != last) {
                        last = pr;
                        t0 = global_ns();
                    } else if (global_ns() - t0 > A.idle_ns) {
                        atomicOr(A.err, DERR_TIMEOUT);
                        act = 2;
                    }
                }
            }
            if (__shfl_sync(FULL, act, 0)) break;
            __nanosleep(64);
        }
        __syncthreads();
    }
    wc.flush(A.stats, A.cls, lane);
    lc.flush(A.stats, A.cls, lane);
    lane_hist_flush(sh32, A);
}

}  // namespace pvt
