// Device code of the SCT walk (see the comment below) and the per-class
// launch templates; each walk_nw*.cu instantiates one bitset width.
#pragma once
// SCT walk and clique counts on the device.
//
// For every root r (a child N+(r) of the SCT's root, Alg. 1 step 3) one warp
//   1. gathers the subgraph induced on N+(r) into a shared-memory bitset
//      adjacency: member i = the i-th out-neighbour of r (ascending id); for
//      every member u it scans N+(u) and sets bits i<->j for the members it
//      finds.  Edges among members are undirected (N(S,u) = N(u) cap S,
//      Sec. 3.2), and each appears in exactly one of the two out-lists.
//   2. walks the SCT below N+(r) depth first with an explicit stack of
//      frames (S as a bitset, h, p) (Sec. 4, "Storage cost"): at a node S the
//      pivot is the member of S with most neighbours in S (Alg. 1 pivot step;
//      ties: lowest member index), the pivot child is N(S,p) with p+1, and the
//      non-neighbours v_1 < ... < v_l of the pivot give hold children
//      N(S,v_i) \ {v_1..v_{i-1}} with h+1 (Alg. 1 hold step).  A node whose S
//      is a clique (every member has |S|-1 neighbours in S) has a single
//      root-to-leaf continuation -- each further pivot is adjacent to all of
//      S, so there are no hold children -- and is closed at once as a leaf
//      with p + |S| pivot links.  At most d+1 frames are ever live: a node of size
//      s with l non-neighbours pushes l+1 children, each of size <= s-1-l.
//   3. tallies every leaf (h = |H(T)|, p = |P(T)|, Alg. 2):
//        global  : a 64-bit histogram over (h, p); the counts
//                  C_k = sum hist[h][p] * C(p, k-h) are combined at the end
//                  in exact multi-word arithmetic (proof of Thm. main);
//        vertex  : Alg. 2 steps ht/pt into the caller's table;
//        edge    : Alg. 2 steps hht/pht/ppt into the caller's table;
//      both local forms add multi-word binomials with carry-propagating
//      64-bit atomics, so results are exact whatever the order.
// Roots come from a device work queue (persistent warps) in descending
// out-degree, one kernel instance per bitset width NW = ceil(d / 32).
#include <algorithm>
#include <string>

#include "pvt_internal.cuh"

namespace pvt {

enum Mode { MODE_GLOBAL = 0, MODE_VERTEX = 1, MODE_EDGE = 2 };

template <int NW>
struct WarpWork {
    static constexpr int D = 32 * NW;                // largest out-degree handled
    static constexpr int RS = NW == 1 ? 1 : NW + 1;  // odd row stride: no bank conflicts
    // wide classes keep their (worst case d+1 frames) DFS stack in per-warp
    // global memory, which leaves room for more resident warps
    static constexpr bool GSTACK = NW >= 8;
    int64_t rs[D];               // start of N+(member) in ocol
    uint32_t ids[D];             // member vertex ids (ascending)
    uint32_t off[D + 1];         // prefix sums of |N+(member)|
    uint32_t adj[D * RS];        // adjacency bitset rows
    uint32_t stk_s[GSTACK ? 1 : (D + 1) * NW];  // DFS stack: S bitsets
    uint32_t *gstk;              // this warp's (D+1)*NW-word stack (GSTACK)
    uint32_t *etab;              // per-edge counts: this warp's D x D edge ids of member pairs
                                 // (written by the gather; null: search the out-lists)
    uint32_t hp[D + 1];          // DFS stack: (h << 16) | p
    // local counts only (point into a shared-memory region of LOCAL_BYTES):
    uint16_t *lk;                // DFS stack: link into the frame
    uint16_t *path;              // link label at each depth of the current path
    uint16_t *memH;              // leaf members: hold vertices (local index, d = root)
    uint16_t *memP;              // leaf members: pivot vertices
    static constexpr size_t LOCAL_BYTES = ((2 * (D + 1) + 3 * 2 * (D + 2)) + 15) / 16 * 16;
    __device__ __forceinline__ void bind_local(unsigned char *base)
    {
        lk = reinterpret_cast<uint16_t *>(base);
        path = lk + (D + 1);
        memH = path + (D + 2);
        memP = memH + (D + 2);
    }
    uint2 cstk[33];              // one-word walk of a compacted subtree: (S, (h << 16) | p)
    uint16_t cmap[32];           // compacted index -> member index
    uint32_t fbuf[36];           // copy of a donated frame taken from the queue
    __device__ __forceinline__ uint32_t *stk() { return GSTACK ? gstk : stk_s; }
};

constexpr uint16_t LINK_PIVOT = 0x8000u;

// --------------------------------------------------- multi-word atomics

// a[0..W) += x (one word), carries propagated with further atomics.
__device__ __forceinline__ void atomic_add_u64_carry(unsigned long long *a, unsigned long long x,
                                                     int W, unsigned *err)
{
    unsigned long long old = atomicAdd(a, x);
    if (old + x >= old) return;
    for (int j = 1; j < W; ++j) {
        old = atomicAdd(a + j, 1ull);
        if (old != ~0ull) return;
    }
    atomicOr(err, DERR_OVERFLOW);
}

// a[0..W) += b[0..W) as one multi-word integer.
__device__ __forceinline__ void atomic_add_multi(unsigned long long *a,
                                                 const unsigned long long *__restrict__ b, int W,
                                                 unsigned *err)
{
    unsigned long long c = 0;
    for (int j = 0; j < W; ++j) {
        unsigned long long bj = b[j];
        if (bj == 0 && c == 0) continue;
        unsigned long long add = bj + c;
        unsigned long long c2 = (add < bj) ? 1ull : 0ull;  // bj = ~0 and c = 1
        unsigned long long old = add ? atomicAdd(a + j, add) : 0ull;
        c = c2 + ((old + add < old) ? 1ull : 0ull);
    }
    if (c) atomicOr(err, DERR_OVERFLOW);
}

__device__ __forceinline__ const unsigned long long *binom_at(const unsigned long long *B, int a,
                                                              int b, int W)
{
    return B + ((size_t)a * (a + 1) / 2 + b) * W;
}

// ------------------------------------------------------- leaf tallies

constexpr unsigned long long SPLIT_IDLE_LIMIT_NS = 120000000000ull;  // 120 s without progress (profilers slow items a lot)
constexpr unsigned long long SPLIT_SLOT_LIMIT_NS = 2000000000ull;  // 2 s for a ring slot to free up

struct CountArgs {
    const int64_t *orow;
    const uint32_t *ocol;
    const uint32_t *oeid;
    const uint32_t *roots;
    unsigned nroots;
    unsigned *qhead;
    unsigned long long *hist;   // global mode: (h, p) histogram, row stride hstride
    int hstride;
    unsigned long long *out;    // local modes: [count][K][W]
    const unsigned long long *B;  // multi-word Pascal table
    int Bw;                       // words per table entry (>= W)
    int W;
    int kmax;
    unsigned *err;
    unsigned long long *stats;  // [0] nodes, [1] leaves, [2] pivot words, [3 + class] words
    int cls;                    // out-degree class of the launch
    unsigned chunk;             // roots per queue access (persistent form)
    // subtree splitting (heavy classes, global counts)
    uint32_t *rootbuf;          // [nroots][32*NW][NW] adjacency rows, published per root
    uint32_t *qframes;          // [qcap][FRAME_WORDS] ring of donated frames (layout below)
    uint32_t *qready;           // [qcap] t+1 once the frame of ticket t is written
    uint32_t *qdone;            // [qcap] t+1 once the frame of ticket t is copied out
    uint32_t *qctl;             // counters, each on its own 128-byte line (Q_* offsets)
    unsigned qcap;              // power of two
    uint32_t *gstack;           // wide classes: per-warp DFS stacks, (32*NW+1)*NW words each
    uint32_t *eidtab;           // per-edge counts: per-warp (32*NW)^2 edge-id tables (or null)
    // two-phase global counts: the wide walk emits every compacted subtree
    // as a frame (layout below) for k_walk_frames; null: walk them in place
    uint32_t *emit;             // [emit_cap][FRAME_WORDS]
    unsigned long long *emit_count;  // compacted subtrees met so far (passes emit_cap once the
                                     // buffer is full; 64-bit: long walks meet billions)
    unsigned emit_cap;
    // bounded waits: an idle warp gives up after idle_ns without progress, a
    // donor after slot_ns for a ring slot (policy.wait_limit_us overrides both)
    unsigned long long idle_ns = SPLIT_IDLE_LIMIT_NS, slot_ns = SPLIT_SLOT_LIMIT_NS;
};

// Work queue of a split launch, a ring of qcap slots.  Idle warps take a
// ticket t (one atomicAdd on the head) and wait on slot t mod qcap until its
// ready word says t+1; busy warps donate a frame whenever tickets are ahead
// of the frames produced (head > tail), after the slot's previous occupant
// (ticket t - qcap) has been copied out.  A warp holding a ticket leaves once
// no item is outstanding: then no warp can produce another frame.
// Head and tail are 64-bit ticket counters (two words each): a long walk
// donates billions of frames.  A ring slot stores the low 32 bits of t+1,
// which tell ticket t from the slot's previous occupant t - qcap.
constexpr int Q_HEAD = 0, Q_TAIL = 32, Q_OUT = 64, Q_ROOT = 96, QCTL_WORDS = 128;
// Frame: [0] kind; wide (1): [1] root index, [2] d, [3] (h<<16)|p, [4..4+NW) S;
// compacted (2): [1] (h<<16)|p, [2] S, [3] out-degree class of the root,
// [4..36) the 32 one-word rows.
constexpr int FRAME_WORDS = 36;
constexpr uint32_t FRAME_WIDE = 1u, FRAME_COMPACT = 2u;

// Block-level (h, p) leaf histogram in shared memory for h < HIST_H, p < HIST_P
// (where almost every leaf falls); other leaves go straight to the global one.
constexpr int HIST_H = 32, HIST_P = 48;

// Walk statistics.  nodes / leaves / words advance in step on every lane of
// the warp; the x* fields count, per lane, the small subtrees that lane
// closed in closed form (close_small), as the nodes, leaves and pivot words
// the walk would have spent on them, until fold() adds their warp sums in.
struct WalkCounters {
    unsigned long long nodes = 0, leaves = 0, words = 0;
    unsigned xnodes = 0, xleaves = 0, xwords = 0;
    // after every walk item (all lanes)
    __device__ __forceinline__ void fold()
    {
        nodes += __reduce_add_sync(0xFFFFFFFFu, xnodes);
        leaves += __reduce_add_sync(0xFFFFFFFFu, xleaves);
        words += __reduce_add_sync(0xFFFFFFFFu, xwords);
        xnodes = xleaves = xwords = 0;
    }
    // add the warp's totals to stats[0..2] and, if cls >= 0, to stats[3 + cls]
    // (all lanes)
    __device__ __forceinline__ void flush(unsigned long long *stats, int cls, int lane)
    {
        fold();
        if (lane == 0 && nodes) {
            atomicAdd(&stats[0], nodes);
            atomicAdd(&stats[1], leaves);
            atomicAdd(&stats[2], words);
            if (cls >= 0) atomicAdd(&stats[3 + cls], words);
        }
    }
};

template <bool SHIST>
__device__ __forceinline__ void tally_leaf(unsigned long long *shist, const CountArgs &A, int lane, int h, int p)
{
    if (lane == 0) {
        if (SHIST && h < HIST_H && p < HIST_P) atomicAdd(&shist[h * HIST_P + p], 1ull);
        else atomicAdd(&A.hist[(size_t)h * A.hstride + p], 1ull);
    }
}

// Leaf tally by the calling lane alone (lanes tally independently).
template <bool SHIST>
__device__ __forceinline__ void tally_lane(unsigned long long *shist, const CountArgs &A, int h, int p)
{
    if (SHIST && h < HIST_H && p < HIST_P) atomicAdd(&shist[h * HIST_P + p], 1ull);
    else atomicAdd(&A.hist[(size_t)h * A.hstride + p], 1ull);
}

// The subtree of a node with label S' of at most two members, reached with
// (h, p), in closed form (global counts): |S'| = 0 is a leaf (h, p); a
// single member or an adjacent pair is a clique, one leaf (h, p + |S'|); a
// non-adjacent pair {a < b} takes a as pivot (a pivot leaf (h, p + 1)) and
// holds b (a leaf (h + 1, p), cut when h + 1 > kmax).  Counts the nodes,
// leaves and pivot words (wpm per member: 1, a label of at most two members
// fits one word) the walk would have spent.
// UNIFORM: every lane calls with the same arguments, lane 0 tallies.
template <bool SHIST, bool UNIFORM>
__device__ __forceinline__ void close_small(unsigned long long *shist, const CountArgs &A, int lane, int cs,
                                            bool adjacent, int h, int p, unsigned wpm, WalkCounters &wc)
{
    if (UNIFORM) {
        wc.nodes += 1 + (cs == 2 && !adjacent) + (cs == 2 && !adjacent && h + 1 <= A.kmax);
        wc.leaves += 1 + (cs == 2 && !adjacent && h + 1 <= A.kmax);
        wc.words += (unsigned long long)cs * wpm;
    } else {
        wc.xnodes += 1u + (cs == 2 && !adjacent) + (cs == 2 && !adjacent && h + 1 <= A.kmax);
        wc.xleaves += 1u + (cs == 2 && !adjacent && h + 1 <= A.kmax);
        wc.xwords += (unsigned)cs * wpm;
    }
    if (UNIFORM && lane != 0) return;
    if (cs <= 1 || adjacent) {
        tally_lane<SHIST>(shist, A, h, p + cs);
        return;
    }
    tally_lane<SHIST>(shist, A, h, p + 1);  // the pivot leaf below the pair
    if (h + 1 <= A.kmax) tally_lane<SHIST>(shist, A, h + 1, p);
}

// Donated frames must carry enough work to pay for the queue round trip.
constexpr int DONATE_MIN_WIDE = 16;     // members of a wide frame's label
constexpr int DONATE_MIN_COMPACT = 14;  // members of a compacted frame's label


__device__ __forceinline__ unsigned vload(const unsigned *p) { return *(const volatile unsigned *)p; }
__device__ __forceinline__ unsigned long long vload64(const uint32_t *p)
{
    return *(const volatile unsigned long long *)p;
}
__device__ __forceinline__ unsigned long long *qword(uint32_t *p)
{
    return reinterpret_cast<unsigned long long *>(p);
}

// Lane 0: are warps waiting on tickets that no frame fills yet?  (Not once
// a wait has given up: the waiting warps have left, and a donation would
// only wait for a slot that no one frees.)
__device__ __forceinline__ bool queue_hungry(const CountArgs &A)
{
    return vload64(A.qctl + Q_HEAD) > vload64(A.qctl + Q_TAIL) && !(vload(A.err) & DERR_TIMEOUT);
}

// How many warps wait on the ring for a frame not yet published (at most
// cap; 0 after a timeout).
__device__ __forceinline__ unsigned queue_waiters(const CountArgs &A, unsigned cap)
{
    const unsigned long long hd = vload64(A.qctl + Q_HEAD), tl = vload64(A.qctl + Q_TAIL);
    if (hd <= tl || (vload(A.err) & DERR_TIMEOUT)) return 0u;
    return (unsigned)min(hd - tl, (unsigned long long)cap);
}

// Reserve the slot of the next frame (one more outstanding item); all lanes
// get its ticket number t.  Returns nullptr (status set) if the slot never
// frees up.
__device__ __forceinline__ uint32_t *frame_reserve(const CountArgs &A, int lane, unsigned &t)
{
    int ok = 1;
    if (lane == 0) {
        atomicAdd(A.qctl + Q_OUT, 1u);
        const unsigned long long t64 = atomicAdd(qword(A.qctl + Q_TAIL), 1ull);
        t = (unsigned)t64;
        if (t64 >= A.qcap) {
            const unsigned want = (unsigned)(t64 - A.qcap + 1u), slot = t & (A.qcap - 1u);
            const unsigned long long t0 = global_ns();
            while (vload(A.qdone + slot) != want) {
                if (global_ns() - t0 > A.slot_ns) { atomicOr(A.err, DERR_TIMEOUT); ok = 0; break; }
                __nanosleep(64);
            }
        }
    }
    t = __shfl_sync(FULL, t, 0);
    ok = __shfl_sync(FULL, ok, 0);
    return ok ? A.qframes + (size_t)(t & (A.qcap - 1u)) * FRAME_WORDS : nullptr;
}

// Publish a written frame.
__device__ __forceinline__ void frame_publish(const CountArgs &A, int lane, unsigned t)
{
    __threadfence();
    __syncwarp();
    if (lane == 0) atomicExch(A.qready + (t & (A.qcap - 1u)), t + 1u);
}


// Edge id of the edge between members a and b (local indices, d = root).
template <int NW>
__device__ __forceinline__ uint32_t member_edge_id(const WarpWork<NW> &Wk, const CountArgs &A,
                                                   int64_t rbeg, int d, int a, int b)
{
    if (a == d) return A.oeid[rbeg + b];
    if (b == d) return A.oeid[rbeg + a];
    if (Wk.etab) return Wk.etab[a * WarpWork<NW>::D + b];
    // the edge sits in exactly one of N+(u_a), N+(u_b): search both
    for (int t = 0; t < 2; ++t) {
        int x = t ? b : a, y = t ? a : b;
        int64_t lo = Wk.rs[x], hi = lo + (Wk.off[x + 1] - Wk.off[x]);
        uint32_t key = Wk.ids[y];
        while (lo < hi) {
            int64_t mid = lo + ((hi - lo) >> 1);
            if (A.ocol[mid] < key) lo = mid + 1; else hi = mid;
        }
        if (lo < Wk.rs[x] + (Wk.off[x + 1] - Wk.off[x]) && A.ocol[lo] == key) return A.oeid[lo];
    }
    atomicOr(A.err, DERR_RANGE);
    return 0xFFFFFFFFu;
}

// Adds C(a, i) at k = s + i (i = 0..a, k <= kmax) to row `cell` ([K][W]).
__device__ __forceinline__ void add_binom_row(unsigned long long *cell, int s, int a,
                                              const CountArgs &A)
{
    for (int i = 0; i <= a; ++i) {
        int k = s + i;
        if (k > A.kmax) break;
        atomic_add_multi(cell + (size_t)k * A.W, binom_at(A.B, a, i, A.Bw), A.W, A.err);
    }
}

// Leaf of a local-count walk: path links at depths 1..t, plus the clique X
// (as extra pivot links) when the leaf closes a clique node.
template <int NW, int MODE>
__device__ void local_leaf(WarpWork<NW> &Wk, const CountArgs &A, int lane, uint32_t r, int64_t rbeg,
                           int d, int h, int p, int t, const uint32_t *X)
{
    constexpr int D = WarpWork<NW>::D;
    // members: H = root + hold links, P = pivot links + X
    int nh = 0, np = 0;
    if (lane == 0) Wk.memH[0] = (uint16_t)d;
    nh = 1;
    for (int base = 1; base <= t; base += 32) {
        int j = base + lane;
        uint16_t l = j <= t ? Wk.path[j] : 0;
        bool valid = j <= t;
        bool piv = valid && (l & LINK_PIVOT);
        bool hold = valid && !(l & LINK_PIVOT);
        unsigned bh = __ballot_sync(FULL, hold), bp = __ballot_sync(FULL, piv);
        unsigned below = (1u << lane) - 1u;
        if (hold) Wk.memH[nh + __popc(bh & below)] = (uint16_t)(l & 0x7FFF);
        if (piv) Wk.memP[np + __popc(bp & below)] = (uint16_t)(l & 0x7FFF);
        nh += __popc(bh);
        np += __popc(bp);
    }
    if (X) {
#pragma unroll
        for (int w = 0; w < NW; ++w) {
            bool in = (X[w] >> lane) & 1u;
            unsigned bx = __ballot_sync(FULL, in);
            if (in) Wk.memP[np + __popc(bx & ((1u << lane) - 1u))] = (uint16_t)(w * 32 + lane);
            np += __popc(bx);
        }
    }
    __syncwarp();
    if (nh != h || np != p || nh + np > D + 1) {
        if (lane == 0) atomicOr(A.err, DERR_RANGE);
        return;
    }
    auto gid = [&](int loc) -> uint32_t { return loc == d ? r : Wk.ids[loc]; };
    if (MODE == MODE_VERTEX) {
        // Alg. 2 step ht: v in H gains C(p, i) at h+i; step pt: v in P gains C(p-1, i) at h+1+i
        for (int q = lane; q < h + p; q += 32) {
            bool inH = q < h;
            uint32_t v = gid(inH ? Wk.memH[q] : Wk.memP[q - h]);
            unsigned long long *cell = A.out + (size_t)v * (A.kmax + 1) * A.W;
            if (inH) add_binom_row(cell, h, p, A);
            else add_binom_row(cell, h + 1, p - 1, A);
        }
    } else {
        // Alg. 2 steps hht / pht / ppt over unordered member pairs, the
        // L(L-1)/2 pairs (a < b) numbered row by row and dealt to the lanes
        const int L = h + p;
        const int npairs = L * (L - 1) / 2;
        for (int t = lane; t < npairs; t += 32) {
            // row a of pair t: the largest a with a(2L - a - 1)/2 <= t
            const float r2 = (float)(2 * L - 1);
            int a = (int)((r2 - sqrtf(r2 * r2 - 8.0f * (float)t)) * 0.5f);
            a = max(0, min(a, L - 2));
            while (a > 0 && a * (2 * L - a - 1) / 2 > t) --a;
            while (a + 1 <= L - 2 && (a + 1) * (2 * L - a - 2) / 2 <= t) ++a;
            const int b = t - a * (2 * L - a - 1) / 2 + a + 1;
            const int la = a < h ? Wk.memH[a] : Wk.memP[a - h];
            const int lb = b < h ? Wk.memH[b] : Wk.memP[b - h];
            const uint32_t e = member_edge_id(Wk, A, rbeg, d, la, lb);
            if (e == 0xFFFFFFFFu) continue;
            unsigned long long *cell = A.out + (size_t)e * (A.kmax + 1) * A.W;
            const int npiv = (a >= h) + (b >= h);
            add_binom_row(cell, h + npiv, p - npiv, A);
        }
    }
    __syncwarp();
}

// ---------------------------------------------------------- one root

// Pending wide frames of the walk that descended into a compacted subtree.
struct Outer {
    int *top, *bot;  // live frames stk[*bot..*top)
    unsigned qi;     // root index within the launch
    int d;           // root out-degree
};

// Donation clock of one warp, shared by the wide and the compacted walks:
// the queue is consulted once every `every` nodes.
struct Clock {
    unsigned nodes = 0, next = 0;
    unsigned every = 16;  // nodes between looks at the queue
};
constexpr unsigned EMIT_CLOCK = 4;  // clock ticks per emitted frame

// Hand wide frame f (of root qi, out-degree d) to the frame queue.
template <int NW>
__device__ __forceinline__ void donate_wide(WarpWork<NW> &Wk, const CountArgs &A, int lane, int f, unsigned qi,
                                            int d)
{
    unsigned t = 0;
    uint32_t *fr = frame_reserve(A, lane, t);
    if (!fr) return;
    if (lane < NW) fr[4 + lane] = Wk.stk()[f * NW + lane];
    if (lane == 0) {
        fr[0] = FRAME_WIDE;
        fr[1] = qi;
        fr[2] = (uint32_t)d;
        fr[3] = Wk.hp[f];
    }
    frame_publish(A, lane, t);
}

// Walk of a subtree in one-word bitsets: lane k holds row k of the adjacency
// induced on the (at most 32) members of the label, S1 and (h, p) describe
// the node.  Same pivot rule, children and leaf tally as the wide walk
// (global counts).  In the split form, pending frames are donated to idle
// warps as self-contained compacted frames (rows travel with the frame).
template <int NW, bool SHIST, bool SPLIT>
__device__ void compact_loop(WarpWork<NW> &Wk, unsigned long long *shist, const CountArgs &A, int lane,
                             uint32_t r1, uint32_t S1, int h, int p, WalkCounters &wc, const Outer *outer,
                             Clock &clk)
{
    auto tally = [&](int hh, int pp) { tally_leaf<SHIST>(shist, A, lane, hh, pp); };
    // this call's nodes, leaves and pivot words (every lane alike; at most a
    // 32-member label's tree, so 32 bits hold them), added to wc on exit
    unsigned cn = 0, cl = 0, cw = 0;
    auto fold = [&]() {
        wc.nodes += cn;
        wc.leaves += cl;
        wc.words += cw;
    };
    int top = 0, bot = 0;
    for (;;) {
        const int s1 = __popc(S1);
        ++cn;
        clk.nodes++;
        bool closed = true;
        if (s1 == 0) {
            ++cl;
            tally(h, p);
        } else {
            const bool in = (S1 >> lane) & 1u;
            const uint32_t c = in ? __popc(r1 & S1) : 0u;
            const uint32_t best = __reduce_max_sync(FULL, in ? (((c + 1u) << 5) | (31u - lane)) : 0u);
            const uint32_t dsum = __reduce_add_sync(FULL, c);
            cw += (unsigned)s1;
            if (dsum == (uint32_t)s1 * (uint32_t)(s1 - 1)) {
                ++cl;
                tally(h, p + s1);
            } else {
                const int piv = 31 - (int)(best & 31u);
                const uint32_t rp = __shfl_sync(FULL, r1, piv);
                const uint32_t R0 = S1 & ~rp & ~(1u << piv);
                // hold children: each lane of R0 forms its child's label; labels
                // of at most two members are closed here, the rest are pushed
                uint32_t R = 0;
                if (R0 && h + 1 <= A.kmax) {
                    const bool inR = (R0 >> lane) & 1u;
                    const uint32_t child = inR ? (r1 & S1 & ~(R0 & ((1u << lane) - 1u))) : 0u;
                    const int cs = __popc(child);
                    const uint32_t ra = __shfl_sync(FULL, r1, (__ffs(child) - 1) & 31);
                    if (inR && cs <= 2)
                        close_small<SHIST, false>(shist, A, lane, cs, (ra >> ((31 - __clz(child)) & 31)) & 1u, h + 1, p,
                                                  1u, wc);
                    R = __ballot_sync(FULL, inR && cs > 2);
                }
                const int nR = __popc(R);
                if (nR > 0) {
                    if (top + nR > 33) {
                        if (SPLIT && bot > 0) {
                            // donated frames left room at the base: move the live ones down
                            __syncwarp();
                            for (int t = lane; t < top - bot; t += 32) Wk.cstk[t] = Wk.cstk[bot + t];
                            top -= bot;
                            bot = 0;
                            __syncwarp();
                        }
                        if (top + nR > 33) {
                            if (lane == 0) atomicOr(A.err, DERR_STACK);
                            fold();
                            return;
                        }
                    }
                    __syncwarp();
                    if ((R >> lane) & 1u) {
                        const uint32_t low = (1u << lane) - 1u;
                        const int f = top + __popc(R & low);
                        Wk.cstk[f] = make_uint2(r1 & S1 & ~(R0 & low), ((uint32_t)(h + 1) << 16) | (uint32_t)p);
                    }
                    top += nR;
                    __syncwarp();
                    if (SPLIT && (int)(clk.nodes - clk.next) >= 0) {
                        clk.next = clk.nodes + clk.every;
                        // waiting warps get the largest pending work first: the
                        // enclosing wide walk's oldest frame, else our oldest
                        int ndon = 0, wide = 0;
                        if (lane == 0 && queue_hungry(A)) {
                            if (outer && *outer->top - *outer->bot >= 1) {
                                int sz = 0;
#pragma unroll
                                for (int w = 0; w < NW; ++w) sz += __popc(Wk.stk()[*outer->bot * NW + w]);
                                wide = sz >= DONATE_MIN_WIDE;
                            }
                            if (!wide && top - bot >= 2 && __popc(Wk.cstk[bot].x) >= DONATE_MIN_COMPACT) ndon = 1;
                        }
                        wide = __shfl_sync(FULL, wide, 0);
                        ndon = __shfl_sync(FULL, ndon, 0);
                        if (wide) {
                            donate_wide<NW>(Wk, A, lane, *outer->bot, outer->qi, outer->d);
                            *outer->bot += 1;
                        } else if (ndon) {
                            unsigned t = 0;
                            uint32_t *fr = frame_reserve(A, lane, t);
                            if (fr) {
                                fr[4 + lane] = r1;
                                if (lane == 0) {
                                    fr[0] = FRAME_COMPACT;
                                    fr[1] = Wk.cstk[bot].y;
                                    fr[2] = Wk.cstk[bot].x;
                                    fr[3] = (uint32_t)A.cls;
                                }
                                frame_publish(A, lane, t);
                                bot += 1;
                            }
                        }
                    }
                }
                // the pivot child N(S, piv): closed at once if it has at most two members
                const uint32_t P1 = rp & S1;
                const int ps = __popc(P1);
                if (ps <= 2) {
                    const uint32_t ra = __shfl_sync(FULL, r1, (__ffs(P1) - 1) & 31);
                    close_small<SHIST, true>(shist, A, lane, ps, (ra >> ((31 - __clz(P1)) & 31)) & 1u, h, p + 1, 1u, wc);
                } else {
                    closed = false;
                    S1 = P1;
                    p += 1;
                }
            }
        }
        if (!closed) continue;
        if (top == bot) break;
        --top;
        const uint2 e = Wk.cstk[top];
        S1 = e.x;
        const uint32_t hp = e.y;
        h = (int)(hp >> 16);
        p = (int)(hp & 0xFFFFu);
    }
    fold();
    __syncwarp();
}

// Compact a node whose label S (in NW-word bitsets over the root's members)
// has s <= 32 members: relabel them 0..s-1 in ascending order; lane k gets
// row k of the induced adjacency -- by symmetry, the ballot over lanes j of
// "member k is in my row" is exactly that row.
template <int NW>
__device__ __forceinline__ uint32_t compact_rows(WarpWork<NW> &Wk, int lane, const uint32_t *S, int s)
{
    constexpr int RS = WarpWork<NW>::RS;
    int before = 0;
#pragma unroll
    for (int w = 0; w < NW; ++w) {
        if ((S[w] >> lane) & 1u) Wk.cmap[before + __popc(S[w] & ((1u << lane) - 1u))] = (uint16_t)(w * 32 + lane);
        before += __popc(S[w]);
    }
    __syncwarp();
    const int mj = lane < s ? Wk.cmap[lane] : 0;
    uint32_t r1 = 0;
    for (int k = 0; k < s; ++k) {
        const int mk = Wk.cmap[k];
        const bool bit = lane < s && ((Wk.adj[mj * RS + (mk >> 5)] >> (mk & 31)) & 1u);
        const uint32_t col = __ballot_sync(FULL, bit);
        if (lane == k) r1 = col;
    }
    __syncwarp();
    return r1;
}

// Walk the compacted subtree in place, or (two-phase global counts) emit it
// as a frame for k_walk_frames while the buffer has room.
template <int NW, bool SHIST, bool SPLIT>
__device__ void walk_compact(WarpWork<NW> &Wk, unsigned long long *shist, const CountArgs &A, int lane,
                             const uint32_t *S, int s, int h, int p, WalkCounters &wc, const Outer *outer,
                             Clock &clk)
{
    const uint32_t r1 = compact_rows<NW>(Wk, lane, S, s);
    const uint32_t S1 = s >= 32 ? FULL : ((1u << s) - 1u);
    if (A.emit) {
        unsigned long long i = 0;
        if (lane == 0) i = atomicAdd(A.emit_count, 1ull);
        i = __shfl_sync(FULL, i, 0);
        if (i < (unsigned long long)A.emit_cap) {
            uint32_t *fr = A.emit + (size_t)i * FRAME_WORDS;
            fr[4 + lane] = r1;
            if (lane == 0) {
                fr[0] = FRAME_COMPACT;
                fr[1] = ((uint32_t)h << 16) | (uint32_t)p;
                fr[2] = S1;
                fr[3] = (uint32_t)A.cls;
            }
            // an emission is where the wide walk spends its time: let it
            // advance the donation clock, so that a heavy root's pending wide
            // frames move to idle warps
            clk.nodes += EMIT_CLOCK;
            return;
        }
    }
    compact_loop<NW, SHIST, SPLIT>(Wk, shist, A, lane, r1, S1, h, p, wc, outer, clk);
}

// One walk item: a whole root r (frame == nullptr), or a frame of root qi's
// subtree that another warp donated (split form).
template <int NW, int MODE, bool SHIST, bool SPLIT>
__device__ void walk_root(WarpWork<NW> &Wk, unsigned long long *shist, const CountArgs &A, int lane,
                          uint32_t r, WalkCounters &wc, unsigned qi = 0, const uint32_t *frame = nullptr)
{
    Clock clk;
    constexpr int D = WarpWork<NW>::D;
    constexpr int RS = WarpWork<NW>::RS;
    constexpr bool REG = NW <= 4;  // keep this lane's adjacency rows in registers
    // the member-word loops of the widest classes stay rolled: unrolled they
    // multiply the code (and its compile time) by NW for a rare class
    constexpr int UNROLL_J = NW <= 8 ? NW : 1;
    int64_t rbeg = 0;
    int d = 0;
    uint32_t S[NW];
    int h = 1, p = 0;
    if (SPLIT && frame) {
        // ---- donated frame: adjacency rows come from the root's published copy
        d = (int)frame[1];
        const uint32_t hp0 = frame[2];
        h = (int)(hp0 >> 16);
        p = (int)(hp0 & 0xFFFFu);
#pragma unroll
        for (int w = 0; w < NW; ++w) S[w] = frame[3 + w];
        const uint32_t *src = A.rootbuf + (size_t)qi * D * NW;
        for (int t = lane; t < d * NW; t += 32) Wk.adj[(t / NW) * RS + (t % NW)] = __ldcg(src + t);
        __syncwarp();
    } else {
    rbeg = A.orow[r];
    d = (int)(A.orow[r + 1] - rbeg);
    if (d > D) {
        if (lane == 0) atomicOr(A.err, DERR_RANGE);
        return;
    }

    // ---- 1. gather: member ids, their out-list extents, bitset adjacency
    uint32_t base = 0;
#pragma unroll
    for (int c = 0; c < NW; ++c) {
        int i = c * 32 + lane;
        uint32_t id = 0xFFFFFFFFu, od = 0;
        int64_t rs = 0;
        if (i < d) {
            id = A.ocol[rbeg + i];
            rs = A.orow[id];
            od = (uint32_t)(A.orow[id + 1] - rs);
        }
        uint32_t inc = od;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t t = __shfl_up_sync(FULL, inc, o);
            if (lane >= o) inc += t;
        }
        Wk.ids[i] = id;
        Wk.rs[i] = rs;
        Wk.off[i + 1] = base + inc;
        base += __shfl_sync(FULL, inc, 31);
    }
    if (lane == 0) Wk.off[0] = 0;
    for (int t = lane; t < d * RS; t += 32) Wk.adj[t] = 0;
    __syncwarp();
    // entry t of the concatenated out-lists belongs to member lo, the largest
    // i with off[i] <= t; a lane's entries rise, so lo only moves forward.
    // Four entries per lane per round keep four loads of ocol in flight.
    const uint32_t T = base;
    int lo = 0;
    for (uint32_t t0 = lane; t0 < T; t0 += 128) {
        uint32_t x[4];
        int mi[4];
        int64_t at[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const uint32_t t = t0 + 32u * q;
            mi[q] = -1;
            if (t < T) {
                while (Wk.off[lo + 1] <= t) ++lo;  // stops by off[d] = T > t
                mi[q] = lo;
                at[q] = Wk.rs[lo] + (t - Wk.off[lo]);
                x[q] = A.ocol[at[q]];
            }
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            if (mi[q] < 0) continue;
            int a = 0, b = d;
            while (a < b) {
                int mid = (a + b) >> 1;
                if (Wk.ids[mid] < x[q]) a = mid + 1; else b = mid;
            }
            if (a < d && Wk.ids[a] == x[q]) {
                const int u = mi[q];
                atomicOr(&Wk.adj[u * RS + (a >> 5)], 1u << (a & 31));
                atomicOr(&Wk.adj[a * RS + (u >> 5)], 1u << (u & 31));
                if (MODE == MODE_EDGE && Wk.etab) {
                    const uint32_t e = A.oeid[at[q]];
                    Wk.etab[u * D + a] = e;
                    Wk.etab[a * D + u] = e;
                }
            }
        }
    }
    __syncwarp();
    if (SPLIT) {
        // publish the adjacency rows so that donated frames can be walked anywhere
        uint32_t *dst = A.rootbuf + (size_t)qi * D * NW;
        for (int t = lane; t < d * NW; t += 32) dst[t] = Wk.adj[(t / NW) * RS + (t % NW)];
        __threadfence();
        __syncwarp();
    }
#pragma unroll
    for (int w = 0; w < NW; ++w) {
        int bits = d - 32 * w;
        S[w] = bits >= 32 ? FULL : (bits <= 0 ? 0u : ((1u << bits) - 1u));
    }
    }

    uint32_t myrow[REG ? NW : 1][REG ? NW : 1];
    if (REG) {
#pragma unroll
        for (int j = 0; j < NW; ++j)
#pragma unroll
            for (int w = 0; w < NW; ++w) {
                int i = j * 32 + lane;
                myrow[j % (REG ? NW : 1)][w % (REG ? NW : 1)] = i < d ? Wk.adj[i * RS + w] : 0u;
            }
    }
    auto row = [&](int j, int w) -> uint32_t {
        if (REG) return myrow[j % (REG ? NW : 1)][w % (REG ? NW : 1)];
        return Wk.adj[(j * 32 + lane) * RS + w];
    };

    // ---- 2. depth-first walk.  The current node lives in registers; hold
    // children go to the stack and the walk continues straight into the
    // pivot child, so a pivot chain costs no stack traffic.
    int top = 0, bot = 0;  // live frames: stk[bot..top); donations leave from the bottom
    uint16_t link = 0;
    if (MODE != MODE_GLOBAL && lane == 0) Wk.path[0] = (uint16_t)d;
    for (;;) {
        const int depth = h + p - 1;
        if (MODE != MODE_GLOBAL && depth > 0) {
            if (lane == 0) Wk.path[depth] = link;
            __syncwarp();
        }
        int s = 0;
#pragma unroll
        for (int w = 0; w < NW; ++w) s += __popc(S[w]);
        bool closed = true;
        if (NW > 1 && MODE == MODE_GLOBAL && s >= 4 && s <= 32) {
            // small label under a wide root: finish this subtree in one-word bitsets
            const Outer outer{&top, &bot, qi, d};
            walk_compact<NW, SHIST, SPLIT>(Wk, shist, A, lane, S, s, h, p, wc, &outer, clk);
        } else if ((wc.nodes++, clk.nodes++, s == 0)) {
            wc.leaves++;
            if (MODE == MODE_GLOBAL) {
                tally_leaf<SHIST>(shist, A, lane, h, p);
            } else {
                local_leaf<NW, MODE>(Wk, A, lane, r, rbeg, d, h, p, depth, nullptr);
            }
        } else {
            // pivot: most neighbours inside S, ties -> lowest member index; the
            // degree sum tells whether S is a clique (every member has s-1)
            uint32_t best = 0, dsum = 0;
#pragma unroll UNROLL_J
            for (int j = 0; j < NW; ++j) {
                if ((S[j] >> lane) & 1u) {
                    uint32_t c = 0;
#pragma unroll
                    for (int w = 0; w < NW; ++w) c += __popc(row(j, w) & S[w]);
                    uint32_t key = ((c + 1u) << 10) | (1023u - (uint32_t)(j * 32 + lane));
                    best = max(best, key);
                    dsum += c;
                }
            }
            best = __reduce_max_sync(FULL, best);
            dsum = __reduce_add_sync(FULL, dsum);
            wc.words += (unsigned long long)s * (unsigned)((s + 31) >> 5);
            const int piv = 1023 - (int)(best & 1023u);
            if (dsum == (uint32_t)s * (uint32_t)(s - 1)) {
                // S is a clique: one leaf with |S| more pivot links
                wc.leaves++;
                if (MODE == MODE_GLOBAL) {
                    tally_leaf<SHIST>(shist, A, lane, h, p + s);
                } else {
                    local_leaf<NW, MODE>(Wk, A, lane, r, rbeg, d, h, p + s, depth, S);
                }
            } else {
                uint32_t R[NW], P[NW];
                int nR = 0;
#pragma unroll
                for (int w = 0; w < NW; ++w) {
                    const uint32_t a = Wk.adj[piv * RS + w];
                    P[w] = a & S[w];
                    R[w] = S[w] & ~a;
                    if (w == (piv >> 5)) R[w] &= ~(1u << (piv & 31));
                    nR += __popc(R[w]);
                }
                if (nR > 0 && h + 1 <= A.kmax) {
                    if (SPLIT && bot > 0 && top + nR > D + 1) {
                        // compact the live frames down to the stack base
                        __syncwarp();
                        for (int t = lane; t < (top - bot) * NW; t += 32) Wk.stk()[t] = Wk.stk()[bot * NW + t];
                        for (int t = lane; t < top - bot; t += 32) Wk.hp[t] = Wk.hp[bot + t];
                        top -= bot;
                        bot = 0;
                        __syncwarp();
                    }
                    if (top + nR > D + 1) {
                        if (lane == 0) atomicOr(A.err, DERR_STACK);
                        return;
                    }
                    __syncwarp();  // every lane is done reading the last popped frame
                    // hold child of member j*32+lane: N(S, v) minus the earlier
                    // members of R; global counts close labels of at most two
                    // members here and push the rest
                    int before = 0;
                    const uint32_t low = (1u << lane) - 1u;
#pragma unroll UNROLL_J
                    for (int j = 0; j < NW; ++j) {
                        const bool inR = (R[j] >> lane) & 1u;
                        bool push = inR;
                        if (MODE == MODE_GLOBAL && inR) {
                            int cs = 0, a = 0, b = 0;
#pragma unroll
                            for (int w = 0; w < NW; ++w) {
                                const uint32_t below = w < j ? R[w] : (w == j ? (R[j] & low) : 0u);
                                const uint32_t cw = row(j, w) & S[w] & ~below;
                                if (cw) {
                                    if (cs == 0) a = w * 32 + __ffs(cw) - 1;
                                    b = w * 32 + 31 - __clz(cw);
                                }
                                cs += __popc(cw);
                            }
                            if (cs <= 2) {
                                const bool adj = cs == 2 && ((Wk.adj[a * RS + (b >> 5)] >> (b & 31)) & 1u);
                                close_small<SHIST, false>(shist, A, lane, cs, adj, h + 1, p, 1u, wc);
                                push = false;
                            }
                        }
                        const uint32_t pushed = __ballot_sync(FULL, push);
                        if (push) {
                            const int f = top + before + __popc(pushed & low);
#pragma unroll
                            for (int w = 0; w < NW; ++w) {
                                const uint32_t below = w < j ? R[w] : (w == j ? (R[j] & low) : 0u);
                                Wk.stk()[f * NW + w] = row(j, w) & S[w] & ~below;
                            }
                            Wk.hp[f] = ((uint32_t)(h + 1) << 16) | (uint32_t)p;
                            if (MODE != MODE_GLOBAL) Wk.lk[f] = (uint16_t)(j * 32 + lane);
                        }
                        before += __popc(pushed);
                    }
                    top += before;
                    __syncwarp();  // pushed frames visible to every lane
                    if (SPLIT && (int)(clk.nodes - clk.next) >= 0) {
                        clk.next = clk.nodes + clk.every;
                        // donate the oldest pending frame (largest subtree) to an idle warp
                        int ndon = 0;
                        if (lane == 0 && top - bot >= 2) {
                            int sz = 0;
#pragma unroll
                            for (int w = 0; w < NW; ++w) sz += __popc(Wk.stk()[bot * NW + w]);
                            if (sz >= DONATE_MIN_WIDE && queue_hungry(A)) ndon = 1;
                        }
                        ndon = __shfl_sync(FULL, ndon, 0);
                        for (int k = 0; k < ndon; ++k) donate_wide<NW>(Wk, A, lane, bot + k, qi, d);
                        bot += ndon;
                    }
                }
                // continue into the pivot child N(S, piv), or close it at once
                // (global counts) if it has at most two members
                int ps = 0, a = 0, b = 0;
                if (MODE == MODE_GLOBAL) {
#pragma unroll
                    for (int w = 0; w < NW; ++w) {
                        if (P[w]) {
                            if (ps == 0) a = w * 32 + __ffs(P[w]) - 1;
                            b = w * 32 + 31 - __clz(P[w]);
                        }
                        ps += __popc(P[w]);
                    }
                }
                if (MODE == MODE_GLOBAL && ps <= 2) {
                    const bool adj = ps == 2 && ((Wk.adj[a * RS + (b >> 5)] >> (b & 31)) & 1u);
                    close_small<SHIST, true>(shist, A, lane, ps, adj, h, p + 1, 1u, wc);
                } else {
                    closed = false;
#pragma unroll
                    for (int w = 0; w < NW; ++w) S[w] = P[w];
                    p += 1;
                    link = (uint16_t)(LINK_PIVOT | piv);
                }
            }
        }
        if (!closed) continue;
        if (top == bot) break;
        --top;
#pragma unroll
        for (int w = 0; w < NW; ++w) S[w] = Wk.stk()[top * NW + w];
        const uint32_t hp = Wk.hp[top];
        h = (int)(hp >> 16);
        p = (int)(hp & 0xFFFFu);
        if (MODE != MODE_GLOBAL) link = Wk.lk[top];
    }
    __syncwarp();
}

template <int NW>
constexpr int warps_per_block()
{
    return NW <= 2 ? 8 : (NW <= 8 ? 4 : (NW <= 16 ? 2 : 1));
}

template <int NW, int MODE, bool SHIST>
constexpr size_t smem_bytes()
{
    return sizeof(WarpWork<NW>) * warps_per_block<NW>() +
           (SHIST ? sizeof(unsigned long long) * HIST_H * HIST_P : 0) +
           (MODE != MODE_GLOBAL ? WarpWork<NW>::LOCAL_BYTES * warps_per_block<NW>() : 0);
}

// Per-warp set-up shared by the walk kernels: local-count arrays in the
// shared-memory region after the histogram, global DFS stack of wide classes.
template <int NW, int MODE>
__device__ __forceinline__ void bind_warp(WarpWork<NW> &Wk, unsigned char *local_base, int wid, uint32_t *gstack,
                                          unsigned warp_global, uint32_t *eidtab = nullptr)
{
    if (MODE != MODE_GLOBAL) Wk.bind_local(local_base + (size_t)wid * WarpWork<NW>::LOCAL_BYTES);
    if (WarpWork<NW>::GSTACK) Wk.gstk = gstack + (size_t)warp_global * (32 * NW + 1) * NW;
    Wk.etab = MODE == MODE_EDGE && eidtab ? eidtab + (size_t)warp_global * WarpWork<NW>::D * WarpWork<NW>::D : nullptr;
}

// Lane 0 of a split launch: the next item -- 2 with v = a fresh item index
// below nitems, 1 with v = the ticket of a donated frame, 3 when no work is
// left (or an error or a timeout ended the launch).
__device__ __forceinline__ int queue_take(const CountArgs &A, unsigned nitems, unsigned &v)
{
    if (vload(A.qctl + Q_ROOT) < nitems) {
        const unsigned rr = atomicAdd(A.qctl + Q_ROOT, 1u);
        if (rr < nitems) { v = rr; return 2; }
    }
    // a ticket for the next donated frame; wait on its own slot
    int kind = 0;
    const unsigned t = (unsigned)atomicAdd(qword(A.qctl + Q_HEAD), 1ull);
    unsigned last_out = 0xFFFFFFFFu, nap = 64;
    unsigned long long t0 = global_ns();
    const unsigned slot = t & (A.qcap - 1u);
    for (;;) {
        if (vload(A.qready + slot) == t + 1u) { kind = 1; v = t; break; }
        const unsigned out = vload(A.qctl + Q_OUT);
        if (out == 0 || (vload(A.err) & (DERR_STACK | DERR_RANGE | DERR_TIMEOUT))) { kind = 3; break; }
        if (out != last_out) { last_out = out; t0 = global_ns(); }
        else if (global_ns() - t0 > A.idle_ns) { atomicOr(A.err, DERR_TIMEOUT); kind = 3; break; }
        __nanosleep(nap);
        nap = min(nap * 2u, 2048u);
    }
    if (kind == 1) __threadfence();
    return kind;
}

// Copy donated frame t out of the ring into fb and release its slot.
__device__ __forceinline__ void frame_take(const CountArgs &A, int lane, unsigned t, uint32_t *fb)
{
    const uint32_t *fr = A.qframes + (size_t)(t & (A.qcap - 1u)) * FRAME_WORDS;
    fb[lane] = __ldcg(fr + lane);
    if (lane < FRAME_WORDS - 32) fb[32 + lane] = __ldcg(fr + 32 + lane);
    __syncwarp();
    if (lane == 0) {
        __threadfence();
        atomicExch(A.qdone + (t & (A.qcap - 1u)), t + 1u);
    }
}

template <int NW, int MODE, bool SHIST, bool PERSIST, bool SPLIT>
__global__ void __launch_bounds__(32 * warps_per_block<NW>())
    k_count(CountArgs A)
{
    constexpr int WPB = warps_per_block<NW>();
    extern __shared__ __align__(16) unsigned char smem[];
    WarpWork<NW> *ww = reinterpret_cast<WarpWork<NW> *>(smem);
    unsigned long long *shist = reinterpret_cast<unsigned long long *>(ww + WPB);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    bind_warp<NW, MODE>(ww[wid],
                        reinterpret_cast<unsigned char *>(shist) + (SHIST ? sizeof(unsigned long long) * HIST_H * HIST_P : 0),
                        wid, A.gstack, blockIdx.x * WPB + wid, A.eidtab);
    WalkCounters wc;
    if (SHIST) {
        for (int i = threadIdx.x; i < HIST_H * HIST_P; i += blockDim.x) shist[i] = 0;
        __syncthreads();
    }
    // roots of the light class are taken from the queue a few at a time
    const unsigned CHUNK = NW == 1 ? A.chunk : 1u;
    unsigned qi = 0, qend = 0;
    if (SPLIT) {
        // heavy roots and donated subtree frames from one device work queue
        for (;;) {
            unsigned v = 0;
            int kind = lane == 0 ? queue_take(A, A.nroots, v) : 0;
            kind = __shfl_sync(FULL, kind, 0);
            v = __shfl_sync(FULL, v, 0);
            if (kind == 3) break;
            if (kind == 1) {
                // copy the frame out and release its ring slot at once
                uint32_t *fb = ww[wid].fbuf;
                frame_take(A, lane, v, fb);
                if (fb[0] == FRAME_COMPACT) {
                    const uint32_t hp0 = fb[1];
                    Clock clk;
                    compact_loop<NW, SHIST, true>(ww[wid], shist, A, lane, fb[4 + lane], fb[2], (int)(hp0 >> 16),
                                                  (int)(hp0 & 0xFFFFu), wc, nullptr, clk);
                } else {
                    walk_root<NW, MODE, SHIST, true>(ww[wid], shist, A, lane, 0u, wc, fb[1], fb + 1);
                }
            } else {
                walk_root<NW, MODE, SHIST, true>(ww[wid], shist, A, lane, A.roots[v], wc, v, nullptr);
            }
            wc.fold();
            __syncwarp();
            if (lane == 0) atomicSub(A.qctl + Q_OUT, 1u);
        }
    } else
    for (;;) {
        if (PERSIST) {
            if (qi == qend) {
                if (lane == 0) qi = atomicAdd(A.qhead, CHUNK);
                qi = __shfl_sync(FULL, qi, 0);
                qend = min(qi + CHUNK, A.nroots);
            }
        } else {
            qi = blockIdx.x * WPB + wid;
        }
        if (qi >= A.nroots) break;
        walk_root<NW, MODE, SHIST, false>(ww[wid], shist, A, lane, A.roots[qi], wc);
        wc.fold();
        ++qi;
        if (!PERSIST) break;
        if (*(volatile unsigned *)A.err & (DERR_STACK | DERR_RANGE)) break;
    }
    wc.flush(A.stats, A.cls, lane);
    if (SHIST) {
        __syncthreads();
        for (int i = threadIdx.x; i < HIST_H * HIST_P; i += blockDim.x) {
            unsigned long long v = shist[i];
            if (v) atomicAdd(&A.hist[(size_t)(i / HIST_P) * A.hstride + (i % HIST_P)], v);
        }
    }
}

template <typename T>
inline pvt_status grow(DevBuf<T> &b, size_t n, cudaStream_t s)
{
    if (b.n >= n) return PVT_OK;
    if (b.p) PVT_CK(cudaFreeAsync(b.p, s));
    b.p = nullptr;
    b.n = 0;
    PVT_CK(cudaMallocAsync(&b.p, n * sizeof(T), s));
    b.n = n;
    return PVT_OK;
}

// Queue counters of a split launch: head, tail, outstanding items (= roots),
// next root, idle warps.
static __global__ void k_split_init(uint32_t *qctl, unsigned nroots)
{
    for (int i = threadIdx.x; i < QCTL_WORDS; i += blockDim.x) qctl[i] = i == Q_OUT ? nroots : 0u;
}

constexpr unsigned SPLIT_QCAP = 1u << 17;

// The lane walk of one-word labels (lanes.cuh, walk_lanes.cu): the frames of
// the two-phase count.
pvt_status launch_lanes_frames(pvt_dag *g, const CountArgs &base, cudaStream_t s);
// The CTA-per-root walk (cta.cuh, walk_cta.cu) of out-degree class cls >= 4.
pvt_status launch_cta_class(pvt_dag *g, const CountArgs &base, int cls, cudaStream_t s);

template <int NW, int MODE, bool SHIST>
pvt_status launch_class(pvt_dag *g, const CountArgs &base, int cls, cudaStream_t s)
{
    const unsigned cnt = (unsigned)g->wcnt[cls];
    if (cnt == 0) return PVT_OK;
    CountArgs A = base;
    A.roots = g->wroots + g->wstart[cls];
    A.nroots = cnt;
    A.qhead = g->d_q + cls;
    A.cls = cls;
    A.chunk = (unsigned)g->policy.chunk;
    constexpr size_t smem = smem_bytes<NW, MODE, SHIST>();
    constexpr int WPB = warps_per_block<NW>();
    // the widest class always runs persistent warps (its stacks are per resident warp)
    const bool persist = g->policy.persistent != 0 || WarpWork<NW>::GSTACK;
    // heavy classes of the global count may split subtrees across warps
    const bool split = persist && NW >= 2 && MODE == MODE_GLOBAL && g->policy.split[cls] != 0;
    // only the variants that can run are instantiated: local counts never
    // split, and the classes with global DFS stacks always run persistent
    void (*kern)(CountArgs) = nullptr;
    if constexpr (MODE == MODE_GLOBAL && NW >= 2) {
        if (split) kern = k_count<NW, MODE, SHIST, true, true>;
    }
    if (!kern) {
        if constexpr (WarpWork<NW>::GSTACK) kern = k_count<NW, MODE, SHIST, true, false>;
        else kern = persist ? k_count<NW, MODE, SHIST, true, false> : k_count<NW, MODE, SHIST, false, false>;
    }
    if (split) {
        pvt_status st;
        if ((st = grow(g->rootbuf[cls], (size_t)cnt * 32 * NW * NW, s)) != PVT_OK) return st;
        if ((st = grow(g->qframes[cls], (size_t)SPLIT_QCAP * FRAME_WORDS, s)) != PVT_OK) return st;
        if ((st = grow(g->qready[cls], (size_t)SPLIT_QCAP * 2, s)) != PVT_OK) return st;
        PVT_CK(cudaMemsetAsync(g->qready[cls].p, 0, (size_t)SPLIT_QCAP * 2 * sizeof(uint32_t), s));
        k_split_init<<<1, 128, 0, s>>>(g->qctl + QCTL_WORDS * cls, cnt);
        PVT_CK(cudaGetLastError());
        g->stats.launches++;
        A.rootbuf = g->rootbuf[cls].p;
        A.qframes = g->qframes[cls].p;
        A.qready = g->qready[cls].p;
        A.qdone = g->qready[cls].p + SPLIT_QCAP;
        A.qctl = g->qctl + QCTL_WORDS * cls;
        A.qcap = SPLIT_QCAP;
    }
    PVT_CK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const unsigned need = (cnt + WPB - 1) / WPB;
    unsigned grid = need;
    if (WarpWork<NW>::GSTACK) {
        // per-warp global stacks: size the grid to the resident warps (these
        // classes always walk their roots from the persistent loop)
        int per_sm = 0;
        PVT_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 32 * WPB, smem));
        grid = std::max(1u, std::min<unsigned>((unsigned)(g->num_sms * std::max(per_sm, 1)), need));
        pvt_status st = grow(g->gstack[cls], (size_t)grid * WPB * (32 * NW + 1) * NW, s);
        if (st != PVT_OK) return st;
        A.gstack = g->gstack[cls].p;
    }
    if (persist) {
        int per_sm = 0;
        PVT_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 32 * WPB, smem));
        if (per_sm < 1) {
            set_error("count kernel cannot be resident (shared memory)");
            return PVT_ECUDA;
        }
        grid = std::min<unsigned>((unsigned)(g->num_sms * per_sm), need);
    }
    if (MODE == MODE_EDGE && persist && NW <= 8) {
        // per-warp edge-id tables of member pairs (the gather fills them)
        constexpr size_t D = WarpWork<NW>::D;
        pvt_status st = grow(g->etab[cls], (size_t)grid * WPB * D * D, s);
        if (st != PVT_OK) return st;
        A.eidtab = g->etab[cls].p;
    }
    phase_begin(g, 1 + cls, s);
    kern<<<grid, 32 * WPB, smem, s>>>(A);
    PVT_CK(cudaGetLastError());
    phase_end(g, 1 + cls, s);
    g->stats.launches++;
    return PVT_OK;
}

// ------------------------------------------------- compacted-frame walk
//
// Second phase of a two-phase global count: every compacted subtree that
// the wide walks of the classes above 32 emitted, walked in one-word bitsets
// (compact_loop).  The per-warp state is small (compact stack, frame copy),
// so far more warps stay resident than in the wide kernels, whose shared
// adjacency rows limit them; idle warps take donated compacted frames from a
// ring queue exactly as in the split form.  Words go to stats slot
// 3 + FRAMES_SLOT, the emitted frame count to stats[3 + FRAMES_SLOT + 1].
constexpr int FRAME_WPB = 8;
constexpr int FRAMES_SLOT = NCLASS;
constexpr unsigned FRAMES_CHUNK = 4;

template <bool SHIST>
__global__ void __launch_bounds__(32 * FRAME_WPB) k_walk_frames(CountArgs A)
{
    extern __shared__ __align__(16) unsigned char smem[];
    WarpWork<1> *ww = reinterpret_cast<WarpWork<1> *>(smem);
    unsigned long long *shist = reinterpret_cast<unsigned long long *>(ww + FRAME_WPB);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const unsigned long long emitted = *(volatile unsigned long long *)A.emit_count;
    const unsigned nframes = (unsigned)min(emitted, (unsigned long long)A.emit_cap);
    if (blockIdx.x == 0 && threadIdx.x == 0) A.stats[3 + FRAMES_SLOT + 1] = emitted;
    WalkCounters wc;
    if (SHIST) {
        for (int i = threadIdx.x; i < HIST_H * HIST_P; i += blockDim.x) shist[i] = 0;
        __syncthreads();
    }
    unsigned cur = 0, end = 0;  // lane 0: claimed emitted frames [cur, end)
    for (;;) {
        unsigned v = 0;
        int kind = 0;
        if (lane == 0) {
            if (cur < end) {
                kind = 2;
                v = cur++;
            } else if (vload(A.qctl + Q_ROOT) < nframes) {
                // FRAMES_CHUNK emitted frames per claim, prefetched into L2
                // (the buffer outgrows L2 once the wide walks are done)
                const unsigned rr = atomicAdd(A.qctl + Q_ROOT, FRAMES_CHUNK);
                if (rr < nframes) {
                    kind = 2;
                    v = rr;
                    cur = rr + 1;
                    end = min(rr + FRAMES_CHUNK, nframes);
                    const char *a = reinterpret_cast<const char *>(A.emit + (size_t)rr * FRAME_WORDS);
                    const char *b = reinterpret_cast<const char *>(A.emit + (size_t)end * FRAME_WORDS);
                    for (; a < b; a += 128) asm volatile("prefetch.global.L2 [%0];" ::"l"(a));
                }
            }
            if (kind == 0) kind = queue_take(A, 0u, v);
        }
        kind = __shfl_sync(FULL, kind, 0);
        v = __shfl_sync(FULL, v, 0);
        if (kind == 3) break;
        const uint32_t *fr;
        if (kind == 1) {
            frame_take(A, lane, v, ww[wid].fbuf);
            fr = ww[wid].fbuf;
        } else {
            fr = A.emit + (size_t)v * FRAME_WORDS;
        }
        const uint32_t r1 = fr[4 + lane], S1 = fr[2], hp0 = fr[1];
        Clock clk;
        clk.every = 32;
        compact_loop<1, SHIST, true>(ww[wid], shist, A, lane, r1, S1, (int)(hp0 >> 16), (int)(hp0 & 0xFFFFu), wc,
                                     nullptr, clk);
        wc.fold();
        __syncwarp();
        if (lane == 0) atomicSub(A.qctl + Q_OUT, 1u);
    }
    wc.flush(A.stats, FRAMES_SLOT, lane);
    if (SHIST) {
        __syncthreads();
        for (int i = threadIdx.x; i < HIST_H * HIST_P; i += blockDim.x) {
            unsigned long long x = shist[i];
            if (x) atomicAdd(&A.hist[(size_t)(i / HIST_P) * A.hstride + (i % HIST_P)], x);
        }
    }
}

// Queue counters of the frame walk: outstanding items = the emitted frames
// (read on the device: the count is final once the wide walks are done).
static __global__ void k_frames_init(uint32_t *qctl, const unsigned long long *emit_count, unsigned cap)
{
    for (int i = threadIdx.x; i < QCTL_WORDS; i += blockDim.x)
        qctl[i] = i == Q_OUT ? (unsigned)min(*emit_count, (unsigned long long)cap) : 0u;
}

// ----------------------------------------------------------- batched form
//
// Roots of many graphs (a served batch) in one persistent launch per
// (query kind, out-degree class): entry = (graph << 32) | root; each warp
// reads the graph's descriptor and walks the root exactly as the
// single-graph kernels do.  Leaf tallies go to the graph's own histogram or
// table with global atomics.

template <int NW, int MODE>
__global__ void __launch_bounds__(32 * warps_per_block<NW>())
    k_count_batch(const BatchGraph *gs, const uint64_t *entries, unsigned nentries, unsigned *qhead,
                  const unsigned long long *B, int Bw, unsigned *err, unsigned long long *stats, uint32_t *gstack)
{
    constexpr int WPB = warps_per_block<NW>();
    extern __shared__ __align__(16) unsigned char smem[];
    WarpWork<NW> *ww = reinterpret_cast<WarpWork<NW> *>(smem);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    bind_warp<NW, MODE>(ww[wid], reinterpret_cast<unsigned char *>(ww + WPB), wid, gstack, blockIdx.x * WPB + wid);
    WalkCounters wc;
    for (;;) {
        unsigned qi = 0;
        if (lane == 0) qi = atomicAdd(qhead, 1u);
        qi = __shfl_sync(FULL, qi, 0);
        if (qi >= nentries) break;
        const uint64_t e = entries[qi];
        const BatchGraph &G = gs[e >> 32];
        CountArgs A{};
        A.orow = G.orow;
        A.ocol = G.ocol;
        A.oeid = G.oeid;
        A.hist = G.hist;
        A.hstride = G.hstride;
        A.out = G.out;
        A.B = B;
        A.Bw = Bw;
        A.W = G.W;
        A.kmax = G.kmax;
        A.err = err;
        A.stats = stats;
        walk_root<NW, MODE, false, false>(ww[wid], nullptr, A, lane, (uint32_t)e, wc);
        wc.fold();
        if (vload(err) & (DERR_STACK | DERR_RANGE)) break;
    }
    (void)WPB;
    wc.flush(stats, -1, lane);
}

template <int NW, int MODE>
pvt_status launch_batch_class(const BatchGraph *gs, const uint64_t *entries, unsigned cnt, unsigned *qhead,
                                     const unsigned long long *B, int Bw, unsigned *err,
                                     unsigned long long *stats, int num_sms, cudaStream_t s)
{
    constexpr size_t smem = smem_bytes<NW, MODE, false>();
    auto kern = k_count_batch<NW, MODE>;
    PVT_CK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    PVT_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 32 * warps_per_block<NW>(), smem));
    if (per_sm < 1) {
        set_error("batched walk kernel cannot be resident");
        return PVT_ECUDA;
    }
    const unsigned need = (cnt + warps_per_block<NW>() - 1) / warps_per_block<NW>();
    const unsigned grid = std::max(1u, std::min<unsigned>((unsigned)(num_sms * per_sm), need));
    uint32_t *gstack = nullptr;
    if (WarpWork<NW>::GSTACK)
        PVT_CK(cudaMallocAsync(&gstack, (size_t)grid * warps_per_block<NW>() * (32 * NW + 1) * NW * sizeof(uint32_t), s));
    kern<<<grid, 32 * warps_per_block<NW>(), smem, s>>>(gs, entries, cnt, qhead, B, Bw, err, stats, gstack);
    PVT_CK(cudaGetLastError());
    if (gstack) PVT_CK(cudaFreeAsync(gstack, s));
    return PVT_OK;
}

}  // namespace pvt
