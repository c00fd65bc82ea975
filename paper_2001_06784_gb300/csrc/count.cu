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
#include <mutex>
#include <string>

#include "pvt_internal.cuh"

namespace pvt {

enum Mode { MODE_GLOBAL = 0, MODE_VERTEX = 1, MODE_EDGE = 2 };

template <int NW>
struct WarpWork {
    static constexpr int D = 32 * NW;                // largest out-degree handled
    static constexpr int RS = NW == 1 ? 1 : NW + 1;  // odd row stride: no bank conflicts
    int64_t rs[D];               // start of N+(member) in ocol
    uint32_t ids[D];             // member vertex ids (ascending)
    uint32_t off[D + 1];         // prefix sums of |N+(member)|
    uint32_t adj[D * RS];        // adjacency bitset rows
    uint32_t stk[(D + 1) * NW];  // DFS stack: S bitsets
    uint32_t hp[D + 1];          // DFS stack: (h << 16) | p
    uint16_t lk[D + 1];          // DFS stack: link into the frame (local modes)
    uint16_t path[D + 2];        // link label at each depth of the current path
    uint16_t memH[D + 2];        // leaf members: hold vertices (local index, d = root)
    uint16_t memP[D + 2];        // leaf members: pivot vertices
    uint32_t stk1[33];           // one-word walk of a compacted subtree: S
    uint32_t hp1[33];            //   and (h << 16) | p
    uint16_t cmap[32];           // compacted index -> member index
    uint32_t fbuf[36];           // copy of a donated frame taken from the queue
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
};

// Work queue of a split launch, a ring of qcap slots.  Idle warps take a
// ticket t (one atomicAdd on the head) and wait on slot t mod qcap until its
// ready word says t+1; busy warps donate a frame whenever tickets are ahead
// of the frames produced (head > tail), after the slot's previous occupant
// (ticket t - qcap) has been copied out.  A warp holding a ticket leaves once
// no item is outstanding: then no warp can produce another frame.
constexpr int Q_HEAD = 0, Q_TAIL = 32, Q_OUT = 64, Q_ROOT = 96, QCTL_WORDS = 128;
// Frame: [0] kind; wide (1): [1] root index, [2] d, [3] (h<<16)|p, [4..4+NW) S;
// compacted (2): [1] (h<<16)|p, [2] S, [4..36) the 32 one-word rows.
constexpr int FRAME_WORDS = 36;
constexpr uint32_t FRAME_WIDE = 1u, FRAME_COMPACT = 2u;

// Block-level (h, p) leaf histogram in shared memory for h < HIST_H, p < HIST_P
// (where almost every leaf falls); other leaves go straight to the global one.
constexpr int HIST_H = 32, HIST_P = 64;

template <bool SHIST>
__device__ __forceinline__ void tally_leaf(unsigned long long *shist, const CountArgs &A, int lane, int h, int p)
{
    if (lane == 0) {
        if (SHIST && h < HIST_H && p < HIST_P) atomicAdd(&shist[h * HIST_P + p], 1ull);
        else atomicAdd(&A.hist[(size_t)h * A.hstride + p], 1ull);
    }
}

// Donated frames must carry enough work to pay for the queue round trip.
constexpr int DONATE_MIN_WIDE = 16;     // members of a wide frame's label
constexpr int DONATE_MIN_COMPACT = 14;  // members of a compacted frame's label

constexpr unsigned long long SPLIT_IDLE_LIMIT_NS = 20000000000ull;  // 20 s without progress
constexpr unsigned long long SPLIT_SLOT_LIMIT_NS = 2000000000ull;  // 2 s for a ring slot to free up

__device__ __forceinline__ unsigned vload(const unsigned *p) { return *(const volatile unsigned *)p; }

// Lane 0: are warps waiting on tickets that no frame fills yet?
__device__ __forceinline__ bool queue_hungry(const CountArgs &A)
{
    return vload(A.qctl + Q_HEAD) > vload(A.qctl + Q_TAIL);
}

// Reserve the slot of the next frame (one more outstanding item); all lanes
// get its ticket number t.  Returns nullptr (status set) if the slot never
// frees up.
__device__ __forceinline__ uint32_t *frame_reserve(const CountArgs &A, int lane, unsigned &t)
{
    int ok = 1;
    if (lane == 0) {
        atomicAdd(A.qctl + Q_OUT, 1u);
        t = atomicAdd(A.qctl + Q_TAIL, 1u);
        if (t >= A.qcap) {
            const unsigned want = t - A.qcap + 1u, slot = t & (A.qcap - 1u);
            const unsigned long long t0 = global_ns();
            while (vload(A.qdone + slot) != want) {
                if (global_ns() - t0 > SPLIT_SLOT_LIMIT_NS) { atomicOr(A.err, DERR_TIMEOUT); ok = 0; break; }
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

struct WalkCounters {
    unsigned long long nodes = 0, leaves = 0, words = 0;
};

// Edge id of the edge between members a and b (local indices, d = root).
template <int NW>
__device__ __forceinline__ uint32_t member_edge_id(const WarpWork<NW> &Wk, const CountArgs &A,
                                                   int64_t rbeg, int d, int a, int b)
{
    if (a == d) return A.oeid[rbeg + b];
    if (b == d) return A.oeid[rbeg + a];
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
        // Alg. 2 steps hht / pht / ppt over unordered member pairs
        const int L = h + p;
        for (int a = 0; a < L - 1; ++a) {
            for (int b = a + 1 + lane; b < L; b += 32) {
                int la = a < h ? Wk.memH[a] : Wk.memP[a - h];
                int lb = b < h ? Wk.memH[b] : Wk.memP[b - h];
                uint32_t e = member_edge_id(Wk, A, rbeg, d, la, lb);
                if (e == 0xFFFFFFFFu) continue;
                unsigned long long *cell = A.out + (size_t)e * (A.kmax + 1) * A.W;
                int npiv = (a >= h) + (b >= h);
                add_binom_row(cell, h + npiv, p - npiv, A);
            }
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
// the queue is consulted once every DONATE_EVERY nodes.
struct Clock {
    unsigned nodes = 0, next = 0;
};
constexpr unsigned DONATE_EVERY = 16;

// Hand wide frame f (of root qi, out-degree d) to the frame queue.
template <int NW>
__device__ __forceinline__ void donate_wide(WarpWork<NW> &Wk, const CountArgs &A, int lane, int f, unsigned qi,
                                            int d)
{
    unsigned t = 0;
    uint32_t *fr = frame_reserve(A, lane, t);
    if (!fr) return;
    if (lane < NW) fr[4 + lane] = Wk.stk[f * NW + lane];
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
    int top = 0, bot = 0;
    for (;;) {
        const int s1 = __popc(S1);
        wc.nodes++;
        clk.nodes++;
        bool closed = true;
        if (s1 == 0) {
            wc.leaves++;
            tally(h, p);
        } else {
            const bool in = (S1 >> lane) & 1u;
            const uint32_t c = in ? __popc(r1 & S1) : 0u;
            const uint32_t best = __reduce_max_sync(FULL, in ? (((c + 1u) << 5) | (31u - lane)) : 0u);
            const uint32_t dsum = __reduce_add_sync(FULL, c);
            wc.words += (unsigned long long)s1;
            if (dsum == (uint32_t)s1 * (uint32_t)(s1 - 1)) {
                wc.leaves++;
                tally(h, p + s1);
            } else {
                closed = false;
                const int piv = 31 - (int)(best & 31u);
                const uint32_t rp = __shfl_sync(FULL, r1, piv);
                const uint32_t R = S1 & ~rp & ~(1u << piv);
                const int nR = __popc(R);
                if (nR > 0 && h + 1 <= A.kmax) {
                    if (SPLIT && bot > 0 && top + nR > 33) {
                        __syncwarp();
                        for (int t = lane; t < top - bot; t += 32) {
                            Wk.stk1[t] = Wk.stk1[bot + t];
                            Wk.hp1[t] = Wk.hp1[bot + t];
                        }
                        top -= bot;
                        bot = 0;
                        __syncwarp();
                    }
                    if (top + nR > 33) {
                        if (lane == 0) atomicOr(A.err, DERR_STACK);
                        return;
                    }
                    __syncwarp();
                    if ((R >> lane) & 1u) {
                        const uint32_t below = R & ((1u << lane) - 1u);
                        const int f = top + __popc(below);
                        Wk.stk1[f] = r1 & S1 & ~below;
                        Wk.hp1[f] = ((uint32_t)(h + 1) << 16) | (uint32_t)p;
                    }
                    top += nR;
                    __syncwarp();
                    if (SPLIT && clk.nodes >= clk.next) {
                        clk.next = clk.nodes + DONATE_EVERY;
                        // waiting warps get the largest pending work first: the
                        // enclosing wide walk's oldest frame, else our oldest
                        int ndon = 0, wide = 0;
                        if (lane == 0 && queue_hungry(A)) {
                            if (outer && *outer->top - *outer->bot >= 1) {
                                int sz = 0;
#pragma unroll
                                for (int w = 0; w < NW; ++w) sz += __popc(Wk.stk[*outer->bot * NW + w]);
                                wide = sz >= DONATE_MIN_WIDE;
                            }
                            if (!wide && top - bot >= 2 && __popc(Wk.stk1[bot]) >= DONATE_MIN_COMPACT) ndon = 1;
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
                                    fr[1] = Wk.hp1[bot];
                                    fr[2] = Wk.stk1[bot];
                                }
                                frame_publish(A, lane, t);
                                bot += 1;
                            }
                        }
                    }
                }
                S1 = rp & S1;
                p += 1;
            }
        }
        if (!closed) continue;
        if (top == bot) break;
        --top;
        S1 = Wk.stk1[top];
        const uint32_t hp = Wk.hp1[top];
        h = (int)(hp >> 16);
        p = (int)(hp & 0xFFFFu);
    }
    __syncwarp();
}

// Compact a node whose label S (in NW-word bitsets over the root's members)
// has s <= 32 members: relabel them 0..s-1 in ascending order; lane k gets
// row k of the induced adjacency -- by symmetry, the ballot over lanes j of
// "member k is in my row" is exactly that row.
template <int NW, bool SHIST, bool SPLIT>
__device__ void walk_compact(WarpWork<NW> &Wk, unsigned long long *shist, const CountArgs &A, int lane,
                             const uint32_t *S, int s, int h, int p, WalkCounters &wc, const Outer *outer,
                             Clock &clk)
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
    compact_loop<NW, SHIST, SPLIT>(Wk, shist, A, lane, r1, s >= 32 ? FULL : ((1u << s) - 1u), h, p, wc, outer,
                                   clk);
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
    const uint32_t T = base;
    for (uint32_t t = lane; t < T; t += 32) {
        int lo = 0, hi = d - 1;  // largest i with off[i] <= t
        while (lo < hi) {
            int mid = (lo + hi + 1) >> 1;
            if (Wk.off[mid] <= t) lo = mid; else hi = mid - 1;
        }
        uint32_t x = A.ocol[Wk.rs[lo] + (t - Wk.off[lo])];
        int a = 0, b = d;
        while (a < b) {
            int mid = (a + b) >> 1;
            if (Wk.ids[mid] < x) a = mid + 1; else b = mid;
        }
        if (a < d && Wk.ids[a] == x) {
            atomicOr(&Wk.adj[lo * RS + (a >> 5)], 1u << (a & 31));
            atomicOr(&Wk.adj[a * RS + (lo >> 5)], 1u << (lo & 31));
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
#pragma unroll
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
            wc.words += (unsigned long long)s * NW;
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
                closed = false;
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
                        for (int t = lane; t < (top - bot) * NW; t += 32) Wk.stk[t] = Wk.stk[bot * NW + t];
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
                    int before = 0;
#pragma unroll
                    for (int j = 0; j < NW; ++j) {
                        if ((R[j] >> lane) & 1u) {
                            const uint32_t low = (1u << lane) - 1u;
                            const int f = top + before + __popc(R[j] & low);
#pragma unroll
                            for (int w = 0; w < NW; ++w) {
                                uint32_t below = w < j ? R[w] : (w == j ? (R[j] & low) : 0u);
                                Wk.stk[f * NW + w] = row(j, w) & S[w] & ~below;
                            }
                            Wk.hp[f] = ((uint32_t)(h + 1) << 16) | (uint32_t)p;
                            if (MODE != MODE_GLOBAL) Wk.lk[f] = (uint16_t)(j * 32 + lane);
                        }
                        before += __popc(R[j]);
                    }
                    top += nR;
                    __syncwarp();  // pushed frames visible to every lane
                    if (SPLIT && clk.nodes >= clk.next) {
                        clk.next = clk.nodes + DONATE_EVERY;
                        // donate the oldest pending frame (largest subtree) to an idle warp
                        int ndon = 0;
                        if (lane == 0 && top - bot >= 2) {
                            int sz = 0;
#pragma unroll
                            for (int w = 0; w < NW; ++w) sz += __popc(Wk.stk[bot * NW + w]);
                            if (sz >= DONATE_MIN_WIDE && queue_hungry(A)) ndon = 1;
                        }
                        ndon = __shfl_sync(FULL, ndon, 0);
                        for (int k = 0; k < ndon; ++k) donate_wide<NW>(Wk, A, lane, bot + k, qi, d);
                        bot += ndon;
                    }
                }
                // continue into the pivot child N(S, piv)
#pragma unroll
                for (int w = 0; w < NW; ++w) S[w] = P[w];
                p += 1;
                link = (uint16_t)(LINK_PIVOT | piv);
            }
        }
        if (!closed) continue;
        if (top == bot) break;
        --top;
#pragma unroll
        for (int w = 0; w < NW; ++w) S[w] = Wk.stk[top * NW + w];
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
    return NW <= 2 ? 8 : (NW <= 8 ? 4 : 2);
}

template <int NW, int MODE, bool SHIST>
constexpr size_t smem_bytes()
{
    return sizeof(WarpWork<NW>) * warps_per_block<NW>() +
           (SHIST ? sizeof(unsigned long long) * HIST_H * HIST_P : 0);
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
            int kind = 0;  // 1: donated frame in slot v, 2: fresh root v, 3: no more work
            unsigned v = 0;
            if (lane == 0) {
                if (vload(A.qctl + Q_ROOT) < A.nroots) {
                    const unsigned rr = atomicAdd(A.qctl + Q_ROOT, 1u);
                    if (rr < A.nroots) { kind = 2; v = rr; }
                }
                if (kind == 0) {
                    // a ticket for the next donated frame; wait on its own slot
                    const unsigned t = atomicAdd(A.qctl + Q_HEAD, 1u);
                    unsigned last_out = 0xFFFFFFFFu, nap = 64;
                    unsigned long long t0 = global_ns();
                    const unsigned slot = t & (A.qcap - 1u);
                    for (;;) {
                        if (vload(A.qready + slot) == t + 1u) { kind = 1; v = t; break; }
                        const unsigned out = vload(A.qctl + Q_OUT);
                        if (out == 0 || (vload(A.err) & (DERR_STACK | DERR_RANGE | DERR_TIMEOUT))) { kind = 3; break; }
                        if (out != last_out) { last_out = out; t0 = global_ns(); }
                        else if (global_ns() - t0 > SPLIT_IDLE_LIMIT_NS) { atomicOr(A.err, DERR_TIMEOUT); kind = 3; break; }
                        __nanosleep(nap);
                        nap = min(nap * 2u, 2048u);
                    }
                    if (kind == 1) __threadfence();
                }
            }
            kind = __shfl_sync(FULL, kind, 0);
            v = __shfl_sync(FULL, v, 0);
            if (kind == 3) break;
            if (kind == 1) {
                // copy the frame out and release its ring slot at once
                const uint32_t *fr = A.qframes + (size_t)(v & (A.qcap - 1u)) * FRAME_WORDS;
                uint32_t *fb = ww[wid].fbuf;
                fb[lane] = __ldcg(fr + lane);
                if (lane < FRAME_WORDS - 32) fb[32 + lane] = __ldcg(fr + 32 + lane);
                __syncwarp();
                if (lane == 0) {
                    __threadfence();
                    atomicExch(A.qdone + (v & (A.qcap - 1u)), v + 1u);
                }
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
        ++qi;
        if (!PERSIST) break;
        if (*(volatile unsigned *)A.err & (DERR_STACK | DERR_RANGE)) break;
    }
    if (lane == 0 && wc.nodes) {
        atomicAdd(&A.stats[0], wc.nodes);
        atomicAdd(&A.stats[1], wc.leaves);
        atomicAdd(&A.stats[2], wc.words);
        atomicAdd(&A.stats[3 + A.cls], wc.words);
    }
    if (SHIST) {
        __syncthreads();
        for (int i = threadIdx.x; i < HIST_H * HIST_P; i += blockDim.x) {
            unsigned long long v = shist[i];
            if (v) atomicAdd(&A.hist[(size_t)(i / HIST_P) * A.hstride + (i % HIST_P)], v);
        }
    }
}

// ------------------------------------------------------ small kernels

// Roots with no out-neighbour: one path each with h = 1, p = 0.
__global__ void k_add_leaf(unsigned long long *cell, unsigned long long count)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) *cell += count;
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

// ------------------------------------------------------------- driver

template <typename T>
static pvt_status grow(DevBuf<T> &b, size_t n, cudaStream_t s)
{
    if (b.n >= n) return PVT_OK;
    if (b.p) PVT_CK(cudaFreeAsync(b.p, s));
    b.p = nullptr;
    b.n = 0;
    PVT_CK(cudaMallocAsync(&b.p, n * sizeof(T), s));
    b.n = n;
    return PVT_OK;
}

static pvt_status ensure_binom(pvt_dag *g, int W, cudaStream_t s)
{
    const int rows = g->alpha + 3;
    if (g->binom_rows == rows && g->binom_W == W) return PVT_OK;
    pvt_status st = grow(g->binom, (size_t)rows * (rows + 1) / 2 * W, s);
    if (st != PVT_OK) return st;
    k_binom<<<1, 1024, 0, s>>>(g->binom.p, rows, W, g->d_err);
    PVT_CK(cudaGetLastError());
    g->stats.launches++;
    g->binom_rows = rows;
    g->binom_W = W;
    return PVT_OK;
}

// Queue counters of a split launch: head, tail, outstanding items (= roots),
// next root, idle warps.
__global__ void k_split_init(uint32_t *qctl, unsigned nroots)
{
    for (int i = threadIdx.x; i < QCTL_WORDS; i += blockDim.x) qctl[i] = i == Q_OUT ? nroots : 0u;
}

constexpr unsigned SPLIT_QCAP = 1u << 17;

template <int NW, int MODE, bool SHIST>
static pvt_status launch_class(pvt_dag *g, const CountArgs &base, int cls, cudaStream_t s)
{
    const unsigned cnt = (unsigned)g->class_cnt[cls];
    if (cnt == 0) return PVT_OK;
    CountArgs A = base;
    A.roots = g->roots + g->class_start[cls];
    A.nroots = cnt;
    A.qhead = g->d_q + cls;
    A.cls = cls;
    A.chunk = (unsigned)g->policy.chunk;
    constexpr size_t smem = smem_bytes<NW, MODE, SHIST>();
    constexpr int WPB = warps_per_block<NW>();
    const bool persist = g->policy.persistent != 0;
    // heavy classes of the global count split subtrees across warps
    const bool split = persist && NW >= 2 && MODE == MODE_GLOBAL;
    auto kern = split ? k_count<NW, MODE, SHIST, true, true>
                      : (persist ? k_count<NW, MODE, SHIST, true, false> : k_count<NW, MODE, SHIST, false, false>);
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
    if (persist) {
        int per_sm = 0;
        PVT_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 32 * WPB, smem));
        if (per_sm < 1) {
            set_error("count kernel cannot be resident (shared memory)");
            return PVT_ECUDA;
        }
        grid = std::min<unsigned>((unsigned)(g->num_sms * per_sm), need);
    }
    phase_begin(g, 1 + cls, s);
    kern<<<grid, 32 * WPB, smem, s>>>(A);
    PVT_CK(cudaGetLastError());
    phase_end(g, 1 + cls, s);
    g->stats.launches++;
    return PVT_OK;
}

template <int MODE>
static pvt_status launch_all(pvt_dag *g, const CountArgs &A, cudaStream_t s)
{
    // heavy classes on side streams so that they overlap the light ones
    PVT_CK(cudaEventRecord(g->ev_fork, s));
    pvt_status st = PVT_OK;
    for (int c = NCLASS - 1; c >= 1 && st == PVT_OK; --c) {
        cudaStream_t cs = g->side[c];
        PVT_CK(cudaStreamWaitEvent(cs, g->ev_fork, 0));
        switch (c) {
            case 1: st = launch_class<1, MODE, MODE == MODE_GLOBAL>(g, A, c, cs); break;
            case 2: st = launch_class<2, MODE, MODE == MODE_GLOBAL>(g, A, c, cs); break;
            case 3: st = launch_class<4, MODE, MODE == MODE_GLOBAL>(g, A, c, cs); break;
            case 4: st = launch_class<8, MODE, MODE == MODE_GLOBAL>(g, A, c, cs); break;
            case 5: st = launch_class<16, MODE, MODE == MODE_GLOBAL>(g, A, c, cs); break;
        }
        PVT_CK(cudaEventRecord(g->ev_join[c], cs));
    }
    for (int c = NCLASS - 1; c >= 1; --c) PVT_CK(cudaStreamWaitEvent(s, g->ev_join[c], 0));
    return st;
}

static void begin_call(pvt_dag *g)
{
    stats_reset(g);
    for (int c = 0; c < NCLASS; ++c) g->stats.roots[c] = (uint64_t)g->class_cnt[c];
}

// Copy the walk statistics back, synchronise and check the device status.
static pvt_status end_call(pvt_dag *g, cudaStream_t s, const char *fn)
{
    PVT_CK(cudaMemcpyAsync(g->h_stats, g->d_stats, (3 + NCLASS) * sizeof(unsigned long long),
                           cudaMemcpyDeviceToHost, s));
    pvt_status st = check_device(g, s, fn);
    g->stats.sct_nodes = g->h_stats[0];
    g->stats.sct_leaves = g->h_stats[1];
    g->stats.pivot_words = g->h_stats[2];
    for (int c = 0; c < NCLASS; ++c) g->stats.class_words[c] = g->h_stats[3 + c];
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

pvt_status count_global(pvt_dag *g, int32_t kmax, int32_t W, uint64_t *C, cudaStream_t s)
{
    pvt_status st = check_args(g, kmax, W, C, 1, "pvt_count_global");
    if (st != PVT_OK) return st;
    begin_call(g);
    const int hstride = g->alpha + 2;
    if ((st = grow(g->hist, (size_t)hstride * hstride, s)) != PVT_OK) return st;
    if ((st = ensure_binom(g, W, s)) != PVT_OK) return st;
    PVT_CK(cudaMemsetAsync(g->d_err, 0, sizeof(unsigned), s));
    PVT_CK(cudaMemsetAsync(g->d_q, 0, 16 * sizeof(unsigned), s));
    PVT_CK(cudaMemsetAsync(g->hist.p, 0, (size_t)hstride * hstride * sizeof(unsigned long long), s));
    PVT_CK(cudaMemsetAsync(g->d_stats, 0, 16 * sizeof(unsigned long long), s));
    if (g->class_cnt[0] && kmax >= 1) {
        k_add_leaf<<<1, 32, 0, s>>>(g->hist.p + hstride, (unsigned long long)g->class_cnt[0]);
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
    if ((st = launch_all<MODE_GLOBAL>(g, A, s)) != PVT_OK) return st;
    phase_begin(g, 7, s);
    k_combine<<<kmax + 1, 256, 0, s>>>(g->hist.p, hstride, g->binom.p, W, kmax,
                                       reinterpret_cast<unsigned long long *>(C), g->d_err);
    PVT_CK(cudaGetLastError());
    phase_end(g, 7, s);
    g->stats.launches++;
    return end_call(g, s, "pvt_count_global");
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
    st = edge ? launch_all<MODE_EDGE>(g, A, s) : launch_all<MODE_VERTEX>(g, A, s);
    if (st != PVT_OK) return st;
    return end_call(g, s, fn);
}


}  // namespace pvt

namespace pvt {

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
                  const unsigned long long *B, int Bw, unsigned *err, unsigned long long *stats)
{
    constexpr int WPB = warps_per_block<NW>();
    extern __shared__ __align__(16) unsigned char smem[];
    WarpWork<NW> *ww = reinterpret_cast<WarpWork<NW> *>(smem);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
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
        if (vload(err) & (DERR_STACK | DERR_RANGE)) break;
    }
    (void)WPB;
    if (lane == 0 && wc.nodes) {
        atomicAdd(&stats[0], wc.nodes);
        atomicAdd(&stats[1], wc.leaves);
        atomicAdd(&stats[2], wc.words);
    }
}

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

template <int NW, int MODE>
static pvt_status launch_batch_class(const BatchGraph *gs, const uint64_t *entries, unsigned cnt, unsigned *qhead,
                                     const unsigned long long *B, int Bw, unsigned *err,
                                     unsigned long long *stats, int num_sms, cudaStream_t s)
{
    constexpr size_t smem = sizeof(WarpWork<NW>) * warps_per_block<NW>();
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
    kern<<<grid, 32 * warps_per_block<NW>(), smem, s>>>(gs, entries, cnt, qhead, B, Bw, err, stats);
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
        if (vload(A.err) & (DERR_STACK | DERR_RANGE)) break;
    }
    (void)WPB;
    if (lane == 0 && wc.nodes) {
        atomicAdd(&A.stats[0], wc.nodes);
        atomicAdd(&A.stats[1], wc.leaves);
        atomicAdd(&A.stats[2], wc.words);
    }
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
    using namespace pvt;
    if (n < 0 || n > 0xFFFFFFFEll || (n > 0 && !orow) || !C || kmax < 0 || alpha < 0 || W < 1) {
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
    if (herr) {
        set_error("pvt_count_global_noalloc: device capacity check failed");
        return PVT_EINTERNAL;
    }
    return PVT_OK;
}
