"""Pins of the CPU oracle to facts outside itself (no GPU).

Each check targets a part of the oracle a plausible mistake could break:
closed forms on complete, disjoint-union and complete multipartite graphs
(binomials, sums, elementary symmetric polynomials), brute-force clique
enumeration on random graphs (all three tables), matrix identities for
triangles, the counting identities of Alg. 2 (sum of local counts), the
unique-encoding theorem (Thm. scr) on explicit SCT paths, relabelling,
truncation, the degeneracy order, textbook graphs, and multi-limb overflow.
"""
from __future__ import annotations

import itertools
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_2001_06784_gb300 import graphgen
from tests import graphs

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "named_graphs.json")


# ------------------------------------------------------------ brute force

def all_cliques(row_ptr, col):
    """Every non-empty clique, each once, grown in increasing vertex order
    (plain backtracking, no pivoting, no orientation)."""
    adj = graphs.adjacency_sets(row_ptr, col)
    n = len(adj)
    out = []

    def grow(clique, cand):
        for i, v in enumerate(cand):
            c = clique + [v]
            out.append(tuple(c))
            grow(c, [u for u in cand[i + 1:] if u in adj[v]])

    grow([], list(range(n)))
    return out


def brute_counts(row_ptr, col, K):
    n = len(row_ptr) - 1
    eid = {tuple(e): i for i, e in enumerate(graphgen.edge_list(row_ptr, col).tolist())}
    C = [0] * (K + 1)
    cv = [[0] * (K + 1) for _ in range(n)]
    ce = [[0] * (K + 1) for _ in range(len(eid))]
    for c in all_cliques(row_ptr, col):
        k = len(c)
        if k > K:
            continue
        C[k] += 1
        for v in c:
            cv[v][k] += 1
        for a, b in itertools.combinations(c, 2):
            ce[eid[(min(a, b), max(a, b))]][k] += 1
    return C, cv, ce


def esym(parts, k):
    """Elementary symmetric polynomial e_k(parts)."""
    return sum(math.prod(c) for c in itertools.combinations(parts, k))


# ------------------------------------------------------------ closed forms

@pytest.mark.parametrize("n", [1, 2, 3, 4, 7, 12, 33, 64])
def test_complete_graph_all_tables(n):
    rp, col = graphs.complete(n)
    r = oracle.count(rp, col, vertex=True, edge=n <= 33)
    K = r["kmax"]
    assert r["C"] == [0] + [math.comb(n, k) for k in range(1, K + 1)]
    cv = oracle.to_int(r["cv"])
    for v in range(n):
        assert cv[v] == [0] + [math.comb(n - 1, k - 1) for k in range(1, K + 1)]
    if n <= 33:
        for row in oracle.to_int(r["ce"]):
            assert row == [0, 0] + [math.comb(n - 2, k - 2) for k in range(2, K + 1)]


def test_complete_graph_many_limbs():
    # C(250, 125) ~ 2^246: exercises carries across eight 32-bit limbs
    n = 250
    rp, col = graphs.complete(n)
    r = oracle.count(rp, col)
    assert r["nl"] >= 8
    assert r["C"] == [0] + [math.comb(n, k) for k in range(1, n + 1)]


@pytest.mark.parametrize("sizes", [[3, 5, 7, 4, 1, 2], [10, 10, 1, 1, 6], [30, 2, 17]])
def test_disjoint_cliques(sizes):
    rp, col = graphs.disjoint_cliques(sizes)
    r = oracle.count(rp, col, vertex=True)
    K = r["kmax"]
    assert r["C"] == [0] + [sum(math.comb(a, k) for a in sizes) for k in range(1, K + 1)]
    cv = oracle.to_int(r["cv"])
    v = 0
    for a in sizes:
        for _ in range(a):
            assert cv[v] == [0] + [math.comb(a - 1, k - 1) for k in range(1, K + 1)]
            v += 1


@pytest.mark.parametrize("parts", [[3, 3, 3, 3, 3, 3], [5, 4, 3, 2, 1], [1, 1, 1, 1], [7, 1], [2, 2, 2, 2, 2, 2, 2]])
def test_complete_multipartite(parts):
    rp, col = graphs.multipartite(parts)
    r = oracle.count(rp, col)
    K = r["kmax"]
    assert r["C"] == [0] + [esym(parts, k) for k in range(1, K + 1)]


def test_named_graphs_golden():
    data = json.load(open(GOLDEN))
    for g in data["graphs"]:
        rp, col = graphgen.from_edges(g["n"], g["edges"])
        r = oracle.count(rp, col)
        C = r["C"] + [0] * 8
        want = g["C"] + [0] * (len(r["C"]) + 8 - len(g["C"]))
        assert C[:len(want)] == want[:len(C)], g["name"]


# ------------------------------------------------------------ brute force

@pytest.mark.parametrize("n,p,seed", [(12, 0.5, 0), (20, 0.5, 1), (30, 0.3, 2), (40, 0.2, 3), (18, 0.75, 4),
                                      (25, 0.6, 5), (36, 0.4, 6)])
def test_bruteforce_random_graphs(n, p, seed):
    rp, col = graphs.gnp(n, p, seed)
    r = oracle.count(rp, col, vertex=True, edge=True)
    K = r["kmax"]
    C, cv, ce = brute_counts(rp, col, K)
    assert r["C"] == C
    assert oracle.to_int(r["cv"]) == cv
    assert oracle.to_int(r["ce"]) == ce


def test_bruteforce_planted():
    rp, col = graphgen.generate(40, er_avg_deg=5.0, planted=[(2, 8, 12, 1.0), (1, 10, 10, 0.8)], seed=3)
    r = oracle.count(rp, col, vertex=True, edge=True)
    C, cv, ce = brute_counts(rp, col, r["kmax"])
    assert r["C"] == C and oracle.to_int(r["cv"]) == cv and oracle.to_int(r["ce"]) == ce


# ------------------------------------------------------------ matrix identities

@pytest.mark.parametrize("kind", ["gnp", "er2k"])
def test_triangles_from_adjacency_powers(kind):
    if kind == "gnp":
        rp, col = graphs.gnp(300, 0.06, 11)
    else:
        rp, col = graphgen.workload("er2k_d20_clique30")
    n = len(rp) - 1
    A = np.zeros((n, n))
    src = np.repeat(np.arange(n), np.diff(rp))
    A[src, col.astype(np.int64)] = 1.0
    A2 = A @ A
    A3diag = np.einsum("ij,ji->i", A2, A)
    r = oracle.count(rp, col, kmax=3, vertex=True, edge=True)
    assert r["C"][3] == int(round(A3diag.sum() / 6))
    cv = oracle.to_int(r["cv"])
    assert [row[3] for row in cv] == [int(round(x / 2)) for x in A3diag]
    ce = oracle.to_int(r["ce"])
    edges = graphgen.edge_list(rp, col)
    assert [row[3] for row in ce] == [int(round(A2[u, v])) for u, v in edges]


# oracle.triangles: a second, SCT-free route to C_3 (used at full size)

@pytest.mark.parametrize("kind", ["gnp", "er2k", "planted"])
def test_triangle_enumeration_pins(kind):
    """orc_triangles equals trace(A^3)/6 and the SCT oracle's C_3, for one
    thread and several."""
    if kind == "gnp":
        rp, col = graphs.gnp(250, 0.08, 5)
    elif kind == "er2k":
        rp, col = graphgen.workload("er2k_d20_clique30")
    else:
        rp, col = graphgen.generate(400, er_avg_deg=6.0, planted=[(3, 10, 25, 0.8)], seed=9)
    n = len(rp) - 1
    A = np.zeros((n, n))
    src = np.repeat(np.arange(n), np.diff(rp))
    A[src, col.astype(np.int64)] = 1.0
    trace = int(round(np.einsum("ij,jk,ki->", A, A, A) / 6))
    t1, t4 = oracle.triangles(rp, col), oracle.triangles(rp, col, threads=4)
    assert t1 == t4 == trace == oracle.count(rp, col, kmax=3)["C"][3]


@pytest.mark.parametrize("n", [0, 1, 2, 3, 5, 17, 64])
def test_triangle_enumeration_closed_forms(n):
    """C(n, 3) on K_n, and disjoint cliques add up; no triangle in a star or
    a complete bipartite graph."""
    rp, col = graphs.complete(n)
    assert oracle.triangles(rp, col) == math.comb(n, 3)
    sizes = [n, 4, 3, 1]
    rp, col = graphs.disjoint_cliques(sizes)
    assert oracle.triangles(rp, col, threads=3) == sum(math.comb(s, 3) for s in sizes)
    rp, col = graphs.multipartite([1, n + 1])
    assert oracle.triangles(rp, col) == 0
    rp, col = graphs.multipartite([n + 2, 7])
    assert oracle.triangles(rp, col) == 0


def test_local_sum_identities():
    rp, col = graphgen.generate(600, er_avg_deg=9.0, planted=[(4, 8, 20, 1.0), (2, 15, 25, 0.85)], seed=21)
    n, m = len(rp) - 1, len(col) // 2
    r = oracle.count(rp, col, vertex=True, edge=True)
    C, cv, ce = r["C"], oracle.to_int(r["cv"]), oracle.to_int(r["ce"])
    K = r["kmax"]
    assert C[1] == n and C[2] == m
    for k in range(K + 1):
        assert sum(row[k] for row in cv) == k * C[k]
        assert sum(row[k] for row in ce) == math.comb(k, 2) * C[k]
    deg = np.diff(rp)
    assert [row[1] for row in cv] == [1] * n
    assert [row[2] for row in cv] == [int(d) for d in deg]
    assert all(row[2] == 1 for row in ce)
    omega = max(k for k in range(K + 1) if C[k])
    assert omega <= r["alpha"] + 1


# ------------------------------------------------------------ Thm. scr

@pytest.mark.parametrize("make", [lambda: graphs.gnp(14, 0.5, 7), lambda: graphs.gnp(18, 0.65, 8),
                                  lambda: graphs.multipartite([2, 3, 2, 2]),
                                  lambda: graphs.complete(6), lambda: graphs.clique_minus_star(9, 2, 3)])
def test_unique_encoding(make):
    """Every clique is H(T) + Q for exactly one path T and Q subset of P(T)."""
    rp, col = make()
    adj = graphs.adjacency_sets(rp, col)
    seen = []
    for H, P in oracle.paths(rp, col):
        members = H + P
        assert len(set(members)) == len(members)
        for a, b in itertools.combinations(members, 2):
            assert b in adj[a], "path vertices must form a clique"
        for k in range(len(P) + 1):
            for Q in itertools.combinations(P, k):
                seen.append(tuple(sorted(H + list(Q))))
    assert len(seen) == len(set(seen)), "a clique is represented twice"
    assert set(seen) == set(tuple(sorted(c)) for c in all_cliques(rp, col))


# ------------------------------------------------------------ invariances

def test_relabelling_invariance():
    rp, col = graphgen.generate(300, er_avg_deg=10.0, planted=[(3, 10, 18, 1.0)], seed=4)
    n = len(rp) - 1
    perm = np.random.default_rng(1).permutation(n)
    rp2, col2 = graphs.relabel(rp, col, perm)
    a = oracle.count(rp, col, vertex=True, edge=True)
    b = oracle.count(rp2, col2, kmax=a["kmax"], vertex=True, edge=True)
    assert a["C"] == b["C"]
    cva, cvb = oracle.to_int(a["cv"]), oracle.to_int(b["cv"])
    assert all(cva[v] == cvb[perm[v]] for v in range(n))
    ea = graphgen.edge_list(rp, col)
    eb = {tuple(e): i for i, e in enumerate(graphgen.edge_list(rp2, col2).tolist())}
    cea, ceb = oracle.to_int(a["ce"]), oracle.to_int(b["ce"])
    for i, (u, v) in enumerate(ea):
        x, y = perm[u], perm[v]
        assert cea[i] == ceb[eb[(min(x, y), max(x, y))]]


def test_truncation_matches_prefix():
    rp, col = graphgen.generate(500, er_avg_deg=12.0, planted=[(2, 12, 20, 1.0)], seed=6)
    full = oracle.count(rp, col, vertex=True, edge=True)
    for kmax in [0, 1, 2, 3, 6]:
        t = oracle.count(rp, col, kmax=kmax, vertex=True, edge=True)
        assert t["C"] == full["C"][:kmax + 1]
        assert (t["cv"] == full["cv"][:, :kmax + 1]).all()
        assert (t["ce"] == full["ce"][:, :kmax + 1]).all()
        assert t["nodes"] <= full["nodes"]


def test_edge_deletion_is_monotone():
    rp, col = graphgen.generate(200, er_avg_deg=14.0, planted=[(2, 10, 14, 1.0)], seed=8)
    e = graphgen.edge_list(rp, col)
    keep = np.random.default_rng(2).random(len(e)) > 0.1
    rp2, col2 = graphgen.from_edges(len(rp) - 1, e[keep])
    a = oracle.count(rp, col)
    b = oracle.count(rp2, col2, kmax=a["kmax"])
    assert all(x >= y for x, y in zip(a["C"], b["C"]))


# ------------------------------------------------------------ degeneracy

def core_numbers(row_ptr, col):
    """k-cores by repeated deletion of vertices of degree < k (definition)."""
    adj = graphs.adjacency_sets(row_ptr, col)
    n = len(adj)
    core = [0] * n
    alive = set(range(n))
    k = 0
    while alive:
        k += 1
        changed = True
        while changed:
            changed = False
            for v in list(alive):
                if len(adj[v] & alive) < k:
                    alive.discard(v)
                    core[v] = k - 1
                    changed = True
    return core


@pytest.mark.parametrize("make", [lambda: graphs.gnp(60, 0.2, 1), lambda: graphs.complete(9),
                                  lambda: graphgen.generate(400, er_avg_deg=6.0, planted=[(2, 9, 15, 1.0)], seed=2)])
def test_degeneracy_order(make):
    rp, col = make()
    rank, core, alpha = oracle.orient(rp, col)
    want = core_numbers(rp, col)
    assert list(core) == want
    assert alpha == max(want)
    # every vertex has at most alpha neighbours ranked after it
    n = len(rp) - 1
    for v in range(n):
        nb = col[rp[v]:rp[v + 1]]
        assert (rank[nb] > rank[v]).sum() <= alpha


def test_limb_overflow_is_reported():
    rp, col = graphs.complete(40)  # C(40,20) > 2^32
    with pytest.raises(RuntimeError, match="overflow"):
        oracle.count(rp, col, nl=1)
    assert oracle.count(rp, col, nl=2)["C"][20] == math.comb(40, 20)


# ------------------------------------------ f_k(b), "Demonstrations of Pivoter"

@pytest.mark.parametrize("sizes", [[5], [4, 7, 7], [1, 3, 9, 12]])
def test_frequency_closed_form(sizes):
    """Disjoint cliques: a vertex of K_a lies in C(a-1, k-1) k-cliques and an
    edge of K_a in C(a-2, k-2)."""
    rp, col = graphs.disjoint_cliques(sizes)
    r = oracle.count(rp, col, vertex=True, edge=True)
    for k in range(r["kmax"] + 1):
        want_v, want_e = {}, {}
        for a in sizes:
            b = math.comb(a - 1, k - 1) if k >= 1 else 0
            want_v[b] = want_v.get(b, 0) + a
            if a >= 2:
                b = math.comb(a - 2, k - 2) if k >= 2 else 0
                want_e[b] = want_e.get(b, 0) + math.comb(a, 2)
        assert oracle.frequency(r["cv"], k) == want_v
        assert oracle.frequency(r["ce"], k) == want_e


@pytest.mark.parametrize("n,p,seed", [(12, 0.5, 1), (16, 0.6, 2), (20, 0.45, 3)])
def test_frequency_bruteforce(n, p, seed):
    """f_k from brute-force per-vertex / per-edge clique counts; the mass and
    first moment identities sum f_k(b) = rows, sum b f_k(b) = k C_k (vertices)
    or C(k,2) C_k (edges)."""
    rp, col = graphs.gnp(n, p, seed)
    r = oracle.count(rp, col, vertex=True, edge=True)
    K = r["kmax"]
    _, bv, be = brute_counts(rp, col, K)
    m = len(col) // 2
    for k in range(K + 1):
        fv = oracle.frequency(r["cv"], k)
        fe = oracle.frequency(r["ce"], k)
        want_v, want_e = {}, {}
        for row in bv:
            want_v[row[k]] = want_v.get(row[k], 0) + 1
        for row in be:
            want_e[row[k]] = want_e.get(row[k], 0) + 1
        assert fv == want_v and fe == want_e
        assert sum(fv.values()) == n and sum(fe.values()) == m
        assert sum(b * c for b, c in fv.items()) == k * r["C"][k]
        assert sum(b * c for b, c in fe.items()) == math.comb(k, 2) * r["C"][k]


@pytest.mark.parametrize("make", [lambda: graphs.complete(12), lambda: graphs.gnp(200, 0.07, 8),
                                  lambda: graphs.disjoint_cliques([1, 5, 9]),
                                  lambda: graphgen.workload("er2k_d20_clique30")])
def test_path_histogram_invariants(make):
    """The invariants the device checks after every walk, on the oracle's
    (h, p) leaf histogram: each root has exactly one all-pivot path (row
    h = 1 sums to n), and the 2-cliques read off rows 1 and 2,
    sum_p p * hist[1][p] + sum_p hist[2][p], are the m edges."""
    rp, col = make()
    n, m = len(rp) - 1, len(col) // 2
    r = oracle.count(rp, col, hist_dim=0)
    H = r["alpha"] + 2
    hist = oracle.count(rp, col, hist_dim=H)["hist"].astype(np.int64)
    assert int(hist[1].sum()) == n
    assert int((np.arange(H) * hist[1]).sum() + (hist[2].sum() if H > 2 else 0)) == m


# ------------------------------------------ root-parallel mode (Sec. 4, "Parallel version")

def threaded_cases():
    """Graphs whose root counts are not multiples of the oracle's 16-root
    chunks, from a brute-force size to a few thousand roots."""
    return [("gnp37", graphs.gnp(37, 0.45, 9)),
            ("cliques83", graphs.disjoint_cliques([1, 2, 3, 5, 8, 13, 21, 30])),
            ("planted2021", graphgen.generate(2021, er_avg_deg=10.0, planted=[(3, 12, 20, 1.0), (1, 25, 25, 0.9)],
                                              seed=31))]


@pytest.mark.parametrize("idx", [0, 1, 2])
def test_root_parallel_equals_sequential(idx):
    """The root-parallel oracle (roots in chunks of 16 over t threads, private
    counts summed at the end) gives the sequential oracle's counts, SCT
    statistics and (h, p) histogram for t = 2, 3, 7, and C_1 = n, C_2 = m."""
    name, (rp, col) = threaded_cases()[idx]
    n, m = len(rp) - 1, len(col) // 2
    H = oracle.orient(rp, col)[2] + 2
    one = oracle.count(rp, col, hist_dim=H)
    assert one["C"][1] == n and one["C"][2] == m
    if n <= 40:
        assert one["C"] == brute_counts(rp, col, one["kmax"])[0]
    if name == "cliques83":
        sizes = [1, 2, 3, 5, 8, 13, 21, 30]
        assert one["C"] == [0] + [sum(math.comb(a, k) for a in sizes) for k in range(1, one["kmax"] + 1)]
    for t in (2, 3, 7):
        r = oracle.count(rp, col, threads=t, hist_dim=H)
        assert r["C"] == one["C"], (name, t)
        assert (r["nodes"], r["leaves"], r["sum_s"]) == (one["nodes"], one["leaves"], one["sum_s"]), (name, t)
        assert np.array_equal(r["hist"], one["hist"]), (name, t)


def test_root_parallel_ranges_add_up():
    """Disjoint root sets counted with several threads add up to the whole
    count (roots are independent subproblems, Sec. 4)."""
    rp, col = threaded_cases()[2][1]
    n = len(rp) - 1
    whole = oracle.count(rp, col)
    perm = np.random.default_rng(4).permutation(n)
    parts = [np.sort(perm[:701]), np.sort(perm[701:1500]), np.sort(perm[1500:])]
    total = [0] * len(whole["C"])
    for i, roots in enumerate(parts):
        r = oracle.count(rp, col, kmax=whole["kmax"], roots=roots, threads=2 + i)
        assert r["C"][1] == len(roots)
        total = [a + b for a, b in zip(total, r["C"])]
    assert total == whole["C"]


# ------------------------------------------ a caller's orientation; SCT statistics

def id_orientation(row_ptr, col, reverse=False):
    """Out-lists of the acyclic orientation "towards the larger id" (or the
    smaller one), each sorted ascending."""
    n = len(row_ptr) - 1
    src = np.repeat(np.arange(n, dtype=np.int64), np.diff(row_ptr))
    dst = col.astype(np.int64)
    keep = dst < src if reverse else dst > src
    orow = np.zeros(n + 1, dtype=np.int64)
    orow[1:] = np.cumsum(np.bincount(src[keep], minlength=n))
    return orow, dst[keep].astype(np.uint32)


@pytest.mark.parametrize("make", [lambda: graphs.gnp(30, 0.4, 12), lambda: graphs.gnp(24, 0.6, 13),
                                  lambda: graphs.multipartite([3, 2, 4, 1])])
def test_any_acyclic_orientation_counts_the_same(make):
    """Every clique is counted once at its first vertex under any acyclic
    orientation (the paper's degeneracy order only bounds the cost, Lemma
    degen): both id orientations give the brute-force tables."""
    rp, col = make()
    ref = oracle.count(rp, col)
    C, cv, ce = brute_counts(rp, col, ref["kmax"])
    for rev in (False, True):
        r = oracle.count(rp, col, kmax=ref["kmax"], vertex=True, edge=True, dag=id_orientation(rp, col, rev))
        assert r["C"] == C and oracle.to_int(r["cv"]) == cv and oracle.to_int(r["ce"]) == ce


def test_bad_orientation_is_refused():
    rp, col = graphs.gnp(12, 0.5, 3)
    orow, ocol = id_orientation(rp, col)
    # both directions of every edge
    with pytest.raises(RuntimeError, match="invalid"):
        oracle.count(rp, col, dag=(rp, col))
    # the last edge of the last non-empty out-list dropped
    last = int(np.nonzero(np.diff(orow))[0][-1])
    bad_row, bad_col = orow.copy(), np.delete(ocol, orow[last + 1] - 1)
    bad_row[last + 1:] -= 1
    with pytest.raises(RuntimeError, match="invalid"):
        oracle.count(rp, col, dag=(bad_row, bad_col))
    # a directed cycle on a triangle 0 -> 1 -> 2 -> 0
    trp, tcol = graphs.complete(3)
    with pytest.raises(RuntimeError, match="invalid"):
        oracle.count(trp, tcol, dag=(np.array([0, 1, 2, 3]), np.array([1, 2, 0], dtype=np.uint32)))


@pytest.mark.parametrize("n", [1, 2, 5, 12, 40])
def test_clique_chain_closed_forms(n):
    """On K_n the label of root r (degeneracy order) is a clique of n-1-r
    members, so the walk visits its chain of n-r nodes: nodes = n(n+1)/2, the
    chains below the topmost clique labels hold C(n, 2) of them, and a walk
    that closes clique labels at once visits n nodes, one per root."""
    rp, col = graphs.complete(n)
    r = oracle.count(rp, col)
    assert r["nodes"] == n * (n + 1) // 2
    assert r["chain"] == math.comb(n, 2)
    assert r["leaves"] == n


def test_clique_chain_disjoint_cliques_and_bounds():
    """Disjoint cliques add up; on any graph the chains are at most the
    nodes minus the leaves (every chain node but its end is internal)."""
    sizes = [1, 4, 6, 9]
    rp, col = graphs.disjoint_cliques(sizes)
    r = oracle.count(rp, col)
    assert r["chain"] == sum(math.comb(a, 2) for a in sizes)
    assert r["nodes"] == sum(a * (a + 1) // 2 for a in sizes)
    for make in (lambda: graphs.gnp(60, 0.3, 2), lambda: graphgen.workload("er2k_d20_clique30")):
        rp, col = make()
        r = oracle.count(rp, col)
        assert 0 < r["chain"] and r["leaves"] <= r["nodes"] - r["chain"]
