"""GPU path vs the CPU oracle, word for word (integer results: tolerance 0).

Every call goes through the C ABI (paper_2001_06784_gb300 binds it with
ctypes).  Graphs span every bitset class of the root out-degree (<=32, <=64,
<=128, <=256, <=512), ragged sizes, empty graphs and isolated vertices.
"""
from __future__ import annotations

import math
import os

import numpy as np
import pytest

import oracle
from paper_2001_06784_gb300 import graphgen
from tests import graphs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pvt():
    import torch  # noqa: F401

    import paper_2001_06784_gb300 as p
    return p


def gpu_dag(pvt, rp, col, validate=True):
    import torch
    dev = torch.device("cuda:0")
    col32 = np.ascontiguousarray(col, dtype=np.uint32).view(np.int32)
    return pvt.orient(torch.from_numpy(np.ascontiguousarray(rp)).to(dev), torch.from_numpy(col32).to(dev),
                      validate=validate)


def check_all(pvt, rp, col, vertex=True, edge=True, kmax=None):
    ref = oracle.count(rp, col, vertex=vertex, edge=edge, kmax=-1 if kmax is None else kmax)
    dag = gpu_dag(pvt, rp, col)
    K = ref["kmax"]
    assert pvt.to_ints(dag.count_global(kmax=K)) == ref["C"]
    if vertex:
        assert pvt.to_ints(dag.count_local_vertex(kmax=K)) == oracle.to_int(ref["cv"])
    if edge:
        got = pvt.to_ints(dag.count_local_edge(kmax=K))
        assert got == oracle.to_int(ref["ce"])
    dag.free()
    return ref


def exact_column_sums(t):
    """Exact sum over rows of a word table [rows, K, W] (uint64 words), as
    K Python ints: 32-bit halves summed in uint64 cannot wrap below 2^32 rows."""
    t = np.asarray(t, dtype=np.uint64)
    lo = (t & np.uint64(0xFFFFFFFF)).sum(axis=0, dtype=np.uint64)
    hi = (t >> np.uint64(32)).sum(axis=0, dtype=np.uint64)
    out = []
    for k in range(t.shape[1]):
        out.append(sum((int(lo[k, w]) + (int(hi[k, w]) << 32)) << (64 * w) for w in range(t.shape[2])))
    return out


SMALL = {
    "K1": lambda: graphs.complete(1),
    "K2": lambda: graphs.complete(2),
    "empty5": lambda: graphgen.from_edges(5, np.zeros((0, 2), dtype=np.int64)),
    "K5": lambda: graphs.complete(5),
    "K32": lambda: graphs.complete(33),          # alpha = 32: top of the 1-word class
    "K34": lambda: graphs.complete(34),          # alpha = 33: 2-word class
    "cliques": lambda: graphs.disjoint_cliques([3, 5, 7, 4, 1, 2, 12]),
    "multipartite": lambda: graphs.multipartite([3, 3, 3, 3, 2, 1]),
    "K50-star": lambda: graphs.clique_minus_star(50, 7, 9),
    "gnp40": lambda: graphs.gnp(40, 0.35, 1),
    "gnp70": lambda: graphs.gnp(70, 0.25, 2),
    "gnp33": lambda: graphs.gnp(33, 0.6, 3),
    "er-planted": lambda: graphgen.generate(500, er_avg_deg=8.0, planted=[(3, 10, 25, 1.0), (2, 30, 45, 0.9)],
                                            seed=11),
}


@pytest.mark.parametrize("name", sorted(SMALL))
def test_small_all_counts(pvt, name):
    rp, col = SMALL[name]()
    check_all(pvt, rp, col)


@pytest.mark.parametrize("n", [70, 100, 130, 200, 257, 300])
def test_wide_cliques_global_vertex(pvt, n):
    # alpha = n-1 covers the 3-, 4-, 5-word... classes; counts are C(n, k)
    rp, col = graphs.complete(n)
    ref = check_all(pvt, rp, col, edge=False)
    assert ref["C"][1:] == [math.comb(n, k) for k in range(1, n + 1)]


@pytest.mark.parametrize("n,centre,k", [(100, 10, 20), (180, 3, 60), (260, 100, 40)])
def test_wide_branching_global(pvt, n, centre, k):
    rp, col = graphs.clique_minus_star(n, centre, k)
    check_all(pvt, rp, col, vertex=True, edge=False)


@pytest.mark.parametrize("n,missing,vertex", [(90, 25, True), (110, 20, True), (200, 16, True), (300, 14, False),
                                               (500, 10, False)])
def test_wide_branching_random(pvt, n, missing, vertex):
    # wide roots (out-degree classes up to <=512) with real branching below them
    rp, col = graphs.clique_minus_random(n, missing, 1)
    check_all(pvt, rp, col, vertex=vertex, edge=False)


@pytest.mark.parametrize("make", [lambda: graphs.clique_minus_random(520, 4, 3), lambda: graphs.complete(530)])
def test_widest_class_global(pvt, make):
    # out-degrees above 512: 32-word bitsets with the DFS stack in global memory
    rp, col = make()
    ref = check_all(pvt, rp, col, vertex=False, edge=False)
    assert ref["alpha"] > 512


def limbs_as_words(limbs, W):
    """Oracle limb array [..., nl] (32-bit, least significant first) as the
    library's layout [..., W] of 64-bit words (higher limbs must be 0)."""
    a = np.asarray(limbs, dtype=np.uint64)
    if a.shape[-1] > 2 * W:
        assert not a[..., 2 * W:].any(), "count wider than W words"
        a = a[..., :2 * W]
    pad = np.zeros(a.shape[:-1] + (2 * W,), dtype=np.uint64)
    pad[..., :a.shape[-1]] = a
    return pad[..., 0::2] | (pad[..., 1::2] << np.uint64(32))


# Per-vertex and per-edge tables of roots in every wide out-degree class,
# element by element against the oracle (Alg. 2 steps ht/pt and
# hht/pht/ppt).  K_n without a few random edges keeps the tree small while
# the roots' out-degrees sweep every class up to n - 2; (name, n, missing
# edges, kmax of the vertex table, kmax of the edge table; -1 = every k).
# Where the full per-edge table would not fit a test (m x (n+1) x W words),
# the edge table is truncated at kmax (Sec. 4): entries k <= kmax are exact.
LOCAL_CLASSES = [("65..128", 90, 12, -1, -1), ("129..256", 140, 10, -1, -1), ("257..512", 270, 6, -1, -1),
                 ("257..512 branching", 300, 14, 6, 6), ("513..1024", 520, 8, -1, 6)]


@pytest.fixture(scope="module")
def local_refs():
    """Oracle tables of every LOCAL_CLASSES case, computed on host threads
    in parallel (the oracle's C code runs outside the interpreter lock)."""
    import concurrent.futures as cf

    def one(case):
        _, n, miss, kv, ke = case
        rp, col = graphs.clique_minus_random(n, miss, 1)
        return (rp, col, oracle.count(rp, col, vertex=True, kmax=kv), oracle.count(rp, col, edge=True, kmax=ke))

    with cf.ThreadPoolExecutor(max_workers=len(LOCAL_CLASSES)) as ex:
        return dict(zip([c[0] for c in LOCAL_CLASSES], ex.map(one, LOCAL_CLASSES)))


@pytest.mark.parametrize("case", LOCAL_CLASSES, ids=[c[0] for c in LOCAL_CLASSES])
def test_local_tables_every_class(pvt, local_refs, case):
    name, n = case[0], case[1]
    rp, col, rv, re_ = local_refs[name]
    dag = gpu_dag(pvt, rp, col)
    assert dag.alpha == rv["alpha"] and dag.alpha >= n - 1 - case[2]
    lo = {"65..128": 65, "129..256": 129, "257..512": 257, "257..512 branching": 257, "513..1024": 513}[name]
    assert dag.alpha >= lo
    W = dag.min_words
    cv = dag.count_local_vertex(kmax=rv["kmax"]).cpu().numpy().view(np.uint64)
    assert np.array_equal(cv, limbs_as_words(rv["cv"], W)), "per-vertex table differs from the oracle"
    del cv
    ce = dag.count_local_edge(kmax=re_["kmax"]).cpu().numpy().view(np.uint64)
    assert np.array_equal(ce, limbs_as_words(re_["ce"], W)), "per-edge table differs from the oracle"
    del ce
    # the global counts of the same graph, as a cross-check of the tables' k range
    assert pvt.to_ints(dag.count_global(kmax=rv["kmax"])) == rv["C"]
    dag.free()


@pytest.mark.parametrize("kmax", [0, 1, 2, 3, 5, 9])
def test_truncation(pvt, kmax):
    rp, col = graphgen.generate(400, er_avg_deg=10.0, planted=[(2, 15, 25, 1.0)], seed=3)
    check_all(pvt, rp, col, kmax=kmax)


def test_extra_words_are_zero(pvt):
    rp, col = graphs.complete(40)
    dag = gpu_dag(pvt, rp, col)
    W = dag.min_words + 2
    C = dag.count_global(W=W).cpu().numpy().view(np.uint64)
    assert (C[:, dag.min_words:] == 0).all()
    assert pvt.to_ints(C) == [0] + [math.comb(40, k) for k in range(1, 41)]  # kmax = alpha + 1 = 40


def test_workload_er2k_all(pvt):
    rp, col = graphgen.workload("er2k_d20_clique30")
    check_all(pvt, rp, col)


def test_repeat_calls_identical(pvt):
    rp, col = graphgen.generate(3000, er_avg_deg=15.0, planted=[(5, 20, 40, 0.95)], seed=9)
    dag = gpu_dag(pvt, rp, col)
    a = pvt.to_ints(dag.count_global())
    b = pvt.to_ints(dag.count_global())
    v1 = dag.count_local_vertex().cpu().numpy()
    v2 = dag.count_local_vertex().cpu().numpy()
    assert a == b and (v1 == v2).all()


@pytest.mark.parametrize("make", [lambda: graphgen.generate(3000, er_avg_deg=12.0, planted=[(6, 20, 70, 0.9)], seed=13),
                                  lambda: graphs.clique_minus_random(200, 16, 2)])
def test_policies_agree(pvt, make):
    """Plain (one warp per root) and persistent (work queue, split subtrees)
    forms, with one-word labels walked per warp or per lane and the classes
    above 128 walked a warp or a block per root, give identical words and
    walk the same tree, and all match the oracle."""
    rp, col = make()
    ref = oracle.count(rp, col)
    dag = gpu_dag(pvt, rp, col)
    out = {}
    nosplit, mixed = (0,) * 7, (0, 0, 1, 0, 1, 0, 1)
    walked = {}
    nocta, allcta = (0,) * 7, (0, 0, 0, 0, 1, 1, 1)
    for form in [(True, 4, None, True, True, None), (False, 1, None, False, True, None),
                 (True, 1, nosplit, True, True, nocta), (True, 32, mixed, True, True, allcta),
                 (True, 4, None, False, True, allcta), (True, 1, nosplit, False, True, None),
                 (True, 4, None, True, False, nocta), (True, 1, nosplit, True, False, allcta),
                 (True, 4, None, False, False, nocta)]:
        persistent, chunk, split, frames, lanes, cta = form
        dag.set_policy(persistent=persistent, chunk=chunk, split=split, frames=frames, lanes=lanes, cta=cta)
        out[form] = pvt.to_ints(dag.count_global(kmax=ref["kmax"]))
        st = dag.stats()
        # the same tree whichever kernels walk it
        walked[form] = (st["sct_nodes"], st["sct_leaves"], st["pivot_words"])
        assert sum(st["class_words"]) + st["frame_words"] == st["pivot_words"]
        if not (persistent and frames):
            assert st["frame_words"] == 0 and st["frames"] == 0
    assert all(v == ref["C"] for v in out.values())
    assert len(set(walked.values())) == 1
    dag.free()


@pytest.mark.parametrize("make", [lambda: graphgen.workload("er2k_d20_clique30"),
                                  lambda: graphs.clique_minus_random(300, 14, 7)])
def test_graph_replay_and_autotune(pvt, make):
    """Global counts replayed from a recorded CUDA graph equal the direct
    launches (three replays, a new recording when kmax or the output
    changes); the autotuner returns a valid policy and exact counts."""
    import torch
    rp, col = make()
    ref = oracle.count(rp, col)
    K = ref["kmax"]
    dag = gpu_dag(pvt, rp, col)
    dag.count_global(kmax=K)  # sizes the scratch and the Pascal table
    direct = pvt.to_ints(dag.count_global(kmax=K))
    launches = dag.stats()["launches"]
    dag.set_policy(graph=True)
    assert dag.policy()["graph"]
    out = torch.empty((K + 1, dag.min_words), dtype=torch.int64, device="cuda:0")
    for i in range(4):  # the first call launches directly and records; the rest replay
        out.fill_(-1)
        dag.count_global(kmax=K, out=out)
        assert pvt.to_ints(out) == ref["C"] == direct, i
        assert dag.stats()["launches"] == launches
    assert pvt.to_ints(dag.count_global(kmax=K - 1)) == ref["C"][:K]
    assert pvt.to_ints(dag.count_global(kmax=K)) == ref["C"]
    pol, ms, C = dag.autotune(kmax=K)
    assert pvt.to_ints(C) == ref["C"]
    assert pol == dag.policy() and pol["graph"] and pol["chunk"] in (1, 4, 16)
    assert all(x in (0, 1) for x in pol["split"]) and pol["split"][:2] == [0, 0]
    assert ms.shape == (3, 7) and (ms >= 0).all() and ms[:, 1:].sum() > 0
    for _ in range(2):
        assert pvt.to_ints(dag.count_global(kmax=K)) == ref["C"]
    with pytest.raises(pvt.PivoterError):
        dag.set_policy(split=[2] * 7)
    dag.free()


# ------------------------------------------------------------ full sizes

@pytest.mark.parametrize("name", ["cl1m_m10m_b2.1_comm500", "cl500k_m8m_b2.3_clq200"])
def test_workload_full_global(pvt, name):
    """Full-size global counts vs the root-parallel oracle on every host core."""
    rp, col = graphgen.workload(name)
    ref = oracle.count(rp, col, threads=os.cpu_count() or 1)
    dag = gpu_dag(pvt, rp, col, validate=True)
    assert dag.alpha <= ref["alpha"] + 0  # both are degeneracies of the same graph
    got = pvt.to_ints(dag.count_global(kmax=ref["kmax"]))
    assert got == ref["C"]
    n, m = len(rp) - 1, len(col) // 2
    assert got[1] == n and got[2] == m


def test_measure_popc_rate(pvt):
    """The measured AND+POPC+ADD ceiling (the walk roofline's peak) is
    positive, below 32 triples per SM per clock at 2.2 GHz, and repeatable."""
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    a, b = pvt.measure_popc_rate("cuda:0"), pvt.measure_popc_rate("cuda:0")
    assert 0 < a < 32 * sms * 2.2e9 and 0 < b < 32 * sms * 2.2e9
    assert abs(a - b) <= 0.1 * max(a, b)


def test_workload_cl3m_truncated(pvt):
    """The 128M-edge com-orkut-shaped graph (degeneracy 733), truncated to
    k <= 3 (Sec. 4, counting for a specific k): its all-k tree (about 1.6e12
    nodes) is far beyond the oracle, but C_1 = n, C_2 = m and C_3 equals the
    oracle's triangle enumeration, at full size, word for word."""
    rp, col = graphgen.workload("cl3m_m117m_b2.0_comm2000")
    n, m = len(rp) - 1, len(col) // 2
    T = oracle.triangles(rp, col, threads=os.cpu_count() or 1)
    dag = gpu_dag(pvt, rp, col, validate=False)
    assert dag.alpha == 733
    C = pvt.to_ints(dag.count_global(kmax=3))
    assert C == [0, n, m, T]
    dag.free()


@pytest.mark.parametrize("make", [
    lambda: graphs.complete(40), lambda: graphs.multipartite([3, 5, 7, 2]), lambda: graphs.gnp(300, 0.1, 3),
    lambda: graphgen.from_edges(5, []), lambda: graphs.disjoint_cliques([1, 2, 33, 70]),
    lambda: graphgen.workload("er2k_d20_clique30"), lambda: graphgen.workload("cl1m_m10m_b2.1_comm500"),
    lambda: graphgen.workload("cl500k_m8m_b2.3_clq200"),
    # mid-size graphs: a few grid levels, then the one-block finish
    lambda: graphgen.generate(60000, chung_lu=(400000, 2.2), seed=11),
    lambda: graphgen.generate(200000, er_avg_deg=9, planted=[(50, 20, 60, 0.7)], seed=12)])
def test_core_numbers(pvt, make):
    """Core numbers of the device peel equal the oracle's (sequential bucket
    peel): they do not depend on the removal order within a level, so the
    comparison is exact; the reported alpha is the largest of them.  The
    orientation is a degeneracy order: every vertex has at most core(v)
    later neighbours (Sec. 3.2), and every edge is oriented once."""
    rp, col = make()
    _, core, _ = oracle.orient(rp, col)
    dag = gpu_dag(pvt, rp, col)
    got = dag.cores().cpu().numpy().view(np.uint32)
    assert np.array_equal(got, core)
    assert dag.alpha == (int(core.max()) if len(core) else 0)
    orow, _ = dag.out_lists()
    outdeg = np.diff(orow.cpu().numpy())
    assert outdeg.sum() == len(col) // 2
    assert (outdeg <= core.astype(np.int64)).all()
    dag.free()


def test_workload_local_sampled(pvt):
    """Per-vertex / per-edge tables at full size (500k vertices, 8M edges),
    checked on sampled rows one by one: c_k(v) = C_{k-1} of the subgraph
    induced on N(v), c_k(uv) = C_{k-2} of the subgraph on N(u) & N(v)
    (definitions, Sec. 3.1), plus the identities sum_v c_k(v) = k C_k and
    sum_e c_k(e) = C(k,2) C_k against the GPU's own global counts."""
    rp, col = graphgen.workload("cl500k_m8m_b2.3_clq200")
    n, m = len(rp) - 1, len(col) // 2
    dag = gpu_dag(pvt, rp, col)
    C = pvt.to_ints(dag.count_global())
    K = max(k for k, c in enumerate(C) if c)  # clique number: every nonzero count
    C = C[:K + 1]
    cv = dag.count_local_vertex(kmax=K).cpu().numpy().view(np.uint64)
    rng = np.random.default_rng(0)
    deg = np.diff(rp)
    sample = list(rng.choice(n, 40, replace=False)) + list(np.argsort(deg)[-5:])
    for v in sample:
        nb = col[rp[v]:rp[v + 1]].astype(np.int64)
        srp, scol = graphgen.induced_subgraph(rp, col, nb)
        sub = oracle.count(srp, scol, kmax=K - 1)["C"] if len(nb) else [0] * K
        sub[0] = 1  # the empty clique extends to {v}
        assert pvt.to_ints(cv[v]) == [0] + sub[:K], f"vertex {v}"
    # identity: sum_v c_k(v) = k * C_k, in exact integers
    assert exact_column_sums(cv) == [k * C[k] for k in range(K + 1)]
    del cv
    ce = dag.count_local_edge(kmax=K).cpu().numpy().view(np.uint64)
    edges = graphgen.edge_list(rp, col)
    for e in rng.choice(m, 30, replace=False):
        u, v = edges[e]
        common = np.intersect1d(col[rp[u]:rp[u + 1]], col[rp[v]:rp[v + 1]]).astype(np.int64)
        if len(common):
            srp, scol = graphgen.induced_subgraph(rp, col, common)
            sub = oracle.count(srp, scol, kmax=max(K - 2, 0))["C"]
        else:
            sub = [0] * (K - 1)
        sub[0] = 1
        assert pvt.to_ints(ce[e]) == [0, 0] + sub[:K - 1], f"edge {e}"
    assert exact_column_sums(ce) == [math.comb(k, 2) * C[k] for k in range(K + 1)]


# ---------------------------------------------------------------- errors

def test_errors(pvt):
    import torch
    rp, col = graphs.complete(10)
    dag = gpu_dag(pvt, rp, col)
    with pytest.raises(pvt.PivoterError) as ei:
        dag.count_global(W=0)
    assert ei.value.status == 1
    with pytest.raises(pvt.PivoterError) as ei:
        dag.count_global(kmax=-1)
    assert ei.value.status == 1
    big_rp, big_col = graphs.complete(70)  # alpha 69: needs 2 words
    dag2 = gpu_dag(pvt, big_rp, big_col)
    with pytest.raises(pvt.PivoterError) as ei:
        dag2.count_global(W=1)
    assert ei.value.status == 4
    # an asymmetric CSR is refused by validation (all indices in range)
    bad_rp = np.array([0, 2, 3, 4], dtype=np.int64)
    bad_col = np.array([1, 2, 0, 1], dtype=np.uint32)  # 0->2 present, 2->0 missing
    with pytest.raises(pvt.PivoterError) as ei:
        gpu_dag(pvt, bad_rp, bad_col, validate=True)
    assert ei.value.status == 2
    # self-loops, an unsorted row (even nnz, indices in range)
    for rp2, col2 in [(np.array([0, 2, 4], np.int64), np.array([0, 1, 0, 1], np.uint32)),
                      (np.array([0, 2, 3, 4], np.int64), np.array([2, 1, 0, 0], np.uint32))]:
        with pytest.raises(pvt.PivoterError) as ei:
            gpu_dag(pvt, rp2, col2, validate=True)
        assert ei.value.status == 2
    # the library stays usable afterwards
    assert pvt.to_ints(dag.count_global())[3] == math.comb(10, 3)
    torch.cuda.synchronize()


# ------------------------------------------------ root ranges, checkpoints

@pytest.mark.parametrize("make", [lambda: graphgen.workload("er2k_d20_clique30"),
                                  lambda: graphs.clique_minus_random(300, 14, 7),
                                  lambda: graphgen.generate(3000, er_avg_deg=12.0, planted=[(6, 20, 70, 0.9)], seed=13),
                                  lambda: graphgen.workload("cl500k_m8m_b2.3_clq200")])
def test_root_ranges_checkpoint(pvt, make):
    """Histograms of disjoint root ranges add up to the whole count: walk
    [0, n) in uneven pieces, passing the histogram through host memory
    between pieces (a checkpoint), combine once; equals the oracle and the
    one-call global count, word for word.  An empty range changes nothing."""
    import torch
    rp, col = make()
    n = len(rp) - 1
    ref = oracle.count(rp, col, threads=os.cpu_count() or 1)
    K = ref["kmax"]
    dag = gpu_dag(pvt, rp, col)
    cuts = sorted({0, n, n // 7, n // 3, (2 * n) // 3, n - 1})
    hist = None
    for a, b in zip(cuts[:-1], cuts[1:]):
        hist = dag.count_hist(a, b, hist=hist, kmax=K)
        hist = hist.cpu().to("cuda:0")  # checkpoint round trip
    before = hist.clone()
    dag.count_hist(5, 5, hist=hist, kmax=K)
    assert torch.equal(before, hist)
    assert pvt.to_ints(dag.combine_hist(hist, kmax=K)) == ref["C"]
    assert pvt.to_ints(dag.count_global(kmax=K)) == ref["C"]
    # one call over [0, n) gives the same histogram
    assert torch.equal(dag.count_hist(0, n, kmax=K), hist)
    with pytest.raises(pvt.PivoterError):
        dag.count_hist(3, 2, kmax=K)
    dag.free()


# ------------------------------------------------ SCT statistics, leaf depths

@pytest.mark.parametrize("make", [lambda: graphs.complete(40), lambda: graphgen.workload("er2k_d20_clique30"),
                                  lambda: graphs.clique_minus_random(300, 14, 7),
                                  lambda: graphgen.generate(3000, er_avg_deg=12.0, planted=[(6, 20, 70, 0.9)], seed=13)])
def test_sct_statistics_match_oracle(pvt, make):
    """The tree the device walks is the oracle's SCT (Alg. 1) under the
    device's own orientation: the same (h, p) leaf histogram, the same leaves,
    leaf depths h + p, and nodes = the oracle's nodes minus the pivot chains
    below clique labels (the device closes a clique label as one leaf).  The
    oracle walks the out-lists the device exports, so both sides walk the
    same roots' children."""
    rp, col = make()
    dag = gpu_dag(pvt, rp, col)
    orow, ocol = dag.out_lists()
    orow_h, ocol_h = orow.cpu().numpy(), ocol.cpu().numpy().view(np.uint32)
    assert orow_h[-1] == dag.m and int(np.diff(orow_h).max()) == dag.alpha
    H = dag.alpha + 2
    ref = oracle.count(rp, col, dag=(orow_h, ocol_h), hist_dim=H)
    assert ref["alpha"] == dag.alpha
    assert pvt.to_ints(dag.count_global(kmax=ref["kmax"])) == ref["C"]
    st = dag.stats()
    assert st["sct_leaves"] == ref["leaves"]
    assert st["sct_nodes"] == ref["nodes"] - ref["chain"]
    depths = dag.leaf_depths()
    want = np.zeros(H, dtype=np.uint64)
    for h in range(H):
        for p in range(H - h):
            want[h + p] += ref["hist"][h, p]
    assert np.array_equal(depths, want) and int(depths.sum()) == ref["leaves"]
    hist = dag.count_hist(0, dag.n, kmax=ref["kmax"]).cpu().numpy().view(np.uint64)
    assert np.array_equal(hist, ref["hist"])
    dag.free()


def test_leaf_depths_need_a_global_count(pvt):
    rp, col = graphs.complete(6)
    dag = gpu_dag(pvt, rp, col)
    with pytest.raises(pvt.PivoterError) as ei:
        dag.leaf_depths()
    assert ei.value.status == 1
    dag.count_global()
    assert list(dag.leaf_depths()) == [0, 1, 1, 1, 1, 1, 1]  # root r: one leaf of depth 6 - r
    dag.free()


# ------------------------------------------------ failure detection

def test_device_wait_expiry_returns_timeout(pvt):
    """A bounded device-side wait that runs out ends the call with
    PVT_ETIMEOUT and leaves the library usable.  K_258 puts one root in the
    257..512 out-degree class, whose split launch has two warps: the second
    waits for a donated frame while the first gathers 257 adjacency rows,
    far longer than the 1 us limit set here, so the wait expires."""
    rp, col = graphs.complete(258)
    dag = gpu_dag(pvt, rp, col)
    dag.set_policy(wait_limit_us=1)
    assert dag.policy()["wait_limit_us"] == 1
    with pytest.raises(pvt.PivoterError) as ei:
        dag.count_global(kmax=8)
    assert ei.value.status == 6 and "timed out" in str(ei.value)
    dag.set_policy()
    assert pvt.to_ints(dag.count_global(kmax=8)) == [0] + [math.comb(258, k) for k in range(1, 9)]
    with pytest.raises(pvt.PivoterError):
        dag.set_policy(wait_limit_us=-1)
    dag.free()
