"""Plant plausible mistakes in a copy of the oracle (CPU only) and check that
the pins catch every one: a dropped carry, shifted or wrong binomial rows in
each Alg. 2 update, hold children that keep the earlier non-neighbours, a
directed (instead of undirected) adjacency inside N+(r), the pivot among its
own hold children, and a wrong term in Pascal's rule.  Mutations that the
theory says cannot change counts (another pivot, another acyclic
orientation) are deliberately absent."""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import tempfile

import pytest

import oracle
from paper_2001_06784_gb300 import graphgen
from tests import graphs
from tests.test_oracle_pins import brute_counts

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle", "pivoter_oracle.c")

MUTATIONS = {
    "dropped carry": ("        c >>= 32;\n", "        c = 0;\n"),
    "global row shifted": ("if (w->C) add_row(w, w->C, h, p);", "if (w->C) add_row(w, w->C, h + 1, p);"),
    "hold-vertex binomial": ("add_row(w, w->cv + (size_t)w->H[i] * K * nl, h, p);",
                             "add_row(w, w->cv + (size_t)w->H[i] * K * nl, h, p - 1);"),
    "pivot-vertex offset": ("add_row(w, w->cv + (size_t)w->P[i] * K * nl, h + 1, p - 1);",
                            "add_row(w, w->cv + (size_t)w->P[i] * K * nl, h, p - 1);"),
    "hold-pair binomial": ("add_row(w, w->ce + (size_t)edge_id(g, w->H[i], w->H[j]) * K * nl, h, p);",
                           "add_row(w, w->ce + (size_t)edge_id(g, w->H[i], w->H[j]) * K * nl, h, p - 1);"),
    "pivot-hold pair offset": ("edge_id(g, w->P[i], w->H[j]) * K * nl, h + 1, p - 1);",
                               "edge_id(g, w->P[i], w->H[j]) * K * nl, h + 2, p - 1);"),
    "pivot-pair offset": ("edge_id(g, w->P[i], w->P[j]) * K * nl, h + 2, p - 2);",
                          "edge_id(g, w->P[i], w->P[j]) * K * nl, h + 1, p - 2);"),
    "earlier non-neighbours kept": ("            if (!earlier) idx[cs++] = j;", "            idx[cs++] = j;"),
    "directed adjacency in N+(r)": ("(uint8_t)(i != j && is_adj(g, v[i], v[j]))",
                                    "(uint8_t)(i < j && is_adj(g, v[i], v[j]))"),
    "pivot among hold children": ("if (j != pi && !A[(size_t)pi * s + j]) R[r++] = j;",
                                  "if (!A[(size_t)pi * s + j] && (j != pi || 1)) R[r++] = j;"),
    "pascal term": ("big_add(row + (size_t)b * nl, prev + (size_t)b * nl, nl, ovf);",
                    "big_add(row + (size_t)b * nl, prev + (size_t)(b - 1) * nl, nl, ovf);"),
    # root-parallel mode (Sec. 4, "Parallel version"): a chunk that ends one
    # root short, and a thread's private counts left out of the final sum
    "root chunk end short": ("int64_t i1 = i0 + 16 < k->nroots ? i0 + 16 : k->nroots;",
                             "int64_t i1 = i0 + 15 < k->nroots ? i0 + 15 : k->nroots;"),
    "thread counts not merged": ("if (C && w->C)\n", "if (C && w->C && t == 0)\n"),
}


def pins_pass() -> bool:
    """A fast subset of the pins; False as soon as one fails."""
    try:
        for n in (4, 7, 40):
            rp, col = graphs.complete(n)
            r = oracle.count(rp, col, vertex=True, edge=n <= 7)
            K = r["kmax"]
            if r["C"] != [0] + [math.comb(n, k) for k in range(1, K + 1)]:
                return False
            if oracle.to_int(r["cv"])[0] != [0] + [math.comb(n - 1, k - 1) for k in range(1, K + 1)]:
                return False
        for make in (lambda: graphs.gnp(20, 0.5, 1), lambda: graphs.gnp(16, 0.7, 2),
                     lambda: graphgen.generate(30, er_avg_deg=6.0, planted=[(1, 9, 9, 1.0)], seed=3)):
            rp, col = make()
            r = oracle.count(rp, col, vertex=True, edge=True)
            C, cv, ce = brute_counts(rp, col, r["kmax"])
            if r["C"] != C or oracle.to_int(r["cv"]) != cv or oracle.to_int(r["ce"]) != ce:
                return False
    except RuntimeError:
        return False
    return threaded_pins_pass()


def threaded_pins_pass() -> bool:
    """The root-parallel oracle against closed forms and the sequential
    oracle: C_1 = n, C_2 = m, sums of C(a, k) over disjoint cliques, and
    t threads equal to one.  Twelve thousand roots in chunks of 16 keep every
    thread busy, so a thread whose counts are dropped changes the sum."""
    sizes = [1, 2, 3, 5, 8, 13, 21, 30]
    rp, col = graphs.disjoint_cliques(sizes)
    for t in (1, 3):
        r = oracle.count(rp, col, threads=t)
        if r["C"] != [0] + [sum(math.comb(a, k) for a in sizes) for k in range(1, r["kmax"] + 1)]:
            return False
    rp, col = graphgen.generate(12021, er_avg_deg=10.0, planted=[(6, 12, 20, 1.0), (1, 25, 25, 0.9)], seed=31)
    n, m = len(rp) - 1, len(col) // 2
    one = oracle.count(rp, col)
    if one["C"][1] != n or one["C"][2] != m:
        return False
    for t in (2, 7):
        if oracle.count(rp, col, threads=t)["C"] != one["C"]:
            return False
    return True


def test_unmutated_oracle_passes():
    assert pins_pass()


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_mutation_is_caught(name, monkeypatch):
    old, new = MUTATIONS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation anchor for {name!r} not unique"
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "mut.c")
        so = os.path.join(d, "libmut.so")
        open(c, "w").write(src.replace(old, new))
        subprocess.check_call(["gcc", "-O1", "-fPIC", "-shared", "-std=c11", "-pthread", c, "-o", so])
        monkeypatch.setattr(oracle, "_lib", oracle.declare(ctypes.CDLL(so)))
        assert not pins_pass(), f"planted mistake {name!r} went unnoticed"


# the SCT-free triangle enumeration has pins of its own
TRI_MUTATIONS = {
    "no orientation filter": ("if (later(rp, (uint32_t)u, col[i])) ocol[k++] = col[i];", "ocol[k++] = col[i];"),
    "marker left set": ("for (int64_t i = k->orow[u]; i < k->orow[u + 1]; ++i) k->mark[k->ocol[i]] = 0;",
                        "(void)0;"),
    "chunk end short": ("const int64_t u1 = u0 + 64 < k->n ? u0 + 64 : k->n;",
                        "const int64_t u1 = u0 + 63 < k->n ? u0 + 63 : k->n;"),
}


def triangle_pins_pass() -> bool:
    """C(n, 3) on complete graphs and trace(A^3)/6 on random graphs, for one
    thread and several; False as soon as one fails."""
    import numpy as np
    for n in (3, 9, 70):
        rp, col = graphs.complete(n)
        if oracle.triangles(rp, col) != math.comb(n, 3) or oracle.triangles(rp, col, threads=3) != math.comb(n, 3):
            return False
    for make in (lambda: graphs.gnp(120, 0.1, 4), lambda: graphgen.workload("er2k_d20_clique30")):
        rp, col = make()
        n = len(rp) - 1
        A = np.zeros((n, n))
        A[np.repeat(np.arange(n), np.diff(rp)), col.astype(np.int64)] = 1.0
        want = int(round(np.einsum("ij,jk,ki->", A, A, A) / 6))
        if oracle.triangles(rp, col) != want or oracle.triangles(rp, col, threads=4) != want:
            return False
    return True


def test_unmutated_triangles_pass():
    assert triangle_pins_pass()


@pytest.mark.parametrize("name", sorted(TRI_MUTATIONS))
def test_triangle_mutation_is_caught(name, monkeypatch):
    old, new = TRI_MUTATIONS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation anchor for {name!r} not unique"
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "mut.c")
        so = os.path.join(d, "libmut.so")
        open(c, "w").write(src.replace(old, new))
        subprocess.check_call(["gcc", "-O1", "-fPIC", "-shared", "-std=c11", "-pthread", c, "-o", so])
        monkeypatch.setattr(oracle, "_lib", oracle.declare(ctypes.CDLL(so)))
        assert not triangle_pins_pass(), f"planted mistake {name!r} went unnoticed"
