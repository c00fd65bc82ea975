"""Small structured test graphs (CSR, numpy) built from edge lists."""
from __future__ import annotations

import itertools

import numpy as np

from paper_2001_06784_gb300 import graphgen


def complete(n):
    return graphgen.from_edges(n, list(itertools.combinations(range(n), 2)))


def disjoint_cliques(sizes):
    edges, base = [], 0
    for a in sizes:
        edges += [(base + i, base + j) for i, j in itertools.combinations(range(a), 2)]
        base += a
    return graphgen.from_edges(base, edges)


def multipartite(parts):
    """Complete multipartite graph K_{a_1,...,a_t}."""
    label = np.concatenate([np.full(a, i) for i, a in enumerate(parts)])
    n = len(label)
    edges = [(u, v) for u, v in itertools.combinations(range(n), 2) if label[u] != label[v]]
    return graphgen.from_edges(n, edges)


def clique_minus_star(n, centre, k):
    """K_n without the k edges (centre, centre+1..centre+k)."""
    gone = {(centre, centre + i) for i in range(1, k + 1)}
    edges = [e for e in itertools.combinations(range(n), 2) if e not in gone]
    return graphgen.from_edges(n, edges)


def clique_minus_random(n, missing, seed):
    """K_n without `missing` random edges: at most 2^missing maximal cliques,
    so the SCT stays small while every root has a wide out-neighbourhood."""
    rng = np.random.default_rng(seed)
    iu = np.triu_indices(n, 1)
    keep = np.ones(len(iu[0]), dtype=bool)
    keep[rng.choice(len(keep), missing, replace=False)] = False
    return graphgen.from_edges(n, np.stack([iu[0][keep], iu[1][keep]], axis=1))


def gnp(n, p, seed):
    rng = np.random.default_rng(seed)
    iu = np.triu_indices(n, 1)
    keep = rng.random(len(iu[0])) < p
    return graphgen.from_edges(n, np.stack([iu[0][keep], iu[1][keep]], axis=1))


def adjacency_sets(row_ptr, col):
    n = len(row_ptr) - 1
    return [set(int(x) for x in col[row_ptr[v]:row_ptr[v + 1]]) for v in range(n)]


def relabel(row_ptr, col, perm):
    """Graph with vertex v renamed perm[v]."""
    e = graphgen.edge_list(row_ptr, col)
    return graphgen.from_edges(len(row_ptr) - 1, perm[e])
