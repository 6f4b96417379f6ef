"""Helpers shared by the oracle pin tests and the GPU parity tests (test-only)."""
from __future__ import annotations

import os

import numpy as np

import synth

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def graph_matrix(N, edges, diag=True):
    """Symmetric 0/1-pattern matrix of an undirected graph (plus diagonal)."""
    rows, cols = [], []
    for a, b in edges:
        rows += [a, b]
        cols += [b, a]
    if diag:
        rows += list(range(N))
        cols += list(range(N))
    return synth.csr_from_coo(N, N, np.array(rows, dtype=np.int64), np.array(cols, dtype=np.int64),
                              np.ones(len(rows)))


def read_rcm_golden():
    out = []
    with open(os.path.join(GOLDEN, "rcm_small_graphs.txt")) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            name, N, edges, perm = [t.strip() for t in line.split("|")]
            E = [tuple(int(v) for v in e.split("-")) for e in edges.split(",")]
            out.append((name, int(N), E, np.array([int(t) for t in perm.split()], np.int32)))
    return out


def sym_adjacency(A):
    """Sorted neighbour lists of pattern(A + A^T) without self loops (python sets)."""
    N = A.m
    nb = [set() for _ in range(N)]
    for i in range(N):
        for c in A.col_idx[A.row_ptr[i]:A.row_ptr[i + 1]]:
            c = int(c)
            if c != i:
                nb[i].add(c)
                nb[c].add(i)
    return [sorted(s) for s in nb]


def check_cuthill_mckee_property(A, perm):
    """Independent check that reversed(perm) is a Cuthill-McKee order: every
    component is contiguous and starts at a root; after the root, every vertex w
    sorts strictly after its predecessor by (position of w's earliest-placed
    neighbour, degree, index).  Returns the list of component roots."""
    nb = sym_adjacency(A)
    N = A.m
    order = np.asarray(perm)[::-1]
    pos = np.empty(N, np.int64)
    pos[order] = np.arange(N)
    deg = np.array([len(s) for s in nb])
    roots = []
    prev_key = None
    for k, w in enumerate(order):
        w = int(w)
        earlier = [pos[u] for u in nb[w] if pos[u] < k]
        if not earlier:
            roots.append(w)  # starts a new component: none of its neighbours came before
            prev_key = None
            # all neighbours must come later in the same component
            continue
        key = (min(earlier), int(deg[w]), w)
        if prev_key is not None:
            assert key > prev_key, f"CM order violated at position {k}: {key} after {prev_key}"
        prev_key = key
    return roots


def bfs_ecc(nb, r):
    """Eccentricity of r and its last level (plain BFS on neighbour lists)."""
    dist = {r: 0}
    frontier = [r]
    while True:
        nxt = []
        for u in frontier:
            for w in nb[u]:
                if w not in dist:
                    dist[w] = dist[u] + 1
                    nxt.append(w)
        if not nxt:
            return dist[frontier[0]], sorted(frontier)
        frontier = nxt


def dense_cos(A):
    D = A.to_dense()
    G = D @ D.T
    nrm = np.sqrt(np.diag(G))
    with np.errstate(invalid="ignore", divide="ignore"):
        C = G / np.outer(nrm, nrm)
    return D, C, nrm
