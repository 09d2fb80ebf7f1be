"""Exact structure search over a local-score table (test infrastructure only).

The downstream use of the all-family scores (Sec. 1 of the paper: structure
learning of a Bayesian network from every child / parent-set score), written
from its definition for checking the CUDA search:

* ``best_parents_by_enumeration``: B[c][U] = min over S subset of U of
  score(c, S), by listing the subsets of every U (small m only);
* ``best_parents``: the same minimum one variable at a time (for each bit, a
  set with the bit takes the minimum of itself and the set without it), the
  textbook subset-minimum recursion, pinned to the enumeration in the tests;
* ``optimal_network``: F[W] = min over c in W of F[W \\ c] + B[c][W \\ c] over
  all subsets W in order of size, then backtracking from the full set;
* ``brute_force_network``: every assignment of parent sets, acyclic ones
  only (m <= 5).

Lower scores are better.  Ties go to the smaller parent set and the smallest
sink, as in the CUDA search.  Tables use the library's layout:
slot c * 2^(m-1) + compress(S, c).
"""
from __future__ import annotations

import itertools

import numpy as np


def expand(comp: int, c: int) -> int:
    """Re-insert a zero bit at position c of a compressed (m-1)-bit mask."""
    return (comp & ((1 << c) - 1)) | ((comp >> c) << (c + 1))


def compress(S: int, c: int) -> int:
    return (S & ((1 << c) - 1)) | ((S >> (c + 1)) << c)


def best_parents_by_enumeration(table, m):
    """(best, argmin) by listing every subset of every candidate set."""
    table = np.asarray(table, np.float64)
    half = 1 << (m - 1)
    best = np.empty(m * half)
    arg = np.empty(m * half, np.int64)
    for c in range(m):
        blk = table[c * half:(c + 1) * half]
        for u in range(half):
            bv, ba = np.inf, -1
            s = u
            subsets = []
            while True:  # every subset of u
                subsets.append(s)
                if s == 0:
                    break
                s = (s - 1) & u
            for s in sorted(subsets):  # smaller masks first; on a tie keep the first seen
                if blk[s] < bv or ba < 0:
                    bv, ba = blk[s], s
            best[c * half + u] = bv
            arg[c * half + u] = ba
    return best, arg


def best_parents(table, m):
    """(best, argmin) by the one-bit-at-a-time subset minimum."""
    half = 1 << (m - 1)
    best = np.array(table, np.float64).reshape(m, half).copy()
    arg = np.tile(np.arange(half, dtype=np.int64), (m, 1))
    for b in range(m - 1):
        idx = np.arange(half)
        hi = idx[(idx >> b) & 1 == 1]
        lo = hi ^ (1 << b)
        take = best[:, lo] <= best[:, hi]  # the subset wins ties
        best[:, hi] = np.where(take, best[:, lo], best[:, hi])
        arg[:, hi] = np.where(take, arg[:, lo], arg[:, hi])
    return best.reshape(-1), arg.reshape(-1)


def optimal_network(table, m, bp=None):
    """(parents, order, total): an optimal DAG's parent bitmask per variable, an ordering of
    the variables with parents first, and its score (FP64 sum of table entries)."""
    half = 1 << (m - 1)
    best, arg = best_parents(table, m) if bp is None else bp
    best = best.reshape(m, half)
    full = (1 << m) - 1
    F = np.full(1 << m, np.inf)
    sink = np.zeros(1 << m, np.int64)
    F[0] = 0.0
    W_all = np.arange(1 << m, dtype=np.int64)
    pop = np.array([bin(int(w)).count("1") for w in range(1 << m)]) if m <= 16 else \
        np.unpackbits(W_all.astype(">u4").view(np.uint8).reshape(-1, 4), axis=1).sum(1)
    for p in range(1, m + 1):
        Ws = W_all[pop == p]
        fb = np.full(len(Ws), np.inf)
        cb = np.zeros(len(Ws), np.int64)
        for c in range(m):  # ascending c with a strict comparison: the smallest sink wins ties
            has = (Ws >> c) & 1 == 1
            U = Ws[has] & ~(1 << c)
            cu = (U & ((1 << c) - 1)) | ((U >> (c + 1)) << c)
            val = F[U] + best[c, cu]
            better = val < fb[has]
            sel = np.flatnonzero(has)[better]
            fb[sel] = val[better]
            cb[sel] = c
        F[Ws] = fb
        sink[Ws] = cb
    parents = [0] * m
    order = [0] * m
    W = full
    for step in range(m - 1, -1, -1):
        c = int(sink[W])
        U = W & ~(1 << c)
        parents[c] = expand(int(arg.reshape(m, half)[c, compress(U, c)]), c)
        order[step] = c
        W = U
    return parents, order, float(F[full])


def is_acyclic(parents, m):
    done = 0
    for _ in range(m):
        progress = False
        for v in range(m):
            if not (done >> v) & 1 and (parents[v] & ~done) == 0:
                done |= 1 << v
                progress = True
        if not progress:
            break
    return done == (1 << m) - 1


def network_score(table, m, parents):
    half = 1 << (m - 1)
    return float(sum(float(table[c * half + compress(parents[c], c)]) for c in range(m)))


def brute_force_network(table, m):
    """(parents, total) minimising the total over every acyclic assignment (m <= 5)."""
    half = 1 << (m - 1)
    best_total, best_par = np.inf, None
    for comps in itertools.product(range(half), repeat=m):
        parents = [expand(comps[c], c) for c in range(m)]
        if not is_acyclic(parents, m):
            continue
        t = sum(float(table[c * half + comps[c]]) for c in range(m))
        if t < best_total:
            best_total, best_par = t, parents
    return best_par, best_total
