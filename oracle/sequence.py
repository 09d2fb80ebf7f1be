"""The paper's integer algorithms, written out for checking (test infrastructure).

All indices follow the paper: positions and swap indices are 1-based, a swap
index i transposes the variables at positions i and i+1 (the GRC_i operator of
Sec. 1.3).  Variables are 0-based integers here.
"""
from __future__ import annotations

from functools import lru_cache
from itertools import combinations
from typing import Iterable, List, Sequence, Tuple


@lru_cache(maxsize=None)
def _greedy(m: int) -> Tuple[int, ...]:
    if m <= 1:
        return ()
    if m == 2:
        return (1,)
    prev = _greedy(m - 1)
    # Algorithm 1: Upsilon(m-1) : [m-1 .. 1] : Upsilon(m-1) shifted by one.
    # The printed listing omits the shift; the recursion stated in Sec. 3 and
    # the recurrence of Sec. 5 both add one to every index of the second copy.
    return prev + tuple(range(m - 1, 0, -1)) + tuple(i + 1 for i in prev)


def greedy_swaps(m: int) -> List[int]:
    """GreedySwaps(m) of Algorithm 1: swap indices, length 2^m - m - 1."""
    return list(_greedy(m))


def apply_swaps(order: Sequence[int], swaps: Iterable[int]) -> List[List[int]]:
    """Every ordering visited: the initial one, then one per GRC_i."""
    cur = list(order)
    out = [list(cur)]
    for i in swaps:
        cur[i - 1], cur[i] = cur[i], cur[i - 1]
        out.append(list(cur))
    return out


def families_of_ordering(order: Sequence[int], prefix_lengths: Iterable[int] | None = None):
    """Families one QRD provides (Sec. 2): child order[j] on parents order[:a], a <= j.

    With prefix_lengths=None every a in 0..m-1 is used (the empty parent set
    included); otherwise only the listed prefix lengths are read out.
    """
    m = len(order)
    lengths = range(m) if prefix_lengths is None else prefix_lengths
    fams = []
    for a in lengths:
        parents = frozenset(order[:a])
        for j in range(a, m):
            fams.append((order[j], parents))
    return fams


def walk_families(order: Sequence[int], swaps: Sequence[int], lo: int = 0, hi: int | None = None):
    """Families read out along a walk with the 'new prefix only' rule.

    The initial QRD contributes prefix lengths lo..hi (default: all); the QRD
    after GRC_i contributes only the prefix of length i, the one prefix set
    that swap creates (Sec. 4: each transposition adds new models only there).
    """
    m = len(order)
    hi = m - 1 if hi is None else hi
    orders = apply_swaps(order, swaps)
    fams = families_of_ordering(orders[0], range(lo, hi + 1))
    for i, o in zip(swaps, orders[1:]):
        fams.extend(families_of_ordering(o, [i]))
    return fams


def seed_path(pid_bits: Sequence[int], m: int):
    """SeedPathCalculator of Algorithm 2, in its corrected reading.

    pid_bits has len(pid_bits) = m - k entries; pid_bits[m - i] decides
    variable i (1-based, i = k+1..m).  Reading: a 1 bit puts the variable at
    the front (it is a parent in every model of that processor), a 0 bit at
    the back; d = sum(pid_bits) is then the number of front variables, which
    is the shift the swap indices need.  (The printed listing tests for 0 and
    runs the loop to n; with that literal reading d counts the back variables
    and the split misses prefix sets.)  Returns (initial ordering as 1-based
    variable labels, swap indices).
    """
    k = m - len(pid_bits)
    upsilon = list(range(1, k + 1))
    for i in range(k + 1, m + 1):
        if pid_bits[m - i] == 1:
            upsilon.insert(0, i)
        else:
            upsilon.append(i)
    d = sum(pid_bits)
    return upsilon, [d + s for s in greedy_swaps(k)]


def split_families(m: int, k_fixed: int):
    """Families read out by all 2^k_fixed processors of the corrected split.

    Ownership: a processor with d front variables reads out its root only for
    prefix lengths d..d+k (the prefix sets whose intersection with the fixed
    variables is exactly its front set) and each swap's new prefix.
    """
    fams = []
    q = m - k_fixed
    for p in range(1 << k_fixed):
        bits = [(p >> b) & 1 for b in range(k_fixed)]
        order1, swaps = seed_path(bits, m)
        order0 = [v - 1 for v in order1]
        d = sum(bits)
        fams.extend(walk_families(order0, swaps, lo=d, hi=min(d + q, m - 1)))
    return fams


def all_families(m: int):
    out = []
    for c in range(m):
        others = [v for v in range(m) if v != c]
        for r in range(m):
            for S in combinations(others, r):
                out.append((c, frozenset(S)))
    return out


def grc_flops(m: int, swaps: Sequence[int]) -> int:
    """Sec. 5 cost model: GRC_i on an m-column R costs 6(m - i + 1) flops."""
    return sum(6 * (m - i + 1) for i in swaps)


def runtime_closed_form(m: int) -> int:
    """T(m) = 3 m 2^m + 6 * 2^m - 3 m^2 - 9 m - 6 (Sec. 5)."""
    return 3 * m * (1 << m) + 6 * (1 << m) - 3 * m * m - 9 * m - 6
