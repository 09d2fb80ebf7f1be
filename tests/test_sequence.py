"""Integer pins of the paper's swap sequence and its parallel split (no GPU).

Pins: the worked examples of Sec. 2 and Sec. 3 (golden fixtures), the length
identity of Sec. 3 / Sec. 5, the runtime closed form of Sec. 5, the optimality
property of Sec. 4 (each transposition creates one new prefix set) and
exactly-once coverage of every family, checked by brute force.
"""
import math
import os
from collections import Counter
from itertools import combinations

import pytest

from oracle import sequence as seq

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
LETTERS = "ABCD"


def _read(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return [ln.split("#")[0].strip() for ln in f if ln.split("#")[0].strip()]


def test_three_variable_example():
    lines = _read("sequence_m3.txt")
    orders = [[LETTERS.index(ch) for ch in ln] for ln in lines[:5]]
    swaps = [int(t) for t in lines[5].split()[1:]]
    assert seq.greedy_swaps(3) == swaps
    assert seq.apply_swaps([0, 1, 2], swaps) == orders
    models = set()
    for ln in lines[6:]:
        par, child = ln.split(">")
        models.add((LETTERS.index(child), frozenset(LETTERS.index(p) for p in par)))
    got = set()
    for o in orders:
        got.update(f for f in seq.families_of_ordering(o) if f[1])
    assert got == models and len(models) == 9


def test_four_variable_listing():
    rows = [ln.split() for ln in _read("sequence_m4.txt")]
    orders = [[LETTERS.index(ch) for ch in r[0]] for r in rows]
    printed = [int(r[1]) for r in rows]
    sw = seq.greedy_swaps(4)
    assert len(sw) == 11
    assert seq.apply_swaps([0, 1, 2, 3], sw) == orders
    # cumulative count of distinct non-empty-parent models after each step
    seen = set()
    counts = []
    for o in orders:
        seen.update(f for f in seq.families_of_ordering(o) if f[1])
        counts.append(len(seen))
    diffs = [i for i, (a, b) in enumerate(zip(counts, printed)) if a != b]
    assert diffs == [10] and counts[10] == 27 and printed[10] == 26
    assert counts[-1] == 4 * (2 ** 3 - 1)


@pytest.mark.parametrize("m", range(2, 17))
def test_length_identity(m):
    sw = seq.greedy_swaps(m)
    assert len(sw) == 2 ** m - m - 1
    if m > 2:
        assert len(sw) == 2 * len(seq.greedy_swaps(m - 1)) + m - 1
    assert min(sw) == 1 and max(sw) == m - 1


@pytest.mark.parametrize("m", list(range(2, 21)) + [26])
def test_runtime_closed_form(m):
    assert seq.grc_flops(m, seq.greedy_swaps(m)) == seq.runtime_closed_form(m)


def test_runtime_m26_value():
    assert seq.runtime_closed_form(26) == 5_637_142_308


@pytest.mark.parametrize("m", range(2, 13))
def test_each_swap_creates_a_new_prefix_set(m):
    """Sec. 4: the walk is optimal, so every transposition adds a new prefix set."""
    sw = seq.greedy_swaps(m)
    orders = seq.apply_swaps(list(range(m)), sw)
    prefixes = {frozenset(orders[0][:a]) for a in range(m + 1)}
    per_index = Counter()
    for i, o in zip(sw, orders[1:]):
        p = frozenset(o[:i])
        assert p not in prefixes
        prefixes.add(p)
        per_index[i] += 1
    assert len(prefixes) == 2 ** m
    for i in range(1, m):
        assert per_index[i] == math.comb(m, i) - 1


@pytest.mark.parametrize("m", range(2, 11))
def test_walk_covers_every_family_exactly_once(m):
    fams = seq.walk_families(list(range(m)), seq.greedy_swaps(m))
    c = Counter(fams)
    assert len(fams) == m * 2 ** (m - 1)
    assert set(c) == set(seq.all_families(m))
    assert max(c.values()) == 1


def test_initial_qrd_family_count():
    """Sec. 2: the initial QRD solves m(m-1)/2 models with a non-empty parent set."""
    for m in range(2, 12):
        fams = seq.families_of_ordering(list(range(m)))
        assert sum(1 for f in fams if f[1]) == m * (m - 1) // 2


@pytest.mark.parametrize("m,k", [(4, 1), (6, 1), (6, 2), (7, 3), (8, 2), (8, 5), (9, 4)])
def test_corrected_split_exactly_once(m, k):
    fams = seq.split_families(m, k)
    c = Counter(fams)
    assert len(fams) == m * 2 ** (m - 1)
    assert set(c) == set(seq.all_families(m))
    assert max(c.values()) == 1


def test_literal_split_reading_misses_prefix_sets():
    """The printed Algorithm 2 (0 bit -> front, d = number of 1 bits) leaves gaps."""
    m, k = 6, 1
    q = m - k
    prefixes = set()
    for p in range(1 << k):
        bits = [(p >> b) & 1 for b in range(k)]
        ups = list(range(1, q + 1))
        for i in range(q + 1, m + 1):
            if bits[m - i] == 0:
                ups.insert(0, i)
            else:
                ups.append(i)
        d = sum(bits)
        order = [v - 1 for v in ups]
        orders = seq.apply_swaps(order, [d + s for s in seq.greedy_swaps(q)])
        prefixes.update(frozenset(orders[0][:a]) for a in range(m + 1))
        for i, o in zip([d + s for s in seq.greedy_swaps(q)], orders[1:]):
            prefixes.add(frozenset(o[:i]))
    assert len(prefixes) < 2 ** m


def test_split_swap_counts():
    """Sec. 6: each of the 2^k processors performs 2^(m-k) - (m-k) - 1 swaps."""
    for m, k in [(8, 3), (10, 4)]:
        for p in range(1 << k):
            bits = [(p >> b) & 1 for b in range(k)]
            _, sw = seq.seed_path(bits, m)
            assert len(sw) == 2 ** (m - k) - (m - k) - 1
            assert min(sw) == sum(bits) + 1 and max(sw) == sum(bits) + m - k - 1


@pytest.mark.parametrize("m", range(2, 17))
def test_consecutive_swaps_are_adjacent(m):
    """Upsilon(m) starts at index 1, ends at m-1 and moves by exactly one per step.

    Induction on the recursion of Sec. 3: Upsilon(m-1) ends at m-2, the chain
    [m-1 .. 1] starts at m-1 and ends at 1, and Upsilon(m-1)+1 starts at 2.
    The CUDA walk relies on this to branch directly between row blocks.
    """
    sw = seq.greedy_swaps(m)
    assert sw[0] == 1 and sw[-1] == m - 1
    assert all(abs(a - b) == 1 for a, b in zip(sw, sw[1:]))


def _blocks_and_chains(Q, H):
    """Upsilon(Q) as the walk's consumers run it: 2^H blocks of Upsilon(Q-H),
    block b shifted by popcount(b), the chain after block b of level L =
    trailing ones of b, [Q-H+L .. 1] shifted by popcount(b >> (L+1))."""
    blk = seq.greedy_swaps(Q - H)
    rows = []
    for b in range(1 << H):
        o = bin(b).count("1")
        rows += [i + o for i in blk]
        if b + 1 == (1 << H):
            break
        L = ((~b) & -(~b)).bit_length() - 1
        oc = bin(b >> (L + 1)).count("1")
        rows += [oc + j for j in range(Q - H + L, 0, -1)]
    return rows


@pytest.mark.parametrize("Q", range(3, 13))
def test_recursion_splits_into_shifted_blocks(Q):
    """Algorithm 1's recursion applied H times: the concatenation of shifted
    blocks and chains is the greedy sequence itself."""
    for H in range(1, Q - 1):
        assert _blocks_and_chains(Q, H) == seq.greedy_swaps(Q)
