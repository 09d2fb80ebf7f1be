"""The slot map of the paired FP32 walk, checked on the host.

A paired block takes the 64 sub-walks of roots CTAs 2c and 2c+1 (W = 5 fixed
variables per CTA lane, fixed variable 5 telling the two CTAs apart); pair
lane l carries the sub-walks with front sets F_x = (c << 6) | (l << 1) and
F_y = F_x | 1.  Items: the Q free variables (both sub-walks), the fixed
variables above 5 outside F (both), variables 1..5 in groups of 16 pair
lanes without the variable in F (both), and variable 0 (x only).  This test
restates that item map in plain Python, together with the map of the
single-sub-walk form (lane l = CTA lane, sub-walk F = (cta << 5) | l), and
checks that both cover every table slot exactly once, that the two forms
write the same slots for each pair of CTAs, and that every two-score store
is 8-byte aligned.  The slot of family (c, S) is c 2^(m-1) + compress(S, c).
"""
import pytest


def _nth_zero_bit(x, nth):
    b = 0
    while True:
        if not (x >> b) & 1:
            if nth == 0:
                return b
            nth -= 1
        b += 1


def _compress(F, v):
    low = (1 << v) - 1
    return (F & low) | ((F >> (v + 1)) << v)


def _single(m, Q, cta):
    """Prefix-0 slot, slot stride and slot count of every (item, lane) of one CTA."""
    k = m - Q
    Fhi = cta << 5
    nu = (k - 5) - bin(cta).count("1")
    out = []
    for it in range(Q + nu + 3):
        for lane in range(32):
            if it < Q:
                j = it
                out.append((((k + j) << (m - 1)) + (Fhi | lane), 1 << k, 1 << (Q - 1)))
                continue
            ell = lane
            if it < Q + nu:
                v = 5 + _nth_zero_bit(cta, it - Q)
            else:
                j = it - Q - nu
                uu, sub = lane // 16, lane % 16
                v = 2 * j + uu
                if v >= 5:
                    continue
                ell = (sub & ((1 << v) - 1)) | ((sub >> v) << (v + 1))
            out.append(((v << (m - 1)) + _compress(Fhi | ell, v), 1 << (k - 1), 1 << Q))
    return out


def _paired(m, Q, pc):
    """(prefix-0 slot of x, stride, count, both) for every (item, pair lane) of one pair."""
    k = m - Q
    nu = (k - 6) - bin(pc).count("1")
    out = []
    for it in range(Q + nu + 3 + 1):
        for lane in range(32):
            pl, both = lane, True
            if it < Q:
                j = it
                Fx = (pc << 6) | (pl << 1)
                out.append((((k + j) << (m - 1)) + Fx, 1 << k, 1 << (Q - 1), True))
                continue
            if it < Q + nu:
                v = 6 + _nth_zero_bit(pc, it - Q)
            elif it < Q + nu + 3:
                j = it - Q - nu
                uu, sub = lane >> 4, lane & 15
                v = 1 + 2 * j + uu
                if v > 5:
                    continue
                b = v - 1
                pl = (sub & ((1 << b) - 1)) | ((sub >> b) << (b + 1))
            else:
                v, both = 0, False
            Fx = (pc << 6) | (pl << 1)
            assert not (Fx >> v) & 1  # x lacks v
            if both:
                assert not ((Fx | 1) >> v) & 1  # and so does y
            out.append(((v << (m - 1)) + _compress(Fx, v), 1 << (k - 1), 1 << Q, both))
    return out


@pytest.mark.parametrize("m,Q", [(11, 5), (12, 6), (13, 7), (14, 4), (16, 6), (17, 7), (19, 8)])
def test_paired_and_single_forms_cover_the_table_alike(m, Q):
    k = m - Q
    n_cta = 1 << (k - 5)
    size = m << (m - 1)
    seen_single, seen_paired = [], []
    for cta in range(n_cta):
        for base, stride, cnt in _single(m, Q, cta):
            seen_single += [base + c * stride for c in range(cnt)]
    for pc in range(n_cta // 2):
        mine = []
        for base, stride, cnt, both in _paired(m, Q, pc):
            for c in range(cnt):
                a = base + c * stride
                if both:
                    assert a % 2 == 0, "8-byte store misaligned"
                    mine += [a, a + 1]
                else:
                    mine.append(a)
        ref = []
        for cta in (2 * pc, 2 * pc + 1):
            for base, stride, cnt in _single(m, Q, cta):
                ref += [base + c * stride for c in range(cnt)]
        assert sorted(mine) == sorted(ref)
        seen_paired += mine
    assert len(seen_single) == len(set(seen_single)) == size
    if n_cta >= 2:
        assert sorted(seen_paired) == sorted(seen_single)
