"""Pins of the oracle's directed 2-opt for the ATSP (Sec. III-D): the move
reverses a path, so its gain includes the path's forward cost minus its
backward cost.  Checked on a one-way ring (where only that term makes the
repair worth it), against exact rational gains of every move the search
may take, and through whole decodes (local_search 1 and 2 on kind 1)."""
import itertools
from fractions import Fraction

import numpy as np
import pytest

from helpers import atsp, is_perm, params


def full_out_lists(cost):
    n = cost.shape[0]
    out = np.empty((n, n - 1), np.int32)
    for i in range(n):
        c = cost[i].astype(np.float64).copy()
        c[i] = np.inf
        out[i] = np.lexsort((np.arange(n), c))[:n - 1]
    return out


def dlen(cost, t):
    return sum(Fraction(float(cost[t[q], t[(q + 1) % len(t)]])) for q in range(len(t)))


def exact_gains(cost, t, nbr):
    """Exact gain of every move the search considers (both sides, g1 > 0)."""
    n = len(t)
    pos = {c: p for p, c in enumerate(t)}
    C = lambda u, v: Fraction(float(cost[u, v]))
    out = []
    for a in range(n):
        for side in (0, 1):
            x = t[(pos[a] + 1) % n] if side == 0 else t[(pos[a] - 1) % n]
            cx = C(a, x) if side == 0 else C(x, a)
            for b in nbr[a]:
                b = int(b)
                g1 = cx - C(a, b)
                if g1 <= 0:
                    break
                y = t[(pos[b] + 1) % n] if side == 0 else t[(pos[b] - 1) % n]
                if b == x or y == a:
                    continue
                i0, i1 = (pos[x], pos[b]) if side == 0 else (pos[a], pos[y])
                L = (i1 - i0) % n + 1
                path = [t[(i0 + k) % n] for k in range(L)]
                F = sum(C(path[k], path[k + 1]) for k in range(L - 1))
                R = sum(C(path[k + 1], path[k]) for k in range(L - 1))
                g = g1 + (C(b, y) if side == 0 else C(y, b)) - C(x, y) + F - R
                out.append(g)
    return out


def test_one_way_ring_needs_the_reversal_term(orc):
    """Arcs i -> i+1 cost 1, i+1 -> i cost 10, all others 5.  The tour
    0 1 5 4 3 2 6 7 runs a stretch backwards; reversing it removes 1->5 and
    2->6 (5 each), adds 1->2 and 5->6 (1 each) and turns 30 into 3."""
    n = 8
    cost = np.full((n, n), 5.0, np.float32)
    for i in range(n):
        cost[i, (i + 1) % n] = 1.0
        cost[(i + 1) % n, i] = 10.0
        cost[i, i] = 0.0
    start = np.array([0, 1, 5, 4, 3, 2, 6, 7], np.int32)
    t, moves = orc.two_opt_directed(atsp(cost), full_out_lists(cost), start)
    assert moves == 1
    assert list(t) == list(range(8))
    assert dlen(cost, list(t)) == 8


@pytest.mark.parametrize("seed", range(10))
def test_no_move_left_and_never_longer(orc, seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(5, 11))
    cost = rng.random((n, n)).astype(np.float32)
    np.fill_diagonal(cost, 0)
    nb = full_out_lists(cost)
    start = rng.permutation(n).astype(np.int32)
    t, moves = orc.two_opt_directed(atsp(cost), nb, start)
    assert is_perm(t, n)
    assert dlen(cost, list(t)) <= dlen(cost, list(start))
    # every move the search considers is non-improving, exactly (the search's
    # threshold is 1e-10 and FP64 rounding is far below 1e-9)
    assert max(exact_gains(cost, list(t), nb), default=0) <= Fraction(1, 10 ** 9)
    t2, again = orc.two_opt_directed(atsp(cost), nb, t)
    assert again == 0


def test_decode_atsp_with_directed_two_opt(orc):
    from paper_2601_19041_gb300 import synth
    inst = synth.atsp_instance(7, 60, K=15)
    for ls in (1, 2):
        p = params(m=5, k=10, iterations=4, rho=0.2, degree_target=1, local_search=ls, ls_k=8, seed=2)
        o = orc.Oracle(inst, p).iterate(4)
        nb = o.get("nbr")
        for t in (o.get("ib_tour"), o.get("gb_tour"), o.get("nn_tour")):
            assert is_perm(t, 60)
            _, again = orc.two_opt_directed(inst, nb, t)
            assert again == 0
        assert o.scalars()["L_ib"] == orc.tour_length(inst, o.get("ib_tour"))
    with pytest.raises(ValueError):
        orc.Oracle(inst, params(m=5, k=10, iterations=1, rho=0.2, degree_target=1, local_search=3, ls_k=8))
