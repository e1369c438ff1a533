"""Pins of the oracle's 3-opt (Sec. III-D): first improvement over sequential
exchanges of up to three edges with neighbour lists and don't-look bits.
With full neighbour lists the result must be 3-optimal, which brute force
over every 2- and 3-exchange checks on small instances; the search never
lengthens a tour and stops at a fixed point."""
import itertools
import math

import numpy as np
import pytest

from helpers import dmat, euclid, is_perm, params


def full_lists(D):
    n = D.shape[0]
    out = np.empty((n, n - 1), np.int32)
    for i in range(n):
        d = D[i].copy()
        d[i] = np.inf
        out[i] = np.lexsort((np.arange(n), d))[:n - 1]
    return out


def length(D, t):
    return math.fsum(D[t[q], t[(q + 1) % len(t)]] for q in range(len(t)))


def best_exchange(D, t):
    """Largest improvement of any 2- or 3-exchange of tour t (brute force)."""
    n = len(t)
    L0 = length(D, t)
    best = 0.0
    for i, j in itertools.combinations(range(n), 2):
        A, B, R = t[:i + 1], t[i + 1:j + 1], t[j + 1:]
        best = max(best, L0 - length(D, A + B[::-1] + R))
    for i, j, k in itertools.combinations(range(n), 3):
        A, B, C, R = t[:i + 1], t[i + 1:j + 1], t[j + 1:k + 1], t[k + 1:]
        for X, Y in ((B, C), (C, B)):
            for rx in (0, 1):
                for ry in (0, 1):
                    new = A + (X[::-1] if rx else X) + (Y[::-1] if ry else Y) + R
                    best = max(best, L0 - length(D, new))
    return best


@pytest.mark.parametrize("seed", range(12))
def test_full_lists_reach_a_3_optimal_tour(orc, seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(5, 10))
    pts = rng.random((n, 2)).astype(np.float32)
    D = dmat(pts)
    start = rng.permutation(n).astype(np.int32)
    t, moves = orc.three_opt(euclid(pts), full_lists(D), start)
    assert is_perm(t, n)
    assert length(D, list(t)) <= length(D, list(start)) + 1e-12
    assert best_exchange(D, list(t)) <= 1e-9
    t2, again = orc.three_opt(euclid(pts), full_lists(D), t)
    assert again == 0 and np.array_equal(t2, t)


def test_three_opt_improves_2_optimal_tours(orc):
    """On tours that the 2-opt leaves, the 3-opt still finds segment moves:
    found on several small random instances, each ending 3-optimal."""
    hits = 0
    for seed in range(150):
        rng = np.random.default_rng(100 + seed)
        n = 9
        pts = rng.random((n, 2)).astype(np.float32)
        D = dmat(pts)
        nb = full_lists(D)
        t2, _ = orc.two_opt(euclid(pts), nb, rng.permutation(n).astype(np.int32))
        if best_exchange(D, list(t2)) <= 1e-9:
            continue
        t3, moves = orc.three_opt(euclid(pts), nb, t2)
        assert moves > 0
        assert length(D, list(t3)) < length(D, list(t2)) - 1e-9
        assert best_exchange(D, list(t3)) <= 1e-9
        hits += 1
    assert hits >= 3


def test_segment_insertion_case(orc):
    """Points on a line, visited 0 1 2 3 4 5 6 7 with the pair (2, 3) moved to
    the far end: no 2-opt move helps more than reversing, but moving the
    segment back is a 3-exchange to the optimum 2 (x_max - x_min)."""
    x = np.array([0, 1, 2, 3, 4, 5, 6, 7], np.float32)
    pts = np.stack([x, np.zeros(8, np.float32)], 1) / 8
    D = dmat(pts)
    start = np.array([0, 1, 4, 5, 6, 2, 3, 7], np.int32)
    t, moves = orc.three_opt(euclid(pts), full_lists(D), start)
    assert moves >= 1
    assert length(D, list(t)) == pytest.approx(2 * 7 / 8, abs=1e-12)


def test_decode_with_three_opt(orc):
    """local_search 3 (T_ib and T_NN) and 4 (every ant): permutations, lengths
    recomputed, and every improved tour is a fixed point of the 3-opt."""
    rng = np.random.default_rng(5)
    pts = rng.random((60, 2)).astype(np.float32)
    for ls in (3, 4):
        p = params(m=6, k=10, iterations=4, rho=0.2, local_search=ls, ls_k=8, seed=3)
        o = orc.Oracle(euclid(pts), p).iterate(4)
        nb = o.get("nbr")
        for t in (o.get("ib_tour"), o.get("gb_tour"), o.get("nn_tour")):
            assert is_perm(t, 60)
            t2, again = orc.three_opt(euclid(pts), nb, t)
            assert again == 0
        assert o.scalars()["L_ib"] == orc.tour_length(euclid(pts), o.get("ib_tour"))
        if ls == 4:
            for a in range(6):
                _, again = orc.three_opt(euclid(pts), nb, o.get("tours")[a])
                assert again == 0


def _exchange_instance():
    """Nine points and the tour 0 1 [4 5 6] [2 3] 7 8 whose segments B = 4 5 6
    and C = 2 3 are swapped without reversal in the optimal-looking order
    0 1 2 3 4 5 6 7 8.  Neighbour lists hold one city: nbr(4) = 3, nbr(7) = 6,
    every other city its farthest city (so no exchange starts there).  The
    points are drawn (seeded) until every exchange these lists allow through
    a closable 2-opt tour is non-improving while the swap improves."""
    rng = np.random.default_rng(77)
    for _ in range(200000):
        pts = rng.random((9, 2)).astype(np.float32)
        d = dmat(pts)
        g1 = d[1, 4] - d[4, 3]
        g2 = g1 + d[3, 7] - d[7, 6]
        ok = (d[4, 5] <= d[4, 3] and d[1, 4] + d[3, 2] <= d[4, 3] + d[2, 1] and d[7, 8] <= d[7, 6]
              and d[7, 3] + d[6, 5] <= d[7, 6] + d[5, 3] and g1 > 1e-3 and g2 > 1e-3
              and g2 + d[6, 2] - d[2, 1] > 1e-3)
        if ok:
            return pts, d
    raise AssertionError("no instance found")


def test_segment_swap_needs_the_non_closable_side(orc):
    """The swap removes (1,4), (6,2), (3,7) and adds (1,2), (3,4), (6,7).  As a
    sequential exchange from t2 = 4, t1 = 1: t3 = 3, then t4 = 7, the neighbour
    of 3 on the side where closing after two edges would split the tour, then
    t5 = 6, t6 = 2.  Every other chain the lists allow is non-improving, so the
    search must take exactly this move and stop: one move, and the middle of
    the array rewritten to 0 1 2 3 4 5 6 7 8."""
    pts, d = _exchange_instance()
    nb = np.empty((9, 1), np.int32)
    for i in range(9):
        nb[i, 0] = int(np.argmax(d[i]))
    nb[4, 0], nb[7, 0] = 3, 6
    start = np.array([0, 1, 4, 5, 6, 2, 3, 7, 8], np.int32)
    t, moves = orc.three_opt(euclid(pts), nb, start)
    assert moves == 1
    assert list(t) == list(range(9))
    assert length(d, list(t)) < length(d, list(start)) - 1e-3


