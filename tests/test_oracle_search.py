"""Pins of the oracle's search: the roulette sampler and start node (Alg. 2),
decoding quality against brute-force and closed-form optima, the per-iteration
invariants of the bounded update (eq. pheromone_update), and the 2-opt
(Sec. III-D)."""
import itertools
import math
from fractions import Fraction

import numpy as np
import pytest

from helpers import (strided_partials_len, brute_force_opt, cycle_heat, dmat, euclid, is_perm, params,
                     tour_len)


# ------------------------------------------------------------------ sampler

def test_roulette_matches_weights_chi_square(orc):
    stats = pytest.importorskip("scipy.stats")
    rng = np.random.default_rng(11)
    w = rng.exponential(1.0, 20).astype(np.float32)
    w[[3, 9, 17]] = 0.0
    N = 200_000
    us = (rng.integers(0, 1 << 24, N) * 2.0 ** -24).astype(np.float32)
    counts = np.bincount([orc.roulette(w, float(u)) for u in us], minlength=20)
    assert counts[[3, 9, 17]].sum() == 0                 # visited slots never chosen
    live = w > 0
    exp = w[live] / w[live].sum() * N
    assert stats.chisquare(counts[live], exp).pvalue > 1e-4


def test_roulette_is_exact_inverse_cdf_away_from_boundaries(orc):
    # brute force over a fine grid of u: the chosen slot is the one whose exact
    # cumulative interval contains u * sum(w), except within float rounding of a boundary
    w = np.array([0.5, 0.0, 1.25, 3.0, 0.75, 0.0, 2.0, 0.125], np.float32)
    cum = np.cumsum([Fraction(float(x)) for x in w])
    tot = cum[-1]
    for q in range(0, 1 << 12):
        u = q / 4096.0
        c = orc.roulette(w, u)
        x = Fraction(u) * tot
        ref = next(i for i in range(8) if w[i] > 0 and x < cum[i])
        near = min(abs(float(x - b)) for b in cum)
        if near > 1e-5:
            assert c == ref
        assert w[c] > 0


def test_roulette_single_live_slot_and_top_draw(orc):
    w = np.zeros(32, np.float32)
    w[29] = 3.5
    for u in (0.0, 0.5, 1.0 - 2 ** -24):
        assert orc.roulette(w, u) == 29


def test_start_node_uniform(orc):
    stats = pytest.importorskip("scipy.stats")
    n = 7
    starts = [((orc.draw(seed, 0, a, 0) * n) >> 32) for seed in range(200) for a in range(50)]
    counts = np.bincount(starts, minlength=n)
    assert stats.chisquare(counts).pvalue > 1e-4


# ------------------------------------------------------------------ decoding quality

@pytest.mark.parametrize("n", [6, 7, 8])
def test_reaches_brute_force_optimum(orc, n):
    hits = 0
    for seed in range(10):
        pts = np.random.default_rng(100 + seed + 17 * n).random((n, 2)).astype(np.float32)
        D = dmat(pts)
        Lopt, _ = brute_force_opt(D)
        tour, L, _ = orc.solve(euclid(pts), params(m=10, k=20, iterations=60, rho=0.2, seed=seed))
        assert is_perm(tour, n)
        assert L >= Lopt - 1e-12
        hits += L <= Lopt + 1e-12
    assert hits >= 9


@pytest.mark.parametrize("n", [7, 9])
def test_concentrated_heatmap_decodes_to_the_optimum(orc, n):
    pts = np.random.default_rng(200 + n).random((n, 2)).astype(np.float32)
    D = dmat(pts)
    Lopt, topt = brute_force_opt(D)
    H = cycle_heat(n, topt, 1.0)
    tour, L, _ = orc.solve(euclid(pts, H), params(m=8, k=20, iterations=15, rho=0.2, seed=3))
    assert L == pytest.approx(Lopt, abs=1e-12)


def test_convex_position_decodes_to_angular_order(orc):
    n = 200
    rng = np.random.default_rng(21)
    ang = np.sort(rng.uniform(0, 2 * np.pi, n))
    pts = np.stack([0.5 + 0.4 * np.cos(ang), 0.5 + 0.4 * np.sin(ang)], 1).astype(np.float32)
    perm = rng.permutation(n)
    P = pts[perm]
    inv = np.argsort(perm)                              # angular rank -> node id
    opt = [int(inv[r]) for r in range(n)]
    H = cycle_heat(n, opt, 0.9)
    tour, L, _ = orc.solve(euclid(P, H), params(m=20, k=20, iterations=30, rho=0.2, seed=1))
    D = dmat(P)
    Lopt = tour_len(D, opt)                              # convex polygon perimeter
    assert L == pytest.approx(Lopt, rel=1e-12)
    # the tour is the angular cycle in one of its two orientations
    r = np.argsort(np.argsort(perm))[np.asarray(tour)]
    steps = np.diff(np.concatenate([r, r[:1]])) % n
    assert np.all(steps == 1) or np.all(steps == n - 1)


def test_even_grid_reaches_closed_form_optimum(orc):
    m = 10                                              # m x m unit grid: optimum = m^2
    pts = np.array([(x, y) for y in range(m) for x in range(m)], np.float32)
    idx = lambda x, y: y * m + x
    cyc = [idx(x, 0) for x in range(m)]
    for c in range(m - 1, 0, -1):
        ys = range(1, m) if (m - 1 - c) % 2 == 0 else range(m - 1, 0, -1)
        cyc += [idx(c, y) for y in ys]
    cyc += [idx(0, y) for y in range(m - 1, 0, -1)]
    assert is_perm(cyc, m * m)
    assert tour_len(dmat(pts), cyc) == m * m
    H = cycle_heat(m * m, cyc, 0.8)
    tour, L, _ = orc.solve(euclid(pts, H), params(m=20, k=12, iterations=40, rho=0.2, seed=2))
    assert L == m * m


# ------------------------------------------------------------------ invariants

def test_invariants_every_iteration(orc):
    from paper_2601_19041_gb300 import synth
    inst = synth.euclid_instance(77, 150, K=30)
    p = params(m=12, k=10, iterations=25, rho=0.2, seed=9)
    o = orc.Oracle(inst, p)
    D = dmat(inst.coords)
    s0 = o.scalars()
    prev_gb = s0["L_nn"]
    cand = o.get("cand")
    real = cand >= 0
    for t in range(p.iterations):
        tau_before = o.get("tau").copy()
        tmax_before, tmin_before = o.scalars()["tau_max"], o.scalars()["tau_min"]
        o.iterate(1)
        s = o.scalars()
        tours, lens = o.get("tours"), o.get("lens")
        for a in range(p.m):
            assert is_perm(tours[a], inst.n)
            assert lens[a] == pytest.approx(tour_len(D, tours[a]), rel=1e-14)
            assert lens[a] == strided_partials_len(D, tours[a])   # the stated order, bitwise
        ib = int(np.argmin(lens))
        assert o.get("trace_ib")[t] == ib
        assert s["L_gb"] <= prev_gb and s["L_gb"] <= s0["L_nn"]
        prev_gb = s["L_gb"]
        tau = o.get("tau")
        assert np.all(tau[real] >= np.float32(s["tau_min"]))
        assert np.all(tau[real] <= np.float32(s["tau_max"]))
        assert np.all(tau[~real] == 0)
        # eq. (pheromone_update) with T+ = T_ib: evaporate everywhere, deposit on
        # the (either-orientation) slots of T_ib's edges, then clamp
        tib = tours[ib]
        on = np.zeros_like(real)
        nxt = {int(tib[q]): int(tib[(q + 1) % inst.n]) for q in range(inst.n)}
        prv = {v: u for u, v in nxt.items()}
        for i in range(inst.n):
            for c in range(o.k_pad):
                on[i, c] = real[i, c] and cand[i, c] in (nxt[i], prv[i])
        x = tau_before * np.float32(1.0 - p.rho)
        x = np.where(on, x + np.float32(1.0 / lens[ib]), x)
        ref = np.minimum(np.float32(s["tau_max"]), np.maximum(np.float32(s["tau_min"]), x))
        assert np.array_equal(tau[real], ref[real])
        assert np.array_equal(o.get("choice")[real], (tau * o.get("W"))[real])
        if s["L_gb"] < prev_gb:
            assert s["tau_max64"] == 1.0 / (p.rho * s["L_gb"])


def test_atsp_deposits_one_orientation(orc):
    rng = np.random.default_rng(31)
    n = 30
    C = rng.random((n, n)).astype(np.float32)
    np.fill_diagonal(C, 0)
    from helpers import atsp
    p = params(m=6, k=8, iterations=1, rho=0.2, degree_target=1, seed=4)
    o = orc.Oracle(atsp(C), p)
    tmax = np.float32(o.scalars()["tau_max"])
    o.iterate(1)
    s = o.scalars()
    tib = o.get("tours")[o.get("trace_ib")[0]]
    nxt = {int(tib[q]): int(tib[(q + 1) % n]) for q in range(n)}
    cand, tau = o.get("cand"), o.get("tau")
    lib_ = o.get("lens").min()
    for i in range(n):
        for c in range(o.k_eff):
            x = np.float32(tmax * np.float32(1 - p.rho))
            if cand[i, c] == nxt[i]:
                x = np.float32(x + np.float32(1.0 / lib_))
            x = min(np.float32(s["tau_max"]), max(np.float32(s["tau_min"]), x))
            assert tau[i, c] == x


def test_tour_length_order_and_accuracy(orc):
    """The strided-partials FP64 sum: exact on integer edge lengths, within the
    error bound of its order (n/32 sequential adds, then a 5-level tree) of the
    exact (rational) sum otherwise."""
    from fractions import Fraction
    m = 8
    pts = np.array([(x, y) for y in range(m) for x in range(m)], np.float32)
    cyc = list(range(m * m))       # row-major snake is not a grid tour; any permutation works
    inst = euclid(pts)
    D = dmat(pts)
    assert orc.tour_length(inst, cyc) == strided_partials_len(D, cyc)
    rng = np.random.default_rng(12)
    for n in (3, 31, 32, 33, 100, 1000):
        P = rng.random((n, 2)).astype(np.float32)
        inst = euclid(P)
        D = dmat(P)
        t = rng.permutation(n)
        L = orc.tour_length(inst, t)
        exact = sum(Fraction(D[t[e], t[(e + 1) % n]]) for e in range(n))
        bound = (5 + math.ceil(n / 32) + 2) * 2.0 ** -53 * float(exact)
        assert abs(Fraction(L) - exact) <= Fraction(bound)
    # four unit edges: (1 + 1) + (1 + 1) = 4 exactly
    sq = euclid(np.array([[0, 0], [1, 0], [1, 1], [0, 1]], np.float32))
    assert orc.tour_length(sq, [0, 1, 2, 3]) == 4.0


# ------------------------------------------------------------------ 2-opt

def _two_opt_gain_left(D, tour, nbr):
    """Largest gain of any neighbour-list 2-opt move still available: a move
    from city a towards b in nbr(a) with d(a, b) < d(a, a's tour neighbour)."""
    n = len(tour)
    pos = np.empty(n, int)
    pos[tour] = np.arange(n)
    best = -math.inf
    for a in range(n):
        for b in nbr[a]:
            for step in (1, -1):
                an = tour[(pos[a] + step) % n]
                bn = tour[(pos[b] + step) % n]
                if len({a, an, b, bn}) < 4 or not D[a, b] < D[a, an]:
                    continue
                best = max(best, D[a, an] + D[b, bn] - D[a, b] - D[an, bn])
    return best


def test_two_opt_reaches_neighbour_list_local_optimum(orc):
    rng = np.random.default_rng(41)
    n, K = 120, 10
    pts = rng.random((n, 2)).astype(np.float32)
    inst = euclid(pts)
    D = dmat(pts)
    nbr = np.argsort(D + np.diag(np.full(n, np.inf)), axis=1, kind="stable")[:, :K]
    tour0 = rng.permutation(n).astype(np.int32)
    tour, moves = orc.two_opt(inst, nbr, tour0)
    assert moves > 0 and is_perm(tour, n)
    assert tour_len(D, tour) < tour_len(D, tour0)
    assert _two_opt_gain_left(D, tour, nbr) <= 1e-9


def test_two_opt_full_lists_is_globally_two_optimal(orc):
    for seed in range(5):
        rng = np.random.default_rng(50 + seed)
        n = 9
        pts = rng.random((n, 2)).astype(np.float32)
        D = dmat(pts)
        nbr = np.argsort(D + np.diag(np.full(n, np.inf)), axis=1, kind="stable")[:, :n - 1]
        tour, _ = orc.two_opt(euclid(pts), nbr, rng.permutation(n))
        L = tour_len(D, tour)
        for i, j in itertools.combinations(range(n), 2):   # every segment reversal
            t2 = list(tour[:i]) + list(tour[i:j + 1][::-1]) + list(tour[j + 1:])
            assert tour_len(D, t2) >= L - 1e-10


def test_two_opt_uncrosses_square(orc):
    pts = np.array([[0, 0], [1, 0], [1, 1], [0, 1]], np.float32)
    nbr = np.array([[1, 3, 2], [0, 2, 3], [1, 3, 0], [0, 2, 1]])
    tour, moves = orc.two_opt(euclid(pts), nbr, np.array([0, 2, 1, 3]))
    assert moves == 1 and tour_len(dmat(pts), tour) == 4.0


def test_local_search_run_keeps_invariants(orc):
    from paper_2601_19041_gb300 import synth
    inst = synth.euclid_instance(91, 300, K=10)
    p = params(m=8, k=10, iterations=6, rho=0.2, local_search=1, seed=5)
    o = orc.Oracle(inst, p)
    D = dmat(inst.coords)
    s0 = o.scalars()
    assert s0["Rhat"] == 600 and s0["tau_max64"] / s0["tau_min64"] == pytest.approx(600, rel=1e-13)
    nbr = o.get("nbr")
    assert _two_opt_gain_left(D, o.get("nn_tour"), nbr) <= 1e-9
    o.iterate(p.iterations)
    ib = o.get("ib_tour")
    assert is_perm(ib, inst.n)
    assert _two_opt_gain_left(D, ib, nbr) <= 1e-9
    assert o.scalars()["L_ib"] == strided_partials_len(D, ib)
    assert o.scalars()["L_gb"] <= s0["L_nn"]


def test_local_search_on_every_ant(orc):
    # Algorithm 1's local search with local_search = 2: every ant's tour is 2-opted before
    # the iteration best is taken; lengths are those of the improved tours
    from paper_2601_19041_gb300 import synth
    inst = synth.euclid_instance(92, 150, K=10)
    p = params(m=6, k=10, iterations=4, rho=0.2, local_search=2, ls_k=10, seed=6)
    o = orc.Oracle(inst, p)
    D = dmat(inst.coords)
    nbr = o.get("nbr")
    o.iterate(p.iterations)
    tours, lens = o.get("tours"), o.get("lens")
    for a in range(p.m):
        assert is_perm(tours[a], inst.n)
        assert _two_opt_gain_left(D, tours[a], nbr) <= 1e-9
        assert lens[a] == strided_partials_len(D, tours[a])
    ib = int(np.argmin(lens))
    assert np.array_equal(o.get("ib_tour"), tours[ib])
    assert o.scalars()["L_ib"] == lens[ib]
    s = o.scalars()
    assert s["Rhat"] == 300 and s["tau_max64"] / s["tau_min64"] == pytest.approx(300, rel=1e-13)
