"""Pins of the oracle's preparation: candidate lists (Sec. III-A), the evidence
factor and its scale (Sec. III-C), the bounds (eqs. tau_init, tau_min_nols) and
the nearest-neighbour tour of Algorithm 1."""
import math

import numpy as np
import pytest

from helpers import atsp, dmat, euclid, params
from paper_2601_19041_gb300 import synth


def test_empty_heatmap_gives_knn_lists_and_classical_weights(orc):
    rng = np.random.default_rng(1)
    pts = rng.random((60, 2)).astype(np.float32)
    inst = euclid(pts)
    o = orc.Oracle(inst, params(m=4, k=20, iterations=0, rho=0.2))
    D = dmat(pts)
    cand = o.get("cand")
    for i in range(60):
        d = D[i].copy()
        d[i] = np.inf
        ref = np.lexsort((np.arange(60), d))[:20]        # 20 nearest by (d, j)
        assert list(cand[i]) == list(ref)
    assert np.all(o.get("conf") == 0.0)
    assert np.all(o.get("base") == 1e-9)
    assert np.all(o.get("evid") == 1.0)
    s = o.scalars()
    assert s["n_lambda"] == 0 and s["kappa"] == 0.0
    # kappa = 0: the weight is the classical MMAS heuristic eta^2 (Sec. III-A)
    eta2 = (1.0 / D[np.arange(60)[:, None], cand]) ** 2
    assert np.array_equal(o.get("W"), eta2.astype(np.float32))


def test_full_uniform_heatmap_gives_unit_evidence(orc):
    rng = np.random.default_rng(2)
    pts = rng.random((40, 2)).astype(np.float32)
    H = np.full((40, 40), 0.5)
    np.fill_diagonal(H, 0)
    o = orc.Oracle(euclid(pts, H), params(m=4, k=12, iterations=0, rho=0.2))
    D = dmat(pts)
    for i in range(40):
        d = D[i].copy()
        d[i] = np.inf
        assert list(o.get("cand")[i][:12]) == list(np.lexsort((np.arange(40), d))[:12])
    # equal scores in a row: b_i = the common value, e_ij = 1 (Sec. III-C)
    assert np.all(o.get("base") == 0.5)
    assert np.all(o.get("evid")[:, :12] == 1.0)
    assert o.scalars()["kappa"] == 0.0


def _hand_instance():
    # 6 points on a line; node 0 sees heat 0.5, 0.3, 0.1, 0.05 on nodes 1..4,
    # node 5 sees heat on exactly two nodes (fewer than d*+1 = 3 positives).
    pts = np.array([[0, 0], [1, 0], [2, 0], [3, 0], [4, 0], [5, 0]], np.float32) / 8
    H = np.zeros((6, 6))
    H[0, 1:5] = [0.5, 0.3, 0.1, 0.05]
    H[5, 3] = 0.2
    H[5, 4] = 0.4
    return pts, H


def test_hand_worked_evidence_rows(orc):
    pts, H = _hand_instance()
    o = orc.Oracle(euclid(pts, H, symmetrize=0), params(m=2, k=8, iterations=0, rho=0.2))
    cand, conf, evid = o.get("cand"), o.get("conf"), o.get("evid")
    assert o.k_eff == 5 and o.k_pad == 8
    # row 0: candidates ordered by distance 1,2,3,4,5 ; c = .5,.3,.1,.05,0
    assert list(cand[0]) == [1, 2, 3, 4, 5, -1, -1, -1]
    assert list(conf[0][:5]) == pytest.approx([0.5, 0.3, 0.1, 0.05, 0.0], abs=1e-7)
    assert o.get("base")[0] == pytest.approx(0.1, rel=1e-7)     # third-highest (d* = 2)
    assert list(evid[0][:5]) == pytest.approx([5.0, 3.0, 1.0, 1.0, 1.0], rel=1e-6)
    assert o.get("logev")[0][0] == pytest.approx(math.log(5.0), rel=1e-6)
    # row 5: two positives -> missing third statistic -> b = eps
    assert o.get("base")[5] == 1e-9
    assert evid[5][list(cand[5]).index(4)] == pytest.approx(0.4 / 1e-9, rel=1e-6)
    # rows without heat: b = eps, e = 1 everywhere
    assert np.all(evid[2][:5] == 1.0)


def test_atsp_degree_target_one(orc):
    pts, H = _hand_instance()
    D = dmat(pts)
    o = orc.Oracle(atsp(D, H), params(m=2, k=8, iterations=0, rho=0.2, degree_target=1))
    assert o.get("base")[0] == pytest.approx(0.3, rel=1e-7)     # second-highest (d* = 1)
    assert o.get("evid")[0][0] == pytest.approx(0.5 / 0.3, rel=1e-6)


def test_baseline_scope_whole_row(orc):
    # node 0 has 4 heat entries but only k=2 candidate slots: the retained pair
    # is the two closest heat nodes, the far ones only count for scope 1.
    pts = np.array([[0, 0], [1, 0], [2, 0], [9, 0], [10, 0], [11, 0]], np.float32) / 16
    H = np.zeros((6, 6))
    H[0, [1, 2, 3, 4]] = [0.2, 0.1, 0.9, 0.8]
    p0 = params(m=2, k=2, iterations=0, rho=0.2, degree_target=1)
    o0 = orc.Oracle(euclid(pts, H, symmetrize=0), p0)
    assert list(o0.get("cand")[0][:2]) == [1, 2]
    assert o0.get("base")[0] == pytest.approx(0.1, rel=1e-7)
    p1 = params(m=2, k=2, iterations=0, rho=0.2, degree_target=1, baseline_scope=1)
    o1 = orc.Oracle(euclid(pts, H, symmetrize=0), p1)
    assert o1.get("base")[0] == pytest.approx(0.8, rel=1e-7)    # 2nd of {.9,.8,.2,.1}
    assert np.all(o1.get("evid")[0][:2] == 1.0)


def test_fill_with_nearest_non_members(orc):
    # |P_i| < k: members kept, remaining slots are the nearest non-members
    rng = np.random.default_rng(3)
    pts = rng.random((30, 2)).astype(np.float32)
    D = dmat(pts)
    H = np.zeros((30, 30))
    far = np.argsort(D[0])[-3:]                          # three far nodes carry heat
    H[0, far] = 0.3
    o = orc.Oracle(euclid(pts, H, symmetrize=0), params(m=2, k=8, iterations=0, rho=0.2))
    c0 = set(o.get("cand")[0].tolist())
    d = D[0].copy(); d[0] = np.inf; d[far] = np.inf
    near5 = set(np.lexsort((np.arange(30), d))[:5].tolist())
    assert c0 == set(far.tolist()) | near5
    # slot order is ascending distance
    assert np.all(np.diff(o.get("cdist")[0]) >= 0)


def test_more_members_than_k_keeps_closest(orc):
    rng = np.random.default_rng(4)
    pts = rng.random((50, 2)).astype(np.float32)
    H = (rng.random((50, 50)) < 0.6) * 0.01
    np.fill_diagonal(H, 0)
    inst = euclid(pts, H, symmetrize=0)
    o = orc.Oracle(inst, params(m=2, k=8, iterations=0, rho=0.2))
    D = dmat(pts)
    for i in range(50):
        mem = [j for j in range(50) if H[i, j] > 1e-4]
        ref = sorted(mem, key=lambda j: (D[i, j], j))[:8]
        if len(mem) >= 8:
            assert list(o.get("cand")[i]) == ref


def test_symmetrisation_and_half_precision(orc):
    rng = np.random.default_rng(5)
    pts = rng.random((25, 2)).astype(np.float32)
    H = np.where(rng.random((25, 25)) < 0.3, rng.random((25, 25)), 0.0)
    np.fill_diagonal(H, 0)
    H16 = H.astype(np.float16).astype(np.float64)
    inst = euclid(pts, H16, symmetrize=1, dtype=np.float16)
    for i in range(25):
        for j in range(25):
            if i != j:
                assert orc.heat(inst, i, j) == (H16[i, j] + H16[j, i]) / 2


def test_kappa_cap_identity_and_dynamic_range(orc):
    """kappa * q90 = c_cap * alpha * ln R (Sec. III-C) and R = tau_max/tau_min."""
    inst, ps = synth.workload("tsp500")
    for ls, alpha in ((0, 1.0), (1, 1.0), (0, 1.5)):
        p = ps[0]
        p.local_search, p.alpha, p.iterations = ls, alpha, 0
        o = orc.Oracle(inst[0], p)
        s = o.scalars()
        logev = o.get("logev")
        lam = np.sort(logev[logev > 0])
        assert s["n_lambda"] == len(lam)
        assert s["q90"] == pytest.approx(np.quantile(lam, 0.9), rel=1e-14)
        assert s["kappa"] * s["q90"] == pytest.approx(0.5 * alpha * math.log(s["Rhat"]), rel=1e-13)
        assert s["tau_max64"] / s["tau_min64"] == pytest.approx(s["Rhat"], rel=1e-13)
        n, k = 500, 20
        if ls:
            assert s["Rhat"] == 2 * n
        else:
            px = 0.05 ** (1.0 / n)
            assert s["p_x"] == pytest.approx(px, rel=1e-14)
            assert s["Rhat"] == pytest.approx((k - 1) / 2 * px / (1 - px), rel=1e-12)


def test_nn_tour_on_a_line(orc):
    # increasing gaps along a line: the nearest-unvisited tour from node 0 visits
    # the points in order and the closed tour has length 2 * (x_max - x_0)
    n = 40
    x = (np.arange(n) ** 2).astype(np.float32) / 1600.0
    pts = np.stack([x, np.zeros(n, np.float32)], 1)
    perm = np.random.default_rng(8).permutation(n)
    perm = np.concatenate([[0], perm[perm != 0]])      # node 0 stays the leftmost point
    o = orc.Oracle(euclid(pts[perm]), params(m=2, k=8, iterations=0, rho=0.2))
    inv = np.argsort(perm)
    assert list(o.get("nn_tour")) == list(inv[np.arange(n)])
    assert o.scalars()["L_nn"] == pytest.approx(2 * float(x[-1]), rel=1e-12)
    s = o.scalars()
    assert s["tau_max64"] == pytest.approx(1.0 / (0.2 * 2 * float(x[-1])), rel=1e-12)


def test_small_n_uses_all_other_nodes(orc):
    pts = np.random.default_rng(9).random((5, 2)).astype(np.float32)
    o = orc.Oracle(euclid(pts), params(m=3, k=20, iterations=2, rho=0.2))
    assert o.k_eff == 4 and o.k_pad == 20
    c = o.get("cand")
    for i in range(5):
        assert sorted(c[i][:4].tolist()) == sorted(set(range(5)) - {i})
        assert np.all(c[i][4:] == -1)


def test_rejects_bad_inputs(orc):
    pts = np.random.default_rng(9).random((5, 2)).astype(np.float32)
    with pytest.raises(ValueError):
        orc.Oracle(euclid(pts[:2]), params(m=3, k=4))
    with pytest.raises(ValueError):
        orc.Oracle(euclid(pts), params(m=3, k=33))
    H = np.zeros((5, 5)); H[0, 1] = 1.5
    with pytest.raises(ValueError):
        orc.Oracle(euclid(pts, H), params(m=3, k=4, rho=0.2))
