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


# ---------------------------------------------------------------------------
# The static weight W = fl32(eta^beta * exp(min(kappa * ln e, clip))) of the end
# of Sec. III-C and eq. (transition), and choice = fl32(tau^alpha * W), checked
# against an independent high-precision evaluation (mpmath) of the same
# definition.  The oracle's FP64 pre-rounding value carries a relative error of
# a few 1e-15 (own exp/ln within 2 ulp, a handful of roundings); a float32
# rounding decision can only depend on it when the exact value lies within
# 1e-12 (relative) of a float32 rounding midpoint, and such slots are counted
# and skipped (there are none in practice).

_MID_TOL = 1e-12


def _fl32_of_exact(x, mpmath):
    """float32 nearest to the mpmath value x > 0, or None when x is within
    _MID_TOL of a float32 rounding midpoint (decision not pinned)."""
    f = np.float32(float(x))                       # a float32 next to x
    lo = f if mpmath.mpf(float(f)) <= x else np.nextafter(f, np.float32(0))
    hi = np.nextafter(lo, np.float32(np.inf))
    mid = (mpmath.mpf(float(lo)) + mpmath.mpf(float(hi))) / 2
    if abs(x - mid) <= _MID_TOL * x:
        return None
    return lo if x < mid else hi


def _exact_weights(o, p, mpmath, kappa=None):
    """W of every real slot from the definition, in 60-digit arithmetic, from the
    oracle's FP64 inputs d_ij, c_ij and b_i (pinned by the tests above) and its
    kappa (pinned by the cap identity)."""
    mpmath.mp.dps = 60
    kap = mpmath.mpf(o.scalars()["kappa"] if kappa is None else kappa)
    cdist, conf, base = o.get("cdist"), o.get("conf"), o.get("base")
    clip, eps, beta = mpmath.mpf(p.logw_clip), mpmath.mpf(p.eps), mpmath.mpf(p.beta)
    out = {}
    for i in range(o.n):
        b = mpmath.mpf(float(base[i]))
        for c in range(o.k_eff):
            d = max(float(cdist[i, c]), 1e-9)
            eta = 1 / mpmath.mpf(d)
            e = max(max(mpmath.mpf(float(conf[i, c])), eps) / b, mpmath.mpf(1))
            lw = kap * mpmath.log(e) if e > 1 else mpmath.mpf(0)
            out[(i, c)] = mpmath.power(eta, beta) * mpmath.exp(min(lw, clip))
    return out


def _check_weights(o, p, mpmath, kappa=None):
    exact = _exact_weights(o, p, mpmath, kappa)
    W = o.get("W")
    skipped = 0
    for (i, c), x in exact.items():
        ref = _fl32_of_exact(x, mpmath)
        if ref is None:
            skipped += 1
            continue
        assert W[i, c] == ref, (i, c, float(W[i, c]), float(x))
    assert skipped <= max(1, len(exact) // 1000)
    assert np.all(W[:, o.k_eff:] == 0.0)
    return exact


def test_weights_with_evidence_match_exact_evaluation(orc):
    """kappa > 0 on the n=500 workload instance: every W equals the float32
    rounding of the exactly evaluated eta^2 * e^kappa.  A dropped or halved
    exponent, a wrong eta power or a misplaced clip changes most slots."""
    mpmath = pytest.importorskip("mpmath")
    inst, ps = synth.workload("tsp500")
    p = ps[0]
    p.iterations = 0
    o = orc.Oracle(inst[0], p)
    s = o.scalars()
    assert s["kappa"] > 0.5 and s["n_lambda"] >= 900           # evidence is active (top 2 per row)
    logev = o.get("logev")
    assert (s["kappa"] * logev).max() > 2.0                   # factors well above 1
    exact = _check_weights(o, p, mpmath)
    # the evidence really enters: W differs from eta^2 on every slot with e > 1
    D = o.get("cdist")
    eta2 = (1.0 / D[:, :o.k_eff]) ** 2
    W = o.get("W")[:, :o.k_eff]
    on = logev[:, :o.k_eff] > 0
    assert np.all(W[on] > eta2[on].astype(np.float32) * 1.0001)
    assert len(exact) == 500 * 20


def test_weight_clip_fires(orc):
    """A log-weight clip below kappa*ln(e) caps the factor at exp(clip)
    (end of Sec. III-C): W = fl32(eta^2 * exp(clip)) on the clipped slots."""
    mpmath = pytest.importorskip("mpmath")
    inst, ps = synth.workload("tsp500")
    p = ps[0]
    p.iterations, p.logw_clip = 0, 1.25
    o = orc.Oracle(inst[0], p)
    kl = o.scalars()["kappa"] * o.get("logev")
    clipped = kl > 1.25
    assert 50 < clipped.sum() < kl.size - 50                   # both sides occur
    _check_weights(o, p, mpmath)
    D = o.get("cdist")
    for i, c in zip(*np.nonzero(clipped)):
        x = (1 / mpmath.mpf(float(D[i, c]))) ** 2 * mpmath.exp(mpmath.mpf(1.25))
        ref = _fl32_of_exact(x, mpmath)
        if ref is not None:
            assert o.get("W")[i, c] == ref


def test_hand_worked_weight_row(orc):
    """Row 0 of the 6-node line: e = 5, 3, 1, 1, 1 over candidates at
    distances 1/8 .. 5/8, so W_0c = 64/c^2 * e_c^kappa."""
    mpmath = pytest.importorskip("mpmath")
    pts, H = _hand_instance()
    p = params(m=2, k=8, iterations=0, rho=0.2)
    o = orc.Oracle(euclid(pts, H, symmetrize=0), p)
    kap = o.scalars()["kappa"]
    assert kap > 0
    W = o.get("W")[0]
    for c, e in enumerate([5, 3, 1, 1, 1]):
        x = mpmath.mpf(64) / (c + 1) ** 2 * mpmath.power(e, mpmath.mpf(kap))
        assert W[c] == _fl32_of_exact(x, mpmath)


def test_weights_beta_three(orc):
    """beta != 2 takes eta^beta = exp(beta ln eta) with the oracle's own exp/ln."""
    mpmath = pytest.importorskip("mpmath")
    inst, ps = synth.workload("tsp500")
    p = ps[0]
    p.iterations, p.beta = 0, 3.0
    o = orc.Oracle(inst[0], p)
    _check_weights(o, p, mpmath)


def test_choice_alpha_power(orc):
    """choice = fl32(tau^alpha * W) (numerator of eq. transition) for alpha=1.5
    after some iterations, against the exact power of the stored tau and W."""
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 60
    inst, ps = synth.workload("tsp500")
    p = ps[0]
    p.iterations, p.alpha, p.m = 3, 1.5, 8
    o = orc.Oracle(inst[0], p).iterate(3)
    tau, W, ch = o.get("tau"), o.get("W"), o.get("choice")
    assert len(np.unique(tau[:, :20])) > 3                    # several pheromone levels
    skipped = 0
    for i in range(0, 500, 7):
        for c in range(20):
            x = mpmath.power(mpmath.mpf(float(tau[i, c])), mpmath.mpf(1.5)) * mpmath.mpf(float(W[i, c]))
            ref = _fl32_of_exact(x, mpmath)
            if ref is None:
                skipped += 1
                continue
            assert ch[i, c] == ref, (i, c)
    assert skipped <= 2


# ---------------------------------------------------------------------------
# The ablation variants of Sec. V-D (kappa_mode) and the candidate density
# Edges/n of Sec. VI-A.

def test_fixed_kappa_one_weights(orc):
    """kappa_mode 1 ("fixed kappa = 1"): W = fl32(eta^2 * e) wherever ln e is
    below the clip; on the hand-worked row 0, eta = 8/c and e = 5, 3, 1, 1, 1."""
    mpmath = pytest.importorskip("mpmath")
    pts, H = _hand_instance()
    p = params(m=2, k=8, iterations=0, rho=0.2, kappa_mode=1)
    o = orc.Oracle(euclid(pts, H, symmetrize=0), p)
    assert o.scalars()["kappa"] == 1.0
    assert list(o.get("W")[0][:5]) == [np.float32(320.0), np.float32(48.0), np.float32(64.0 / 9.0),
                                       np.float32(4.0), np.float32(64.0 / 25.0)]
    inst, ps = synth.workload("tsp500")
    q = ps[0]
    q.iterations, q.kappa_mode = 0, 1
    o = orc.Oracle(inst[0], q)
    assert o.scalars()["kappa"] == 1.0
    _check_weights(o, q, mpmath, kappa=1.0)


def test_no_cap_kappa(orc):
    """kappa_mode 2 ("no cap"): the cap factor c_cap leaves eq. (kappa), so
    kappa * q90 = alpha * ln R and kappa is 1/c_cap times the default one."""
    mpmath = pytest.importorskip("mpmath")
    inst, ps = synth.workload("tsp500")
    p = ps[0]
    p.iterations = 0
    base = orc.Oracle(inst[0], p).scalars()
    for alpha in (1.0, 1.5):
        p.alpha, p.kappa_mode = alpha, 2
        o = orc.Oracle(inst[0], p)
        s = o.scalars()
        assert s["q90"] == base["q90"] and s["Rhat"] == base["Rhat"]
        assert s["kappa"] * s["q90"] == pytest.approx(alpha * math.log(s["Rhat"]), rel=1e-13)
        if alpha == 1.0:
            assert s["kappa"] == pytest.approx(2.0 * base["kappa"], rel=1e-14)
            _check_weights(o, p, mpmath)
    p.kappa_mode = 3
    with pytest.raises(ValueError):
        orc.Oracle(inst[0], p)


def test_edges_per_node(orc):
    """Edges/n = |{(i, j): h_ij > theta_h}| / (2n) over the heatmap as the decoder
    reads it (Sec. VI-A), counted here from the dense matrix."""
    pts, H = _hand_instance()
    o = orc.Oracle(euclid(pts, H, symmetrize=0), params(m=2, k=8, iterations=0, rho=0.2))
    assert o.scalars()["edges_per_n"] == 6 / 12
    o = orc.Oracle(euclid(pts, H, symmetrize=1), params(m=2, k=8, iterations=0, rho=0.2))
    Hs = (H + H.T) / 2
    assert o.scalars()["edges_per_n"] == np.count_nonzero(Hs > 1e-4) / 12
    inst = synth.euclid_instance(5, 300, K=12)
    Hd = np.zeros((300, 300))
    for i in range(300):
        Hd[i, inst.col[inst.rowptr[i]:inst.rowptr[i + 1]]] = inst.val[inst.rowptr[i]:inst.rowptr[i + 1]]
    Hs = (Hd + Hd.T) * 0.5
    o = orc.Oracle(inst, params(m=2, k=8, iterations=0, rho=0.2))
    assert o.scalars()["edges_per_n"] == np.count_nonzero(Hs > 1e-4) / 600
    o = orc.Oracle(euclid(pts), params(m=2, k=4, iterations=0, rho=0.2))
    assert o.scalars()["edges_per_n"] == 0.0
