"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

Bar (both sides evaluate every FP step in the same fixed order): integer and
index results bit-exact (candidate lists, tours, iteration-best ants);
floating-point prep arrays, lengths and pheromone bit-exact as well, which
is stricter than the 1e-6 relative pheromone tolerance the path promises.
"""
import dataclasses
import math

import numpy as np
import pytest

from helpers import atsp, dmat, euclid, is_perm, params
from paper_2601_19041_gb300 import synth

pytestmark = pytest.mark.gpu

TAU_RTOL = 1e-6      # stated pheromone tolerance; observed differences are 0


@pytest.fixture(scope="module")
def hac():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2601_19041_gb300 import build, heataco
    build.build()
    return heataco


def prep_equal(bt, b, o):
    for f, of in [("CAND", "cand"), ("CDIST", "cdist"), ("CONF", "conf"), ("BASE", "base"),
                  ("EVID", "evid"), ("W", "W"), ("NN_TOUR", "nn_tour"), ("TAU", "tau"),
                  ("CHOICE", "choice")]:
        g, r = bt.read(b, f), o.get(of)
        assert g.shape == r.shape, f
        assert np.array_equal(g, r), f"{f}: {np.argwhere(g != r)[:5]}"
    gs, os_ = bt.scalars(b), o.scalars()
    for key in ("q90", "Rhat", "kappa", "p_x", "L_nn", "tau_max64", "tau_min64", "tau_max",
                "tau_min", "n_lambda", "edges_per_n"):
        assert gs[key] == os_[key], key


def search_equal(bt, b, o, iters):
    tr = bt.read(b, "TRACE")
    assert np.array_equal(tr[:iters, 0].astype(np.int64), o.get("trace_ib")[:iters]), "ib ants"
    assert np.array_equal(tr[:iters, 1], o.get("trace_Lib")[:iters]), "L_ib"
    assert np.array_equal(tr[:iters, 2], o.get("trace_Lgb")[:iters]), "L_gb"
    if iters:
        assert np.array_equal(bt.read(b, "TOURS"), o.get("tours")), "tours"
        assert np.array_equal(bt.read(b, "LENS"), o.get("lens")), "lens"
        assert np.array_equal(bt.read(b, "IB_TOUR"), o.get("ib_tour")), "ib tour"
    gt, rt = bt.read(b, "TAU"), o.get("tau")
    assert np.allclose(gt, rt, rtol=TAU_RTOL, atol=0)
    assert np.array_equal(gt, rt), "tau bitwise"
    assert np.array_equal(bt.read(b, "CHOICE"), o.get("choice")), "choice"
    assert np.array_equal(bt.read(b, "GB_TOUR"), o.get("gb_tour")), "gb tour"
    gs, os_ = bt.scalars(b), o.scalars()
    assert gs["L_gb"] == os_["L_gb"]
    assert int(gs["n_fallback"]) == o.ints()["n_fallback"]


def run_case(hac, orc, insts, ps, iters=None, exec_=None):
    bt = hac.Batch(insts, ps, exec_)
    try:
        bt.sync()
        for b in range(len(insts)):
            prep_equal(bt, b, orc.Oracle(insts[b], dataclasses.replace(ps[b])))
        bt.run().sync()
        for b in range(len(insts)):
            o = orc.Oracle(insts[b], ps[b]).iterate(ps[b].iterations)
            search_equal(bt, b, o, ps[b].iterations)
        tours, lens = bt.results()
        for b in range(len(insts)):
            assert is_perm(tours[b], insts[b].n)
    finally:
        bt.close()


def _pts(seed, n):
    return np.random.default_rng(seed).random((n, 2)).astype(np.float32)


CASES = {
    "sym50nn_k20": lambda: (synth.euclid_instance(11, 300, K=50), params(m=20, k=20, iterations=12, rho=0.2, seed=5)),
    "sym10nn_k10_ragged": lambda: (synth.euclid_instance(12, 257, K=10), params(m=13, k=10, iterations=10, rho=0.2, seed=6)),
    "k32": lambda: (synth.euclid_instance(13, 150, K=40), params(m=9, k=32, iterations=8, rho=0.2, seed=7)),
    "k7_pad": lambda: (synth.euclid_instance(14, 123, K=12), params(m=7, k=7, iterations=9, rho=0.8, seed=8)),
    "n_le_k": lambda: (synth.euclid_instance(15, 6, K=3), params(m=5, k=20, iterations=6, rho=0.2, seed=9)),
    "n3": lambda: (euclid(_pts(3, 3)), params(m=4, k=20, iterations=3, rho=0.2, seed=1)),
    "empty_heatmap": lambda: (euclid(_pts(16, 140)), params(m=10, k=20, iterations=8, rho=0.2, seed=10)),
    "dense_heatmap": lambda: (euclid(_pts(17, 70), np.where(np.eye(70) > 0, 0, np.random.default_rng(1).random((70, 70)))),
                              params(m=8, k=20, iterations=6, rho=0.2, seed=11)),
    "asym_no_symmetrize": lambda: (dataclasses.replace(synth.euclid_instance(18, 180, K=20), symmetrize=0),
                                   params(m=10, k=12, iterations=7, rho=0.2, seed=12)),
    "fp16_heatmap": lambda: (synth.euclid_instance(19, 222, K=50, dtype=np.float16), params(m=12, k=20, iterations=7, rho=0.2, seed=13)),
    "baseline_row_scope": lambda: (synth.euclid_instance(20, 160, K=50), params(m=8, k=8, iterations=6, rho=0.2, seed=14, baseline_scope=1)),
    "alpha_beta_powers": lambda: (synth.euclid_instance(21, 130, K=30), params(m=8, k=16, iterations=6, rho=0.3, seed=15, alpha=1.5, beta=3.0)),
    "duplicate_points": lambda: (euclid(np.repeat(_pts(22, 40), 2, axis=0)), params(m=6, k=8, iterations=5, rho=0.2, seed=16)),
    "atsp": lambda: (synth.atsp_instance(23, 200, K=30), params(m=10, k=20, iterations=8, rho=0.2, degree_target=1, seed=17)),
    "two_opt": lambda: (synth.euclid_instance(24, 350, K=10), params(m=10, k=10, iterations=6, rho=0.2, local_search=1, seed=18)),
    # an exact 17 x 17 grid: equal edge lengths make many gains exactly zero, which
    # the FP32 estimate cannot decide and the FP64 test does; an odd list length
    # leaves a partial group of four
    "two_opt_grid": lambda: (euclid(np.stack(np.meshgrid(np.arange(17), np.arange(17)), -1).reshape(-1, 2) / 16.0),
                             params(m=10, k=10, iterations=6, rho=0.2, local_search=1, ls_k=7, seed=23)),
    # zero-length edges and the longest neighbour list
    "two_opt_dup": lambda: (euclid(np.repeat(_pts(28, 45), 2, axis=0)),
                            params(m=8, k=8, iterations=5, rho=0.2, local_search=1, ls_k=32, seed=24)),
    # the ablation variants of Sec. V-D: fixed kappa = 1, and kappa without the cap factor
    "kappa_fixed_one": lambda: (synth.euclid_instance(29, 240, K=50), params(m=12, k=20, iterations=7, rho=0.2, seed=25, kappa_mode=1)),
    "kappa_no_cap": lambda: (synth.euclid_instance(30, 260, K=50), params(m=12, k=20, iterations=7, rho=0.2, seed=26, kappa_mode=2)),
    # the SoftDist control heatmap (Sec. V-C): a softmax of negated distances
    "softdist": lambda: (synth.softdist_instance(32, 280), params(m=12, k=20, iterations=7, rho=0.2, seed=27)),
    # 3-opt (Sec. III-D) on T_ib and T_NN; on every ant
    "three_opt": lambda: (synth.euclid_instance(33, 260, K=10), params(m=10, k=10, iterations=6, rho=0.2, local_search=3, seed=28)),
    "three_opt_grid": lambda: (euclid(np.stack(np.meshgrid(np.arange(13), np.arange(13)), -1).reshape(-1, 2) / 12.0),
                               params(m=8, k=10, iterations=5, rho=0.2, local_search=3, ls_k=9, seed=29)),
    "three_opt_every_ant": lambda: (synth.euclid_instance(34, 140, K=10), params(m=7, k=10, iterations=4, rho=0.2, local_search=4, ls_k=12, seed=30)),
    # the directed 2-opt of the ATSP (Sec. III-D): on T_ib and T_NN; on every ant
    "atsp_two_opt": lambda: (synth.atsp_instance(35, 180, K=20), params(m=8, k=12, iterations=5, rho=0.2, degree_target=1, local_search=1, ls_k=10, seed=31)),
    "atsp_two_opt_every_ant": lambda: (synth.atsp_instance(36, 90, K=15), params(m=6, k=10, iterations=4, rho=0.2, degree_target=1, local_search=2, ls_k=8, seed=32)),
    "clustered": lambda: (synth.euclid_instance(25, 300, K=50, family="gmm"), params(m=12, k=20, iterations=6, rho=0.2, seed=19)),
    "grid": lambda: (synth.euclid_instance(26, 289, K=50, family="grid"), params(m=12, k=20, iterations=6, rho=0.2, seed=20)),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_case_parity(hac, orc, name):
    inst, p = CASES[name]()
    run_case(hac, orc, [inst], [p])


@pytest.mark.parametrize("apw,wpb,graph,fbl", [(1, 4, 1, 0), (2, 8, 0, 32), (4, 2, 1, 32), (4, 8, 0, 0),
                                              (16, 4, 1, 32), (16, 8, 0, 0), (32, 4, 1, 32), (32, 2, 0, 0)])
def test_exec_variants_do_not_change_results(hac, orc, apw, wpb, graph, fbl):
    inst = synth.euclid_instance(31, 410, K=50)
    p = params(m=21, k=20, iterations=23, rho=0.2, seed=3)
    run_case(hac, orc, [inst], [p], exec_=hac.make_exec(apw, wpb, graph, fallback_list=fbl))


FUSED = [dict(apw=2, clog=0, fbl=32), dict(apw=4, clog=1, fbl=0), dict(apw=4, clog=3, fbl=32),
         dict(apw=2, clog=2, fbl=32), dict(apw=16, clog=0, fbl=32), dict(apw=16, clog=1, fbl=0),
         dict(apw=16, clog=3, fbl=32), dict(apw=32, clog=0, fbl=32), dict(apw=32, clog=2, fbl=0)]


@pytest.mark.parametrize("cfg", FUSED, ids=lambda c: f"apw{c['apw']}_C{1 << c['clog']}_fbl{c['fbl']}")
@pytest.mark.parametrize("name", ["sym50nn_k20", "sym10nn_k10_ragged", "k32", "k7_pad", "n3",
                                  "empty_heatmap", "atsp", "two_opt", "two_opt_grid", "alpha_beta_powers",
                                  "kappa_no_cap", "three_opt", "three_opt_every_ant", "atsp_two_opt",
                                  "atsp_two_opt_every_ant"])
def test_fused_kernel_parity(hac, orc, name, cfg):
    inst, p = CASES[name]()
    if cfg["apw"] == 32 and p.local_search in (2, 4):
        pytest.skip("local search on every ant needs ant-major tours")
    ex = hac.make_exec(cfg["apw"], 0, 1, fused=1, fallback_list=cfg["fbl"], cluster_log2=cfg["clog"])
    run_case(hac, orc, [inst], [p], exec_=ex)


def test_fused_mixed_batch_groups(hac, orc):
    # different sizes land in different cluster-size groups that run concurrently
    insts, ps = [], []
    # n = 1400 fits one CTA only without its lookup lists: the one-CTA group then
    # reads every member's lists from global memory
    for b, (n, k, m) in enumerate([(90, 20, 9), (1900, 20, 40), (4000, 12, 20), (333, 10, 17), (12, 8, 5),
                                   (1400, 20, 24)]):
        insts.append(synth.euclid_instance(70 + b, n, K=20))
        ps.append(params(m=m, k=k, iterations=3 + b, rho=0.2, seed=170 + b))
    run_case(hac, orc, insts, ps, exec_=hac.make_exec(4, 0, 1, fused=1, fallback_list=32))
    run_case(hac, orc, insts, ps, exec_=hac.make_exec(32, 0, 1, fused=1, fallback_list=32))
    run_case(hac, orc, insts, ps, exec_=hac.make_exec(16, 0, 1, fused=1, fallback_list=32))
    run_case(hac, orc, insts, ps, exec_=hac.make_exec(32, 4, 1, fused=0, fallback_list=32))
    run_case(hac, orc, insts, ps, exec_=hac.make_exec(16, 4, 1, fused=0, fallback_list=32))
    # ants per warp chosen per instance: 4 on one CTA where the table, masks and
    # coordinates fit, else 2 on a cluster
    run_case(hac, orc, insts, ps, exec_=hac.make_exec(0, 0, 1, fused=1, fallback_list=32))
    run_case(hac, orc, insts, ps, exec_=hac.make_exec(0, 0, 1, fused=1, fallback_list=0))


def test_mixed_batch_parity(hac, orc):
    insts, ps = [], []
    for b, (n, k, m, kind, ls) in enumerate([(120, 20, 9, 0, 0), (333, 10, 17, 0, 1), (64, 8, 4, 1, 0),
                                              (501, 20, 33, 0, 0), (7, 20, 3, 0, 0)]):
        if kind == 1:
            insts.append(synth.atsp_instance(40 + b, n, K=20))
            ps.append(params(m=m, k=k, iterations=5 + b, rho=0.2, degree_target=1, seed=100 + b))
        else:
            insts.append(synth.euclid_instance(40 + b, n, K=20))
            ps.append(params(m=m, k=k, iterations=5 + b, rho=0.2, local_search=ls, seed=100 + b))
    run_case(hac, orc, insts, ps)
    # the per-step kernels with the instances split into parts on their own streams
    for parts, apw, graph in ((2, 4, 1), (3, 16, 0), (5, 1, 1)):
        run_case(hac, orc, insts, ps, exec_=hac.make_exec(apw, 4, graph, fallback_list=32, parts=parts))


def test_iterate_in_steps_equals_run(hac, orc):
    inst = synth.euclid_instance(50, 200, K=50)
    p = params(m=16, k=20, iterations=27, rho=0.2, seed=4)
    with hac.Batch([inst], [p]) as bt:
        for chunk in (1, 2, 10, 3, 11, 50):
            bt.iterate(chunk)
        bt.sync()
        o = orc.Oracle(inst, p).iterate(27)
        search_equal(bt, 0, o, 27)
        assert bt.scalars(0)["t"] == 27


def test_batch_membership_does_not_change_results(hac):
    insts, ps = synth.workload("batch128", count=6)
    for p in ps:
        p.iterations = 15
    _, lens_all = hac.solve_batch(insts, ps)
    for b in (0, 3, 5):
        t1, l1 = hac.solve(insts[b], ps[b])
        assert l1 == lens_all[b]


def test_full_size_tsp500(hac, orc):
    insts, ps = synth.workload("tsp500")
    run_case(hac, orc, insts, ps)
    run_case(hac, orc, insts, ps, exec_=_layout(hac, insts, ps, "autotuned"))
    run_case(hac, orc, insts, ps, exec_=hac.make_exec(**FIXED_EXEC["apw4"]))


_ORACLE_RUNS = {}


def _oracle_many(orc, insts, ps):
    import concurrent.futures as cf
    def one(b):
        return orc.Oracle(insts[b], ps[b]).iterate(ps[b].iterations)
    with cf.ThreadPoolExecutor(max_workers=8) as ex:   # the C oracle releases the GIL
        return list(ex.map(one, range(len(insts))))


# fixed layouts run at full size besides the autotuner's pick (which is what
# bench.py times): 4 ants per warp on the fewest CTAs, and 2 ants per warp on
# clusters of at least 2 CTAs
FIXED_EXEC = {"apw4": dict(ants_per_warp=4, fused=1, fallback_list=32),
              "apw2_C2": dict(ants_per_warp=2, fused=1, fallback_list=32, cluster_log2=1)}


def _layout(hac, insts, ps, which):
    if which == "autotuned":                       # the layout bench.py picks and times
        ex, _ = hac.autotune(insts, ps, trial_iters=10, inputs_on_device=False)
        return ex
    return hac.make_exec(**FIXED_EXEC[which])


@pytest.mark.parametrize("layout", ["autotuned", "apw4", "apw2_C2"])
@pytest.mark.parametrize("name,sample", [("batch128", (0, 37, 90, 127)), ("atsp1000", (0, 31, 63))])
def test_full_size_workload_sampled(hac, orc, name, sample, layout):
    insts, ps = synth.workload(name)
    bt = hac.Batch(insts, ps, _layout(hac, insts, ps, layout))
    try:
        bt.run().sync()
        key = (name, sample)
        if key not in _ORACLE_RUNS:                # the same for every layout
            _ORACLE_RUNS[key] = _oracle_many(orc, [insts[b] for b in sample], [ps[b] for b in sample])
        for b, o in zip(sample, _ORACLE_RUNS[key]):
            search_equal(bt, b, o, ps[b].iterations)
    finally:
        bt.close()


@pytest.mark.parametrize("layout", ["autotuned", "apw4"])
def test_full_size_tsp10k_two_opt_sampled(hac, orc, layout):
    insts, ps = synth.workload("tsp10k_2opt")
    bt = hac.Batch(insts, ps, _layout(hac, insts, ps, layout))
    try:
        bt.run().sync()
        if "tsp10k" not in _ORACLE_RUNS:
            _ORACLE_RUNS["tsp10k"] = _oracle_many(orc, [insts[5]], [ps[5]])[0]
        o = _ORACLE_RUNS["tsp10k"]
        search_equal(bt, 5, o, ps[5].iterations)
        D_ok = is_perm(bt.read(5, "GB_TOUR"), 10000)
        assert D_ok
    finally:
        bt.close()


# ------------------------------------------------------------------ MMAS schedule (Sec. III-B)

def _schedule_batch():
    rng = np.random.default_rng(3)
    insts = [euclid(rng.random((10, 2))),                                  # restarts within 700 iterations
             synth.euclid_instance(81, 60, K=10),
             synth.atsp_instance(82, 14, K=8),
             synth.euclid_instance(83, 40, K=10)]
    ps = [params(m=10, k=8, iterations=700, rho=0.2, seed=5, schedule=1),
          params(m=12, k=10, iterations=420, rho=0.2, seed=6, schedule=1),
          params(m=8, k=6, iterations=650, rho=0.2, degree_target=1, seed=7, schedule=1),
          params(m=8, k=10, iterations=400, rho=0.2, local_search=1, ls_k=10, seed=8, schedule=1)]
    return insts, ps


@pytest.mark.parametrize("ex", [dict(apw=4, fused=1, fbl=32, clog=0), dict(apw=32, fused=1, fbl=32, clog=1),
                                dict(apw=2, fused=0, fbl=32, clog=0), dict(apw=1, fused=0, fbl=0, clog=0)],
                         ids=lambda e: f"apw{e['apw']}_fused{e['fused']}_C{1 << e['clog']}")
def test_mmas_schedule_parity(hac, orc, ex):
    """Restart-best tour, u_gb elite choice, branching-factor restarts: the
    per-iteration trace (ib ant, L_ib, L_gb, L_rb, elite/restart code), the
    pheromone and T_gb bit-exact against the oracle."""
    insts, ps = _schedule_batch()
    run_case(hac, orc, insts, ps,
             exec_=hac.make_exec(ex["apw"], 8 if not ex["fused"] else 0, 1, fused=ex["fused"],
                                 fallback_list=ex["fbl"], cluster_log2=ex["clog"]))
    bt = hac.Batch(insts, ps, hac.make_exec(ex["apw"], 8 if not ex["fused"] else 0, 1, fused=ex["fused"],
                                            fallback_list=ex["fbl"], cluster_log2=ex["clog"]))
    try:
        bt.run().sync()
        restarts = 0
        for b in range(len(insts)):
            o = orc.Oracle(insts[b], ps[b]).iterate(ps[b].iterations)
            tr = bt.read(b, "TRACE")
            I = ps[b].iterations
            assert np.array_equal(tr[:I, 3], o.get("trace_Lrb")[:I]), b
            assert np.array_equal(tr[:I, 4].astype(np.int64), o.get("trace_code")[:I]), b
            gs = bt.scalars(b)
            assert gs["n_restarts"] == o.ints()["n_restarts"]
            assert gs["u_gb"] == o.ints()["u_gb"] and gs["t_restart"] == o.ints()["t_restart"]
            restarts += int(gs["n_restarts"])
        assert restarts >= 1
    finally:
        bt.close()


# ------------------------------------------------------------------ 2-opt on every ant (Algorithm 1's local search)

@pytest.mark.parametrize("ex", [dict(apw=4, fused=1, clog=0), dict(apw=2, fused=1, clog=1),
                                dict(apw=4, fused=0, clog=0), dict(apw=1, fused=0, clog=0)],
                         ids=lambda e: f"apw{e['apw']}_fused{e['fused']}_C{1 << e['clog']}")
def test_two_opt_every_ant_parity(hac, orc, ex):
    insts = [synth.euclid_instance(91, 300, K=10), synth.euclid_instance(92, 77, K=10),
             synth.euclid_instance(93, 150, K=20)]
    ps = [params(m=9, k=10, iterations=5, rho=0.2, local_search=2, ls_k=10, seed=21),
          params(m=6, k=8, iterations=40, rho=0.2, local_search=2, ls_k=8, seed=22, schedule=1),
          params(m=5, k=12, iterations=6, rho=0.2, local_search=0, seed=23)]
    run_case(hac, orc, insts, ps,
             exec_=hac.make_exec(ex["apw"], 8 if not ex["fused"] else 0, 1, fused=ex["fused"], fallback_list=32,
                                 cluster_log2=ex["clog"]))


def test_two_opt_every_ant_rejects_lane_mode(hac):
    inst = synth.euclid_instance(94, 50, K=10)
    p = params(m=4, k=8, iterations=2, rho=0.2, local_search=2, ls_k=8, seed=1)
    with pytest.raises(hac.HeatACOError) as e:
        hac.Batch([inst], [p], hac.make_exec(32, 0, 1, fused=1))
    assert e.value.status == hac.HAC_EUNSUPPORTED


def test_hac_solve_host_buffers_without_workspace(hac, orc):
    """The one-shot call of the decoding problem (Sec. II-B, Algorithm 1) with
    host inputs and no workspace: the library takes one from the stream-ordered
    pool; tour, length and the stats equal the oracle's."""
    for inst, p in (CASES["sym50nn_k20"](), CASES["two_opt"](), CASES["atsp"]()):
        tour, length, st = hac.hac_solve(inst, p)
        o = orc.Oracle(inst, p).iterate(p.iterations)
        assert np.array_equal(tour, o.get("gb_tour"))
        assert length == o.scalars()["L_gb"]
        assert st["iterations"] == p.iterations
        assert st["ant_steps"] == p.m * inst.n * p.iterations
        assert st["fallback_steps"] == o.ints()["n_fallback"]
        assert st["kappa"] == o.scalars()["kappa"]
        assert st["edges_per_n"] == o.scalars()["edges_per_n"]
        assert st["L_nn"] == o.scalars()["L_nn"]
        assert st["seconds"] > 0.0
