"""The autotuner and the CUDA-graph replay of the fused kernel change no result.

hac_batch_autotune must return one of its candidate layouts, and decoding with
it must give exactly the default layout's tours.  The fused path with graphs
on (captured fork/join of the cluster-size groups, replayed; re-captured when
the iteration count of a call changes) must match the path without graphs,
iteration chunk by iteration chunk, and both must match the oracle.
"""
import numpy as np
import pytest

from paper_2601_19041_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hac():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2601_19041_gb300 import build, heataco
    build.build()
    return heataco


def _mixed():
    sizes = (150, 420, 900, 2600)
    insts = [synth.euclid_instance(500 + q, n, K=30) for q, n in enumerate(sizes)]
    ps = [synth.Params(m=24, k=20, iterations=14, rho=0.2, seed=500 + q) for q in range(len(sizes))]
    return insts, ps


def test_autotune_returns_a_candidate_with_identical_results(hac):
    insts, ps = _mixed()
    best, ms = hac.autotune(insts, ps, trial_iters=4)
    assert ms > 0.0
    assert best.use_graph == 1
    if best.fused:
        assert best.ants_per_warp in (2, 4, 32) and best.cluster_log2 in (0, 1, 2)
        assert best.fallback_list in (0, 32)
    else:
        assert best.ants_per_warp in (1, 2, 4) and best.warps_per_block in (4, 8)
    t_best, l_best = hac.solve_batch(insts, ps, best)
    t_def, l_def = hac.solve_batch(insts, ps, hac.make_exec())
    for a, b in zip(t_best, t_def):
        assert np.array_equal(a, b)
    assert np.array_equal(l_best, l_def)


@pytest.mark.parametrize("apw", [4, 32])
def test_fused_graph_replay_matches_direct_launches(hac, orc, apw):
    insts, ps = _mixed()
    runs = {}
    for graph in (0, 1):
        ex = hac.make_exec(apw, 0, graph, fused=1, fallback_list=32)
        with hac.Batch(insts, ps, ex) as bt:
            for chunk in (3, 3, 5, 9):       # graph captured for 3, replayed, re-captured for 5, clamped
                bt.iterate(chunk)
            bt.sync()
            runs[graph] = ([bt.read(b, "TAU") for b in range(len(insts))], bt.results())
            assert bt.launches() > 0
    (tau0, (t0, l0)), (tau1, (t1, l1)) = runs[0], runs[1]
    for b in range(len(insts)):
        assert np.array_equal(tau0[b], tau1[b])
        assert np.array_equal(t0[b], t1[b])
    assert np.array_equal(l0, l1)
    o = orc.Oracle(insts[1], ps[1]).iterate(ps[1].iterations)
    assert np.array_equal(t1[1], o.get("gb_tour"))
    assert l1[1] == o.scalars()["L_gb"]
