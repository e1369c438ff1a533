"""The nearest-unvisited lookup lists built on the GPU (the 32-entry list and
the second level of the next 256 nodes), compared entry by entry with their
definition written out in numpy: for node i, the nodes u != i, not in C_i when
every candidate's choice value stays positive, in the order of the FP32 key
(squared distance from FP32 coordinate differences, or the FP32 cost) and then
of the node index.  The construction kernels take the first unvisited node of
these lists as the nearest unvisited node of the fallback (Alg. 2), so the
lists must be exact prefixes of that order, ties included."""
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


def _keys(inst, i):
    if inst.kind == 1:
        return inst.cost[i].astype(np.float32)
    xy = inst.coords.astype(np.float32)
    dx = (xy[:, 0] - xy[i, 0]).astype(np.float32)     # one FP32 rounding per operation
    dy = (xy[:, 1] - xy[i, 1]).astype(np.float32)
    return (dx * dx).astype(np.float32) + (dy * dy).astype(np.float32)


def _expected(inst, cand, excl):
    n = inst.n
    fbl = np.full((n, 32), -1, np.int64)
    fbl2 = np.full((n, 256), 0xffff, np.int64)
    for i in range(n):
        ok = np.ones(n, bool)
        ok[i] = False
        if excl:
            c = cand[i]
            ok[c[c >= 0]] = False
        u = np.nonzero(ok)[0]
        order = u[np.lexsort((u, _keys(inst, i)[u]))]
        fbl[i, :min(32, order.size)] = order[:32]
        rest = order[32:288]
        fbl2[i, :rest.size] = rest
    return fbl, fbl2


def _lattice_instance(side, seed):
    # exact lattice: many equal keys, so the index order of ties matters
    g = np.arange(side * side)
    pts = np.stack([(g % side) / side, (g // side) / side], 1).astype(np.float32)
    rng = np.random.default_rng(seed)
    nbr, nd = synth.knn_euclid(pts, 20)
    rowptr, col, val = synth.knn_heatmap(rng, nbr, nd, np.float32)
    return synth.Instance(n=side * side, kind=0, coords=pts, cost=None, rowptr=rowptr, col=col, val=val,
                          symmetrize=1, seed=seed)


CASES = {
    "uniform_700": lambda: (synth.euclid_instance(901, 700, K=50), 20),
    "lattice_900": lambda: (_lattice_instance(30, 902), 20),
    "atsp_400": lambda: (synth.atsp_instance(903, 400, K=50), 20),
    "small_40": lambda: (synth.euclid_instance(904, 40, K=20), 10),     # fewer than 288 nodes
    "tiny_5": lambda: (synth.euclid_instance(905, 5, K=4), 2),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_lookup_lists_equal_their_definition(hac, name):
    inst, k = CASES[name]()
    p = synth.Params(m=8, k=k, iterations=1, rho=0.2, seed=7,
                     degree_target=1 if inst.kind == 1 else 2)
    ex = hac.make_exec(4, 0, 0, fallback_list=32)
    with hac.Batch([inst], [p], ex) as bt:
        cand = bt.read(0, "CAND")
        W = bt.read(0, "W")
        tau_min = np.float32(bt.scalars(0)["tau_min"])
        excl = bool(np.all((tau_min * W[cand >= 0]).astype(np.float32) > 0))
        got1 = bt.read(0, "FBL").astype(np.int64)
        got2 = bt.read(0, "FBL2").astype(np.int64)
    want1, want2 = _expected(inst, cand, excl)
    assert np.array_equal(got1, want1)
    assert np.array_equal(got2, want2)


def test_no_second_level_without_lists(hac):
    inst = synth.euclid_instance(906, 100, K=20)
    p = synth.Params(m=8, k=10, iterations=1, rho=0.2, seed=3)
    with hac.Batch([inst], [p], hac.make_exec(4, 0, 0, fallback_list=0)) as bt:
        with pytest.raises(hac.HeatACOError):
            bt.read(0, "FBL2")
