"""Serving (continuous batching) through the hac_server_* calls.

A request must decode to the same tour and length alone and in a mix: the
mix here has requests of different sizes, kinds and iteration counts, some
submitted while others are already several ticks into their search.  Each
result is checked against the CPU oracle (bit-exact, as for the batch path)
and against hac_solve.  Admission follows free workspace memory and slots.
"""
import numpy as np
import pytest

from helpers import atsp, is_perm
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


def _requests():
    rng = np.random.default_rng(7)
    reqs = []
    for r, (n, it, fam) in enumerate([(120, 7, "uniform"), (333, 12, "gmm"), (64, 0, "grid"),
                                      (700, 9, "uniform"), (250, 15, "grid"), (90, 4, "gmm")]):
        inst = synth.euclid_instance(900 + r, n, K=20, family=fam, dtype=np.float16 if r % 2 else np.float32)
        reqs.append((inst, synth.Params(m=int(rng.integers(8, 40)), k=int(rng.choice([8, 10, 20])),
                                        iterations=it, rho=0.2, seed=900 + r)))
    cost = synth.atsp_instance(77, 150)
    reqs.append((cost, synth.Params(m=20, k=12, iterations=8, rho=0.2, degree_target=1, seed=77)))
    ls = synth.euclid_instance(78, 200, K=10)
    reqs.append((ls, synth.Params(m=16, k=10, iterations=6, rho=0.2, local_search=1, seed=78)))
    # the MMAS schedule with restarts, and 2-opt on every ant
    reqs.append((synth.euclid_instance(79, 10, K=5), synth.Params(m=10, k=8, iterations=320, rho=0.2, seed=79,
                                                                   schedule=1)))
    reqs.append((synth.euclid_instance(80, 150, K=10), synth.Params(m=8, k=10, iterations=5, rho=0.2, seed=80,
                                                                    local_search=2, ls_k=10)))
    return reqs


def _drain(srv, tickets, out, max_ticks=1000, max_seconds=120.0):
    import time
    t0 = time.perf_counter()
    ticks = 0
    while ticks < max_ticks or time.perf_counter() - t0 < max_seconds:
        for t in list(tickets):
            res = srv.poll(t)
            if res is not None:
                out[t] = res
                tickets.remove(t)
        if not tickets:
            return
        srv.tick()
        ticks += 1
        if ticks >= max_ticks:
            time.sleep(0.001)     # a large request may still be in its preparation
    raise AssertionError("requests did not finish")


@pytest.mark.parametrize("apw,ipt,spt,smin,sapw", [(4, 3, 0, 0, 1), (32, 5, 1500, 0, 1), (2, 4, 0, 0, 1),
                                                   (4, 3, 1500, 300, 1), (32, 4, 0, 100, 2), (4, 5, 0, 3, 4)])
def test_mix_equals_alone_and_oracle(hac, orc, apw, ipt, spt, smin, sapw):
    reqs = _requests()
    if apw == 32:   # 2-opt on every ant needs ant-major tours
        reqs = [(i, p) for i, p in reqs if p.local_search != 2]
    srv = hac.Server(64 << 20, max_slots=10, iters_per_tick=ipt, max_n=1000, steps_per_tick=spt,
                     step_min_n=smin, step_ants_per_warp=sapw, step_warps_per_block=4 if sapw == 4 else 8,
                     exec_=hac.make_exec(ants_per_warp=apw, fused=1, fallback_list=32 if apw != 2 else 0))
    try:
        tickets, order, out = [], [], {}
        # staggered admission: two requests, then one more after every tick
        for q, (inst, p) in enumerate(reqs):
            t = srv.submit(inst, p)
            assert t is not None
            tickets.append(t)
            order.append(t)
            if q >= 1:
                srv.tick()
        _drain(srv, tickets, out)
        assert srv.stats(device_error=True) == dict(resident=0, finished=0, free_bytes=srv.stats()["free_bytes"],
                                                    device_error=0)
    finally:
        srv.close()
    for t, (inst, p) in zip(order, reqs):
        tour, length = out[t]
        assert is_perm(tour, inst.n)
        t_alone, l_alone = hac.solve(inst, p)
        assert np.array_equal(tour, t_alone), (inst.n, p)
        assert length == l_alone
        o = orc.Oracle(inst, p).iterate(p.iterations)
        assert np.array_equal(tour, o.get("gb_tour"))
        assert length == o.scalars()["L_gb"]


def test_admission_by_memory_and_slots(hac):
    a = synth.euclid_instance(11, 400, K=20)
    b = synth.euclid_instance(12, 300, K=20)
    pa = synth.Params(m=16, k=10, iterations=6, rho=0.2, seed=11)
    pb = synth.Params(m=16, k=10, iterations=4, rho=0.2, seed=12)
    need_a = hac.hac_server_request_bytes(a, pa)
    need_b = hac.hac_server_request_bytes(b, pb)
    assert need_a > need_b > 0
    # room for one request of either size, not for both
    srv = hac.Server(need_a + need_b // 2 + (64 << 10), max_slots=4, iters_per_tick=2, max_n=500,
                     exec_=hac.make_exec(fused=1))
    try:
        free0 = srv.stats()["free_bytes"]
        assert need_a <= free0 < need_a + need_b
        ta = srv.submit(a, pa)
        assert ta is not None
        assert srv.submit(b, pb) is None              # HAC_EBUSY: no region free
        assert srv.stats()["resident"] == 1
        assert srv.poll(ta) is None                   # HAC_EBUSY: still running
        out = {}
        _drain(srv, [ta], out)
        assert srv.stats()["free_bytes"] == free0     # region returned and coalesced
        tb = srv.submit(b, pb)
        assert tb is not None
        _drain(srv, [tb], out)
        with pytest.raises(hac.HeatACOError):
            srv.poll(tb)                              # ticket already collected
    finally:
        srv.close()
    assert np.array_equal(out[ta][0], hac.solve(a, pa)[0])
    assert np.array_equal(out[tb][0], hac.solve(b, pb)[0])

    srv = hac.Server(64 << 20, max_slots=1, iters_per_tick=4, max_n=500, exec_=hac.make_exec(fused=1))
    try:
        t1 = srv.submit(b, pb)
        assert srv.submit(b, pb) is None              # HAC_EBUSY: no slot free
        with pytest.raises(hac.HeatACOError):
            srv.submit(synth.euclid_instance(13, 600, K=20), pb)   # n > max_n
        _drain(srv, [t1], {})
        assert srv.submit(b, pb) is not None
    finally:
        srv.close()


def test_atsp_request_alone_in_server(hac, orc):
    inst = atsp(np.random.default_rng(5).random((40, 40)) + 0.1)
    p = synth.Params(m=12, k=8, iterations=5, rho=0.2, degree_target=1, seed=5)
    srv = hac.Server(16 << 20, max_slots=2, iters_per_tick=2, max_n=100, exec_=hac.make_exec(fused=1))
    try:
        t = srv.submit(inst, p)
        out = {}
        _drain(srv, [t], out)
    finally:
        srv.close()
    o = orc.Oracle(inst, p).iterate(p.iterations)
    assert np.array_equal(out[t][0], o.get("gb_tour"))
    assert out[t][1] == o.scalars()["L_gb"]


def test_upload_ring_wraps_without_corrupting_inputs(hac):
    # 24 ATSP requests of ~4.3 MB of inputs each: more than the 64 MB pinned
    # upload ring, so submission wraps around it and waits for earlier copies
    insts = [synth.atsp_instance(300 + q, 1000, K=20) for q in range(24)]
    ps = [synth.Params(m=8, k=8, iterations=2, rho=0.2, degree_target=1, seed=300 + q) for q in range(24)]
    srv = hac.Server(1 << 30, max_slots=32, iters_per_tick=1, max_n=1000, exec_=hac.make_exec(fused=1),
                     step_min_n=900)
    try:
        tickets = [srv.submit(i, p) for i, p in zip(insts, ps)]
        assert all(t is not None for t in tickets)
        out = {}
        _drain(srv, list(tickets), out)
    finally:
        srv.close()
    for t, i, p in zip(tickets, insts, ps):
        ref_t, ref_l = hac.solve(i, p)
        assert np.array_equal(out[t][0], ref_t)
        assert out[t][1] == ref_l


def test_full_size_request_on_the_per_step_route(hac, orc):
    """A stream-sized request (n = 5000, FP16 heatmap) goes to the per-step
    kernels (step_min_n = 3000, as the serving benchmark runs them) while a
    small one runs in the cluster kernel; both equal the oracle (few
    iterations keep the oracle cheap)."""
    big = synth.euclid_instance(40123, 5000, K=50, family="gmm", dtype=np.float16)
    pbig = synth.Params(m=64, k=20, iterations=3, rho=0.2, seed=40123)
    small = synth.euclid_instance(40124, 500, K=50, family="grid", dtype=np.float16)
    psmall = synth.Params(m=64, k=20, iterations=5, rho=0.2, seed=40124)
    srv = hac.Server(1 << 30, max_slots=8, iters_per_tick=10, max_n=10000, steps_per_tick=4000, step_min_n=3000,
                     step_ants_per_warp=1, step_warps_per_block=8,
                     exec_=hac.make_exec(ants_per_warp=4, fused=1, fallback_list=32))
    try:
        tb = srv.submit(big, pbig)
        ts = srv.submit(small, psmall)
        out = {}
        _drain(srv, [tb, ts], out)
    finally:
        srv.close()
    for t, (inst, p) in ((tb, (big, pbig)), (ts, (small, psmall))):
        o = orc.Oracle(inst, p).iterate(p.iterations)
        assert np.array_equal(out[t][0], o.get("gb_tour"))
        assert out[t][1] == o.scalars()["L_gb"]
