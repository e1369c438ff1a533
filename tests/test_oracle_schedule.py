"""Oracle pins for the MMAS machinery that HeatACO keeps (Sec. III-B,
Algorithm 1): the u_gb elite schedule, the restart-best tour, the branching
factor and the restarts.

The paper fixes: the depositing tour alternates between T_ib and T_rb with a
period u_gb that shrinks from 25 to 1; a check every 100 iterations resets
the trails to tau_max and forgets T_rb (keeping T_gb) when T_rb is more than
250 iterations old and the branching factor (band 0.05) is under 1 + 1e-5.
The checks below derive each of these from the run's own trace and from
pheromone matrices of known form."""
import numpy as np
import pytest

from helpers import euclid, params


def test_ugb_tightens_from_25_to_1(orc):
    u = [orc.ugb(s) for s in range(0, 2000)]
    assert u[0] == 25 and u[-1] == 1
    assert all(a >= b for a, b in zip(u, u[1:]))


def test_branching_factor_of_known_matrices(orc):
    n, kp = 7, 12
    cand = np.tile(np.arange(kp, dtype=np.int32), (n, 1))
    cand[:, 10:] = -1                                   # k_eff = 10, two padding slots
    tau = np.full((n, kp), 0.25, np.float32)
    tau[:, 10:] = 1e30                                  # padding never counts
    assert orc.branching(tau, cand, 2) == 10 / 2        # all equal: every real slot
    conv = np.full((n, kp), 0.01, np.float32)           # converged: d* slots at tau_max
    conv[:, 3] = 2.0
    conv[:, 7] = 2.0
    conv[:, 10:] = 1e30
    assert orc.branching(conv, cand, 2) == 1.0
    lin = np.arange(1, 11, dtype=np.float32)[None, :].repeat(n, 0)   # 1..10 per row
    lin = np.concatenate([lin, np.zeros((n, 2), np.float32)], 1)
    # cut = 1 + 0.05 * 9 = 1.45: the slots 2..10 count, 9 per row
    assert orc.branching(lin, cand, 1) == 9.0


def _run(orc, inst, p):
    o = orc.Oracle(inst, p)
    rows = []
    real = o.get("cand") >= 0
    for t in range(1, p.iterations + 1):
        tau0 = o.get("tau").copy()
        s0 = o.scalars()
        o.iterate(1)
        s = o.scalars()
        rows.append(dict(t=t, tau0=tau0, tau=o.get("tau").copy(), code=int(o.get("trace_code")[t - 1]),
                         Lrb=float(o.get("trace_Lrb")[t - 1]), Lib=s["L_ib"], Lgb=s["L_gb"], Lgb0=s0["L_gb"],
                         ib=o.get("ib_tour").copy(), rb=o.get("rb_tour").copy(), tmax=s["tau_max"],
                         tmin=s["tau_min"], choice=o.get("choice").copy()))
    return o, real, rows


def test_schedule_elites_restarts_and_bounds(orc):
    rng = np.random.default_rng(3)
    inst = euclid(rng.random((10, 2)))
    p = params(m=10, k=8, iterations=700, rho=0.2, seed=5, schedule=1)
    o, real, rows = _run(orc, inst, p)
    cand, W = o.get("cand"), o.get("W")
    restarts = [r["t"] for r in rows if r["code"] & 2]
    assert restarts, "the run is long enough for a stagnation restart"
    u, t_restart, last_imp, L_rb = 25, 0, 0, np.inf
    for r in rows:
        t = r["t"]
        if r["Lib"] < L_rb:
            L_rb, last_imp = r["Lib"], t
        use_rb = t % u == 0
        assert bool(r["code"] & 1) == use_rb
        assert r["Lgb"] <= r["Lgb0"] and r["Lgb"] <= r["Lib"]
        if r["code"] & 2:
            # only at a check, after > 250 iterations without restart-best improvement
            assert t % 100 == 0 and t - last_imp > 250
            assert np.all(r["tau"][real] == np.float32(r["tmax"]))
            assert np.isinf(r["Lrb"])
            L_rb, t_restart, last_imp = np.inf, t, t
        else:
            assert r["Lrb"] == L_rb
            # eq. (pheromone_update) with T+ = T_rb when the schedule says so, else T_ib
            elite = r["rb"] if use_rb else r["ib"]
            L_el = L_rb if use_rb else r["Lib"]
            nxt = {int(elite[q]): int(elite[(q + 1) % inst.n]) for q in range(inst.n)}
            prv = {v: k for k, v in nxt.items()}
            on = np.array([[real[i, c] and cand[i, c] in (nxt[i], prv[i]) for c in range(cand.shape[1])]
                           for i in range(inst.n)])
            x = r["tau0"] * np.float32(1.0 - p.rho)
            x = np.where(on, x + np.float32(1.0 / L_el), x)
            ref = np.minimum(np.float32(r["tmax"]), np.maximum(np.float32(r["tmin"]), x))
            assert np.array_equal(r["tau"][real], ref[real]), t
        assert np.array_equal(r["choice"][real], (r["tau"] * W)[real])
        u = orc.ugb(t - t_restart)
    # a check that found the pheromone converged but T_rb still improving does not restart
    assert all(t % 100 == 0 for t in restarts)
    assert o.ints()["n_restarts"] == len(restarts)


def test_schedule_off_is_iteration_best_only(orc):
    rng = np.random.default_rng(4)
    inst = euclid(rng.random((12, 2)))
    p = params(m=8, k=6, iterations=350, rho=0.2, seed=2, schedule=0)
    o = orc.Oracle(inst, p).iterate(p.iterations)
    assert not np.any(o.get("trace_code"))
    assert o.ints()["n_restarts"] == 0
