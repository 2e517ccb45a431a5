"""Batching with step limits and the continuous-batching server.

Every simulation's arithmetic is per node and per instance, so a simulation's
fields are bit-identical whether it runs alone, in a batch, or in the server's
changing mix of resident simulations.
"""
import numpy as np
import pytest

from paper_1410_3464_gb300 import inputs

pytestmark = pytest.mark.gpu

FIELDS = ("rho1", "rho2", "ux", "uy", "conc", "type", "vol")


@pytest.fixture(scope="module")
def pslbm():
    from paper_1410_3464_gb300 import build, pslbm as m
    build.build()
    return m


def alone(pslbm, sc, steps, precision):
    with pslbm.Simulation(sc["mask"], sc["params"], sc["rho1"], sc["rho2"], sc["conc"], sc["vol"],
                          precision=precision) as s:
        s.step(steps)
        return s.read()


def test_step_limit_freezes_state(pslbm):
    sc = inputs.porous_discs(nx=96, ny=64, seed=4)
    ref = alone(pslbm, sc, 30, pslbm.FP32)
    with pslbm.Simulation(sc["mask"], sc["params"], sc["rho1"], sc["rho2"], sc["conc"], sc["vol"],
                          precision=pslbm.FP32) as s:
        s.set_step_limit(30)
        s.step(50)
        assert s.steps() == 30
        got = s.read()
    for k in FIELDS:
        assert np.array_equal(got[k], ref[k]), k


def test_batch_members_with_different_limits(pslbm):
    scs = [inputs.porous_discs(nx=80 + 16 * i, ny=48 + 8 * i, seed=10 + i) for i in range(3)]
    limits = [17, 40, 29]
    refs = [alone(pslbm, sc, n, pslbm.FP32) for sc, n in zip(scs, limits)]
    sims = [pslbm.Simulation(sc["mask"], sc["params"], sc["rho1"], sc["rho2"], sc["conc"], sc["vol"],
                             precision=pslbm.FP32) for sc in scs]
    for s, n in zip(sims, limits):
        s.set_step_limit(n)
    b = pslbm.Batch(sims)
    b.step(90)
    b.sync()
    b.close()
    for s, n, ref in zip(sims, limits, refs):
        assert s.steps() == n
        got = s.read()
        for k in FIELDS:
            assert np.array_equal(got[k], ref[k]), k
        s.close()


def test_server_results_equal_alone_and_queueing(pslbm):
    """Five requests of different sizes and budgets, an HBM budget that holds
    only about two of them at a time (so later ones queue and are admitted as
    memory frees), chunks of 25 steps: every result equals the request run
    alone for the same number of steps."""
    reqs = [dict(nx=64, ny=64, seed=31, budget=40), dict(nx=128, ny=96, seed=32, budget=110),
            dict(nx=96, ny=160, seed=33, budget=75), dict(nx=160, ny=64, seed=34, budget=50),
            dict(nx=112, ny=112, seed=35, budget=130)]
    scenes = [inputs.porous_discs(nx=r["nx"], ny=r["ny"], seed=r["seed"]) for r in reqs]
    est = [pslbm.estimate_device_bytes(sc["params"], pslbm.FP32) for sc in scenes]
    budget = int(2.2 * max(est))
    srv = pslbm.Server(precision=pslbm.FP32, hbm_budget_bytes=budget, chunk_steps=25)
    ids = []
    max_active, saw_queue = 0, False
    for i, (r, sc) in enumerate(zip(reqs, scenes)):
        ids.append(srv.submit(sc["mask"], sc["params"], sc["rho1"], sc["rho2"], sc["conc"], sc["vol"],
                              step_budget=r["budget"], keep_fields=True))
        if i % 2 == 1:        # requests arrive while others are resident
            a, q, d = srv.advance()
            max_active = max(max_active, a)
            saw_queue |= q > 0
    for _ in range(100):
        a, q, d = srv.advance()
        max_active = max(max_active, a)
        saw_queue |= q > 0
        if all(srv.poll(i)[0] == pslbm.REQ_DONE for i in ids):
            break
    assert saw_queue, "the HBM budget never made a request wait"
    assert 2 <= max_active <= 3
    for rid, r, sc in zip(ids, reqs, scenes):
        st, n, b = srv.poll(rid)
        assert st == pslbm.REQ_DONE and n == r["budget"]
        got = srv.fetch(rid)
        ref = alone(pslbm, sc, r["budget"], pslbm.FP32)
        for k in FIELDS:
            assert np.array_equal(got[k], ref[k]), (rid, k)
        assert b[-1] == r["budget"]
    srv.close()


def test_server_stops_on_solid_volume_change(pslbm):
    """A fast-dissolving request with a 1 % solid-volume stop is retired at the
    first chunk boundary after the change, well before its step budget."""
    sc = inputs.porous_discs(nx=96, ny=64, seed=41, k2=0.2)
    conc = sc["conc"].copy()
    conc[0][sc["mask"] == 0] = 1.0          # plenty of B to dissolve D(s)
    vol = np.zeros((2,) + sc["mask"].shape)
    vol[0][sc["mask"] == 2] = 0.05
    srv = pslbm.Server(precision=pslbm.FP32, chunk_steps=20)
    rid = srv.submit(sc["mask"], sc["params"], sc["rho1"], sc["rho2"], conc, vol, step_budget=5000, stop_dv=0.01)
    for _ in range(300):
        srv.advance()
        st, n, b = srv.poll(rid)
        if st == pslbm.REQ_DONE:
            break
    assert st == pslbm.REQ_DONE
    assert 0 < n < 5000 and n % 20 == 0
    ns = sc["params"]["n_species"]
    v0 = vol[0].sum()
    assert abs(b[3 + ns] + b[4 + ns] - v0) >= 0.01 * v0
    srv.close()


def test_server_isolates_a_failing_request(pslbm):
    """A request whose initial density holds a NaN (injected on the host) is
    retired as failed after its first chunk; the request batched with it runs to
    its budget with the same result as alone."""
    good = inputs.porous_discs(nx=96, ny=64, seed=51)
    bad = inputs.porous_discs(nx=80, ny=48, seed=52)
    rho1 = bad["rho1"].copy()
    fy, fx = np.argwhere(bad["mask"] == 0)[10]
    rho1[fy, fx] = np.nan
    srv = pslbm.Server(precision=pslbm.FP32, chunk_steps=10)
    gid = srv.submit(good["mask"], good["params"], good["rho1"], good["rho2"], good["conc"], good["vol"],
                     step_budget=30, keep_fields=True)
    bid = srv.submit(bad["mask"], bad["params"], rho1, bad["rho2"], bad["conc"], bad["vol"], step_budget=30)
    for _ in range(10):
        srv.advance()
        if srv.poll(gid)[0] == pslbm.REQ_DONE and srv.poll(bid)[0] in (pslbm.REQ_DONE, pslbm.REQ_FAILED):
            break
    assert srv.poll(bid)[0] == pslbm.REQ_FAILED
    assert srv.poll(gid)[0] == pslbm.REQ_DONE
    got = srv.fetch(gid)
    ref = alone(pslbm, good, 30, pslbm.FP32)
    for k in FIELDS:
        assert np.array_equal(got[k], ref[k]), k
    srv.close()


def test_batch_monitor_and_profile(pslbm):
    """pslbm_batch_monitor gathers every member's step count and status in one
    read; pslbm_batch_profile_step times the three kernels of each step and
    advances the members like pslbm_batch_step (same results)."""
    scs = [inputs.porous_discs(nx=64 + 16 * i, ny=48, seed=20 + i) for i in range(3)]
    refs = [alone(pslbm, sc, 12, pslbm.FP32) for sc in scs]
    sims = [pslbm.Simulation(sc["mask"], sc["params"], sc["rho1"], sc["rho2"], sc["conc"], sc["vol"],
                             precision=pslbm.FP32) for sc in scs]
    sims[1].set_step_limit(7)
    b = pslbm.Batch(sims)
    b.step(5)
    assert b.monitor() == (5, 0)
    k, total = b.profile_step(7)
    assert all(v > 0 for v in k.values()) and total >= k["bulk"]
    steps, status = b.monitor()
    assert steps == 7 and status == 0          # the smallest step count: member 1 froze at 7
    b.close()
    for i, (s, ref) in enumerate(zip(sims, refs)):
        assert s.steps() == (7 if i == 1 else 12)
        if i != 1:
            got = s.read()
            for f in FIELDS:
                assert np.array_equal(got[f], ref[f]), f
        s.close()
