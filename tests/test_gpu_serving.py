"""Re-planning server: every request's result (tour and cost) is the same
whether it runs alone (dpso_plan) or inside the server's continuous batch,
whatever else is admitted before, beside or after it; admission honours the
device-memory budget and the slot limit."""
import time

import numpy as np
import pytest

from gpu_helpers import torch  # noqa: F401
import oracle
from paper_1706_04399_gb300 import dpso, inputs

pytestmark = pytest.mark.gpu


def _requests():
    """Mixed requests: sizes, obstacles, swarm sizes, budgets and parameters."""
    specs = [(40, 2, 48, 30, {}), (150, 5, 64, 12, {"w": 0.5}),
             (23, 0, 32, 40, {"two_opt_trigger": 1}),
             (310, 8, 40, 9, {"flags": dpso.FLAG_DET_INIT | dpso.FLAG_MUTATION}),
             (12, 1, 100, 25, {"mut_period": 2, "mut_swaps": 4}),
             (520, 4, 24, 6, {"max_moves": 7}), (77, 3, 60, 0, {}),
             (9, 0, 16, 17, {"w": 0.0, "phi1": 0.8, "phi2": 0.9}),
             (96, 2, 56, 21, {"stall_limit": 3}), (205, 6, 36, 14, {})]
    out = []
    for k, (n, m, S, T, kw) in enumerate(specs):
        inst = inputs.random_instance(n, m, 700 + k)
        p = dpso.default_params(swarm=S)
        for key, val in kw.items():
            setattr(p, key, val)
        cp = dpso.default_cost_params(uav_radius_m=0.1 * (k % 3))
        out.append((inst, cp, p, 4000 + k, T))
    return out


def _solo(req):
    inst, cp, p, seed, T = req
    return dpso.dpso_plan(inst.xyz, inst.boxes, inst.tags, cp, p, seed, T)


def _wait_all(server, ids, timeout_s=600.0):
    out = {}
    for rid in ids:
        assert server.wait(rid, timeout_s) == 1, rid
        state, tour, cost, lat = server.poll(rid)
        assert state == 1 and lat > 0.0
        out[rid] = (tour, cost)
    return out


def test_results_identical_alone_and_in_the_mix():
    reqs = _requests()
    want = [_solo(r) for r in reqs]
    server = dpso.Server(dpso.default_server_params(generations_per_tick=5))
    # the first half starts together; the rest arrive while it runs
    ids = [server.submit(inst.xyz, inst.boxes, inst.tags, cp, p, seed, T)
           for inst, cp, p, seed, T in reqs[:5]]
    time.sleep(0.05)
    for inst, cp, p, seed, T in reqs[5:]:
        ids.append(server.submit(inst.xyz, inst.boxes, inst.tags, cp, p, seed, T))
        time.sleep(0.01)
    got = _wait_all(server, ids)
    for rid, (tour, cost), (wt, wc), req in zip(ids, got.values(), want, reqs):
        assert cost == wc, (req[0].n, cost, wc)
        assert np.array_equal(tour, wt), req[0].n
        assert sorted(tour.tolist()) == list(range(req[0].n))
    st = server.stats()
    assert st["completed"] == len(reqs) and st["failed"] == 0 and st["queued"] == 0
    assert st["peak_active"] > 1
    assert st["particle_iterations"] == sum(r[2].swarm * r[4] for r in reqs)
    server.close()


def test_server_result_matches_the_oracle():
    """Two small requests served together equal the oracle's plain runs."""
    server = dpso.Server()
    cases = []
    for k, (n, S, T) in enumerate(((30, 32, 25), (18, 20, 40))):
        inst = inputs.random_instance(n, 2, 800 + k)
        p = dpso.default_params(swarm=S)
        cp = dpso.default_cost_params()
        rid = server.submit(inst.xyz, inst.boxes, inst.tags, cp, p, 60 + k, T)
        cases.append((rid, inst, S, T, 60 + k))
    for rid, inst, S, T, seed in cases:
        assert server.wait(rid) == 1
        _, tour, cost, _ = server.poll(rid)
        C, _ = oracle.cost_matrix(inst.xyz, inst.boxes, 0.0, 1_000_000)
        ref = oracle.Swarm(C, inst.tags, swarm=S, seed=seed, flags=oracle.ALL)
        ref.run(T)
        rs = ref.state()
        assert cost == rs["gf"]
        assert np.array_equal(tour, rs["G"].astype(np.int32))
    server.close()


def test_memory_budget_serialises_admission():
    """A budget that holds one request at a time: results unchanged, never two
    requests resident, and a request larger than the budget fails cleanly."""
    cp = dpso.default_cost_params()
    reqs = []
    for k, (n, m, T) in enumerate(((100, 2, 12), (112, 0, 8), (124, 5, 15), (136, 3, 10))):
        p = dpso.default_params(swarm=40)
        reqs.append((inputs.random_instance(n, m, 750 + k), cp, p, 30 + k, T))
    fps = sorted(dpso.dpso_server_footprint(i.xyz, i.boxes, i.tags, c, p, s, T)
                 for i, c, p, s, T in reqs)
    budget = fps[-1]
    assert budget < fps[0] + fps[1]  # no two requests fit together
    big = inputs.random_instance(600, 2, 999)
    bp = dpso.default_params(swarm=64)
    assert dpso.dpso_server_footprint(big.xyz, big.boxes, big.tags, cp, bp, 5, 3) > budget
    server = dpso.Server(dpso.default_server_params(memory_budget_bytes=budget))
    ids = [server.submit(i.xyz, i.boxes, i.tags, c, p, s, T) for i, c, p, s, T in reqs]
    too_big = server.submit(big.xyz, big.boxes, big.tags, cp, bp, 5, 3)
    got = _wait_all(server, ids)
    for (tour, cost), req in zip(got.values(), reqs):
        wt, wc = _solo(req)
        assert cost == wc and np.array_equal(tour, wt)
    assert server.wait(too_big) == dpso.ERR_NO_MEMORY
    st = server.stats()
    assert st["peak_active"] == 1
    assert st["failed"] == 1 and st["completed"] == len(reqs)
    assert st["memory_used_bytes"] == 0
    server.close()


def test_slot_limit_and_zero_budget_requests():
    reqs = _requests()[:4]
    server = dpso.Server(dpso.default_server_params(max_active=2, generations_per_tick=3))
    ids = [server.submit(i.xyz, i.boxes, i.tags, cp, p, s, T) for i, cp, p, s, T in reqs]
    inst, cp, p, seed, _ = reqs[0]
    zero = server.submit(inst.xyz, inst.boxes, inst.tags, cp, p, seed, 0)
    got = _wait_all(server, ids + [zero])
    for rid, req in zip(ids, reqs):
        wt, wc = _solo(req)
        assert got[rid][1] == wc and np.array_equal(got[rid][0], wt)
    wt, wc = _solo((inst, cp, p, seed, 0))
    assert got[zero][1] == wc and np.array_equal(got[zero][0], wt)
    assert server.stats()["peak_active"] <= 2
    server.close()


def test_submit_rejects_bad_requests():
    server = dpso.Server()
    inst = inputs.random_instance(20, 1, 3)
    cp = dpso.default_cost_params()
    with pytest.raises(dpso.DpsoError) as e:
        server.submit(inst.xyz, inst.boxes, inst.tags, cp, dpso.default_params(swarm=0), 1, 5)
    assert e.value.status == dpso.ERR_ARG
    with pytest.raises(dpso.DpsoError) as e:
        server.submit(inst.xyz, inst.boxes, inst.tags, cp, dpso.default_params(), 1, -1)
    assert e.value.status == dpso.ERR_ARG
    with pytest.raises(dpso.DpsoError) as e:
        server.submit(inst.xyz, inst.boxes, inst.tags,
                      dpso.default_cost_params(uav_radius_m=-1.0), dpso.default_params(), 1, 5)
    assert e.value.status == dpso.ERR_ARG
    with pytest.raises(dpso.DpsoError):
        server.poll(12345)
    server.close()


def test_shortest_first_admission_keeps_results():
    """Least-estimated-work-first admission with two slots: the small requests
    (submitted last) are admitted before the large ones; every result is
    still the solo run's."""
    reqs = sorted(_requests(), key=lambda r: -r[0].n)[:6]  # largest first
    server = dpso.Server(dpso.default_server_params(max_active=2, generations_per_tick=4,
                                                    policy=dpso.SERVE_SHORTEST_FIRST, lanes=1))
    ids = [server.submit(i.xyz, i.boxes, i.tags, cp, p, s, T) for i, cp, p, s, T in reqs]
    got = _wait_all(server, ids)
    for rid, req in zip(ids, reqs):
        wt, wc = _solo(req)
        assert got[rid][1] == wc and np.array_equal(got[rid][0], wt)
    lat = {rid: server.poll(rid)[3] for rid in ids}
    # the smallest request (submitted last) finished before the largest one
    assert lat[ids[-1]] < lat[ids[0]]
    server.close()


@pytest.mark.parametrize("lanes", [1, 3, 8])
def test_lanes_keep_results_and_let_small_requests_pass(lanes):
    """Size-class lanes: every result is still the solo run's, with one lane
    (a single lock-step batch) and with several; with several lanes a small
    request submitted after a large one finishes first."""
    reqs = _requests()
    big = (inputs.random_instance(420, 3, 991), dpso.default_cost_params(),
           dpso.default_params(swarm=512), 17, 300)
    small = (inputs.random_instance(30, 1, 992), dpso.default_cost_params(),
             dpso.default_params(swarm=32), 18, 10)
    server = dpso.Server(dpso.default_server_params(generations_per_tick=4, lanes=lanes))
    order = [big] + reqs + [small]
    ids = [server.submit(i.xyz, i.boxes, i.tags, cp, p, s, T) for i, cp, p, s, T in order]
    got = _wait_all(server, ids)
    for rid, req in zip(ids, order):
        wt, wc = _solo(req)
        assert got[rid][1] == wc and np.array_equal(got[rid][0], wt), req[0].n
    if lanes > 1:
        assert server.poll(ids[-1])[3] < server.poll(ids[0])[3]
    st = server.stats()
    assert st["completed"] == len(order) and st["failed"] == 0 and st["memory_used_bytes"] == 0
    server.close()


def test_server_rejects_bad_lane_counts():
    for lanes in (-1, 9):
        with pytest.raises(dpso.DpsoError) as e:
            dpso.Server(dpso.default_server_params(lanes=lanes))
        assert e.value.status == dpso.ERR_ARG
