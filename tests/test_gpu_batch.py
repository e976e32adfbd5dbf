"""Batched generations: every member of a batch must follow exactly the
trajectory it follows alone (same tours, velocities, pbests, histories,
counters), whatever its size, parameters or starting generation."""
import numpy as np
import pytest

from gpu_helpers import DEV, assert_same_state, cost_matrix_gpu, torch  # noqa: F401
import oracle
from paper_1706_04399_gb300 import dpso, inputs

pytestmark = pytest.mark.gpu

KEYS = ("X", "V", "P", "G", "F", "PF", "history")


def _members():
    """(instance, params) pairs with mixed sizes and parameters."""
    out = []
    specs = [(37, 3, 24, {}), (120, 4, 64, {"w": 0.5}), (71, 0, 33, {"two_opt_trigger": 1}),
             (260, 6, 40, {"flags": dpso.FLAG_DET_INIT | dpso.FLAG_MUTATION}),
             (15, 1, 130, {"mut_period": 2, "mut_swaps": 4}), (400, 5, 16, {"max_moves": 5}),
             (9, 0, 7, {"w": 0.0, "phi1": 0.8, "phi2": 0.9}), (88, 2, 50, {"stall_limit": 4})]
    for k, (n, m, S, kw) in enumerate(specs):
        inst = inputs.random_instance(n, m, 500 + k)
        p = dpso.default_params(swarm=S)
        for key, val in kw.items():
            setattr(p, key, val)
        out.append((inst, p, 900 + k))
    return out


def _solo_state(C, inst, p, seed, gens):
    sw = dpso.Swarm(C, inst.n, inst.tags, p, seed)
    sw.step(gens)
    st = sw.state()
    stats = sw.stats()
    sw.close()
    return st, stats


def test_batch_members_match_solo_runs():
    members = _members()
    Cs = [cost_matrix_gpu(inst) for inst, _, _ in members]
    swarms = [dpso.Swarm(C, inst.n, inst.tags, p, seed) for C, (inst, p, seed) in zip(Cs, members)]
    batch = dpso.Batch(swarms)
    batch.step(4)
    batch.step(7)
    for C, sw, (inst, p, seed) in zip(Cs, swarms, members):
        got = sw.state()
        want, want_stats = _solo_state(C, inst, p, seed, 11)
        for key in KEYS:
            assert np.array_equal(got[key], want[key]), (inst.n, key)
        assert (got["t"], got["gf"], got["done"]) == (want["t"], want["gf"], want["done"])
        st = sw.stats()
        for key in ("two_opt_pairs", "two_opt_moves", "two_opt_runs"):
            assert st[key] == want_stats[key], (inst.n, key)
    batch.close()


def test_batch_members_at_different_generations():
    # members join the batch after different numbers of solo generations, so
    # mutation generations fall at different steps for each
    members = _members()[:5]
    Cs = [cost_matrix_gpu(inst) for inst, _, _ in members]
    swarms = []
    for k, (C, (inst, p, seed)) in enumerate(zip(Cs, members)):
        sw = dpso.Swarm(C, inst.n, inst.tags, p, seed)
        sw.step(k)
        swarms.append(sw)
    batch = dpso.Batch(swarms)
    batch.step(6)
    for k, (C, sw, (inst, p, seed)) in enumerate(zip(Cs, swarms, members)):
        want, _ = _solo_state(C, inst, p, seed, k + 6)
        got = sw.state()
        for key in KEYS:
            assert np.array_equal(got[key], want[key]), (k, key)
    batch.close()


def test_batch_autotune_keeps_results_and_matches_oracle():
    members = _members()[:4]
    Cs = [cost_matrix_gpu(inst) for inst, _, _ in members]
    swarms = [dpso.Swarm(C, inst.n, inst.tags, p, seed) for C, (inst, p, seed) in zip(Cs, members)]
    batch = dpso.Batch(swarms)
    rows, tpc, tg = batch.autotune()
    assert rows in (32, 30, 24, 16, 8) and tpc in (1, 2, 4) and tg in (1, 2)
    batch.step(5)
    for C, sw, (inst, p, seed) in zip(Cs, swarms, members):
        C_np, _ = oracle.cost_matrix(inst.xyz, inst.boxes)
        ref = oracle.Swarm(C_np, inst.tags, swarm=p.swarm, w=p.w, phi1=p.phi1, phi2=p.phi2,
                           mut_period=p.mut_period, mut_swaps=p.mut_swaps,
                           det_frac_pct=p.det_frac_pct, stall_limit=p.stall_limit, flags=p.flags,
                           trigger=p.two_opt_trigger, max_moves=p.max_moves, seed=seed)
        ref.run(5)
        assert_same_state(sw.state(), ref, f"batched n={inst.n}")
    batch.close()


def test_batched_workload_sample_matches_solo():
    # a slice of the batched workload (sizes log-uniform in 50..1500), with
    # smaller swarms and fewer generations so the solo reruns stay quick
    insts = inputs.batched(count=12)
    Cs = [cost_matrix_gpu(inst) for inst in insts]
    params = [dpso.default_params(swarm=min(inst.swarm, 96)) for inst in insts]
    swarms = [dpso.Swarm(C, inst.n, inst.tags, p, inst.seed)
              for C, inst, p in zip(Cs, insts, params)]
    batch = dpso.Batch(swarms)
    batch.autotune()
    batch.step(3)
    for C, sw, inst, p in zip(Cs, swarms, insts, params):
        want, _ = _solo_state(C, inst, p, inst.seed, 3)
        got = sw.state()
        for key in KEYS:
            assert np.array_equal(got[key], want[key]), (inst.n, key)
    batch.close()


def test_batch_rejects_bad_members():
    inst = inputs.random_instance(20, 1, 3)
    C = cost_matrix_gpu(inst)
    sw = dpso.Swarm(C, inst.n, inst.tags, dpso.default_params(swarm=8), 1)
    with pytest.raises(dpso.DpsoError):
        dpso.Batch([sw, sw])
    with pytest.raises(dpso.DpsoError):
        dpso.Batch([])


@pytest.mark.parametrize("rows", [32, 30, 24, 16, 8])
def test_every_two_opt_shape_gives_identical_states(rows):
    """Each (tile height, tours per CTA) launch shape that fits gives the same
    trajectories: members of uneven size under one shape match solo runs."""
    specs = [(23, 0, 40), (70, 2, 24), (121, 3, 33), (190, 1, 17)]
    members = []
    for k, (n, m, S) in enumerate(specs):
        inst = inputs.random_instance(n, m, 880 + k)
        members.append((inst, dpso.default_params(swarm=S), 60 + k))
    Cs = [cost_matrix_gpu(inst) for inst, _, _ in members]
    want = [_solo_state(C, inst, p, seed, 6)[0] for C, (inst, p, seed) in zip(Cs, members)]
    for tpc, tg in ((1, 1), (2, 1), (4, 1), (1, 2)):
        swarms = [dpso.Swarm(C, inst.n, inst.tags, p, seed)
                  for C, (inst, p, seed) in zip(Cs, members)]
        batch = dpso.Batch(swarms)
        batch.set_two_opt_shape(rows, tpc, tg)
        batch.step(6)
        for sw, w, (inst, _, _) in zip(swarms, want, members):
            got = sw.state()
            for key in KEYS:
                assert np.array_equal(got[key], w[key]), (rows, tpc, tg, inst.n, key)
        batch.close()
        for sw in swarms:
            sw.close()
