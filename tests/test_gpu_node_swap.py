"""Node-swap exchange on the GPU against the oracle: the standalone entry
point (tours, costs, pair and move counts bit-exact), swarms that exchange by
node swap, and batches that mix both exchange kinds."""
import numpy as np
import pytest

from gpu_helpers import DEV, assert_same_state, cost_matrix_gpu, torch  # noqa: F401
import oracle
from paper_1706_04399_gb300 import dpso, inputs

pytestmark = pytest.mark.gpu


def _node_swap_case(C_np, tours, max_moves=0):
    n = C_np.shape[0]
    C = torch.from_numpy(C_np).to(DEV)
    T = torch.from_numpy(tours.view(np.int16).copy()).to(DEV)
    cost = torch.empty(len(tours), dtype=torch.int64, device=DEV)
    pairs, moves = dpso.dpso_node_swap(C, n, T, len(tours), cost, max_moves)
    got_t = T.cpu().numpy().view(np.uint16)
    got_c = cost.cpu().numpy()
    tot_p = tot_m = 0
    for k, x in enumerate(tours):
        y, f, mv, pr = oracle.node_swap(C_np, x, max_moves)
        assert np.array_equal(got_t[k], y), (n, k)
        assert got_c[k] == f, (n, k)
        tot_p += pr
        tot_m += mv
    assert (pairs, moves) == (tot_p, tot_m)


@pytest.mark.parametrize("n,count", [(3, 5), (4, 7), (5, 9), (6, 4), (9, 12), (33, 10), (34, 9),
                                     (35, 8), (64, 12), (100, 16), (257, 4), (400, 3)])
def test_node_swap_to_convergence_bitwise(n, count):
    C_np = inputs.random_cost_matrix(n, 11 * n, hi=1_000_000)
    _node_swap_case(C_np, inputs.random_tours(n, count, 5 * n))


def test_node_swap_grid_ties_bitwise():
    # integer grid costs: many equal deltas exercise the (delta, i, j) order
    inst = inputs.planar_grid(120, 1.0, np.zeros((0, 6)), "g120", 1, 1, 1)
    C_np, _ = oracle.cost_matrix(inst.xyz, inst.boxes)
    _node_swap_case(C_np, inputs.random_tours(120, 10, 6))


@pytest.mark.parametrize("n,moves", [(1200, 6), (2000, 3)])
def test_node_swap_large_capped_bitwise(n, moves):
    # shorter tile heights for long tours; capped moves keep the oracle quick
    C_np = inputs.random_cost_matrix(n, n, hi=1_000_000)
    _node_swap_case(C_np, inputs.random_tours(n, 3, n + 1), max_moves=moves)


def test_node_swap_costs_at_the_limit():
    n = 61
    rng = np.random.default_rng(n)
    top = rng.integers(dpso.NODE_SWAP_COST_MAX - 3, dpso.NODE_SWAP_COST_MAX + 1, size=(n, n))
    top = np.triu(top, 1)
    C_np = np.ascontiguousarray((top + top.T).astype(np.int32))
    _node_swap_case(C_np, inputs.random_tours(n, 6, n + 2))


def test_node_swap_rejects_out_of_range():
    n = 20
    C_np = inputs.random_cost_matrix(n, 4)
    C_np[3, 5] = C_np[5, 3] = dpso.NODE_SWAP_COST_MAX + 1
    C = torch.from_numpy(C_np).to(DEV)
    T = torch.from_numpy(inputs.random_tours(n, 2, 1).view(np.int16)).to(DEV)
    cost = torch.empty(2, dtype=torch.int64, device=DEV)
    with pytest.raises(dpso.DpsoError) as e:
        dpso.dpso_node_swap(C, n, T, 2, cost)
    assert e.value.status == dpso.ERR_RANGE
    big = 6000  # no tile of three extra rows fits in shared memory
    with pytest.raises(dpso.DpsoError) as e:
        dpso.dpso_node_swap(C, big, T, 0, cost)
    assert e.value.status == dpso.ERR_RANGE


FLAGS_NS = dpso.FLAGS_ALL | dpso.FLAG_NODE_SWAP


@pytest.mark.parametrize("n,m,S,T,trigger", [(30, 2, 24, 15, 0), (77, 4, 40, 9, 0),
                                             (50, 3, 33, 12, 1)])
def test_swarm_with_node_swap_matches_oracle(n, m, S, T, trigger):
    inst = inputs.random_instance(n, m, 40 + n)
    C_np, _ = oracle.cost_matrix(inst.xyz, inst.boxes)
    C = cost_matrix_gpu(inst)
    p = dpso.default_params(swarm=S, flags=FLAGS_NS, two_opt_trigger=trigger)
    gpu = dpso.Swarm(C, n, inst.tags, p, 17)
    ref = oracle.Swarm(C_np, inst.tags, swarm=S, seed=17, flags=FLAGS_NS, trigger=trigger)
    for t in range(T):
        gpu.step(1)
        ref.iterate()
        assert_same_state(gpu.state(), ref, f"node swap n={n} generation {t + 1}")
    st = gpu.stats()
    assert st["two_opt_pairs"] == ref.counters()["pairs"]
    gpu.close()


def test_swarm_node_swap_rejects_costs_above_its_limit():
    inst = inputs.random_instance(25, 1, 3)
    C = cost_matrix_gpu(inst)
    C[2, 7] = C[7, 2] = dpso.NODE_SWAP_COST_MAX + 5
    with pytest.raises(dpso.DpsoError) as e:
        dpso.Swarm(C, 25, inst.tags, dpso.default_params(swarm=8, flags=FLAGS_NS), 1)
    assert e.value.status == dpso.ERR_RANGE
    # the edge exchange accepts the same matrix
    dpso.Swarm(C, 25, inst.tags, dpso.default_params(swarm=8), 1).close()


def test_batch_mixing_exchange_kinds_matches_solo():
    specs = [(40, 2, 24, FLAGS_NS), (90, 3, 32, dpso.FLAGS_ALL), (150, 1, 20, FLAGS_NS),
             (23, 0, 40, dpso.FLAGS_ALL)]
    members = []
    for k, (n, m, S, flags) in enumerate(specs):
        inst = inputs.random_instance(n, m, 620 + k)
        members.append((inst, dpso.default_params(swarm=S, flags=flags), 90 + k))
    Cs = [cost_matrix_gpu(inst) for inst, _, _ in members]
    want = []
    for C, (inst, p, seed) in zip(Cs, members):
        sw = dpso.Swarm(C, inst.n, inst.tags, p, seed)
        sw.step(7)
        want.append(sw.state())
        sw.close()
    swarms = [dpso.Swarm(C, inst.n, inst.tags, p, seed) for C, (inst, p, seed) in zip(Cs, members)]
    batch = dpso.Batch(swarms)
    batch.autotune()
    batch.step(3)
    batch.step(4)
    for sw, w, (inst, p, _) in zip(swarms, want, members):
        got = sw.state()
        for key in ("X", "V", "P", "G", "F", "PF", "history"):
            assert np.array_equal(got[key], w[key]), (inst.n, p.flags, key)
    batch.close()
