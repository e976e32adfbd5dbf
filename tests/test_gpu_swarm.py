"""GPU parity of the whole DPSO loop against the CPU oracle, through the C ABI.

Full trajectories are compared bit-exactly (positions, velocities as
permutations, pbests, fitness, gbest, history) at sizes the oracle finishes in
seconds; at the full facade and bridge sizes the initial swarm and the first
generation's particle update are compared for every particle and the edge
exchange for sampled particles.
"""
import numpy as np
import pytest

from gpu_helpers import DEV, assert_same_state, both_swarms, cost_matrix_gpu, torch  # noqa: F401
import oracle
from paper_1706_04399_gb300 import dpso, inputs

pytestmark = pytest.mark.gpu

F = dpso


def _setup(inst):
    C = cost_matrix_gpu(inst)
    C_np, st = oracle.cost_matrix(inst.xyz, inst.boxes)
    assert st == 0
    return C, C_np


def test_tiny_full_run_bitwise():
    inst = inputs.tiny()
    C, C_np = _setup(inst)
    gpu, ref = both_swarms(C_np, C, inst.tags, inst.swarm, inst.seed)
    assert_same_state(gpu.state(), ref, "init")
    for chunk in (1, 2, 3, 14, 30, 150):
        gpu.step(chunk)
        ref.run(chunk)
        assert_same_state(gpu.state(), ref, f"t={ref.t}")
    tour, cost = gpu.best()
    assert cost == 30_000
    assert np.array_equal(tour, ref.state()["G"])
    st = gpu.stats()
    c = ref.counters()
    assert (st["two_opt_pairs"], st["two_opt_moves"], st["two_opt_runs"]) == \
        (c["pairs"], c["moves"], c["two_opt_runs"])


CASES = {
    "all": dict(flags=F.FLAGS_ALL),
    "no_two_opt": dict(flags=F.FLAG_DET_INIT | F.FLAG_MUTATION),
    "no_mutation": dict(flags=F.FLAG_DET_INIT | F.FLAG_TWO_OPT),
    "move_only": dict(flags=0),
    "w_half": dict(flags=F.FLAGS_ALL, w=0.5),
    "w_zero": dict(flags=F.FLAGS_ALL, w=0.0, phi1=0.7, phi2=0.9),
    "trigger1": dict(flags=F.FLAGS_ALL, trigger=1),
    "stall": dict(flags=F.FLAGS_ALL, stall_limit=3),
    "swaps5_period2": dict(flags=F.FLAGS_ALL, mut_swaps=5, mut_period=2, det_frac_pct=40),
    "max_moves": dict(flags=F.FLAGS_ALL, max_moves=3),
}


@pytest.mark.parametrize("case", list(CASES))
def test_random_instance_trajectory_bitwise(case):
    inst = inputs.random_instance(71, 4, 17)
    C, C_np = _setup(inst)
    gpu, ref = both_swarms(C_np, C, inst.tags, 45, 99, **CASES[case])
    for chunk in (1, 1, 1, 4, 8):
        gpu.step(chunk)
        ref.run(chunk)
        assert_same_state(gpu.state(), ref, f"{case} t={ref.t}")


@pytest.mark.parametrize("n,S,T", [(96, 64, 10), (130, 33, 6), (40, 257, 9)])
def test_grid_trajectory_bitwise(n, S, T):
    inst = inputs.planar_grid(n, 1.5, inputs.random_instance(1, 3, n).boxes * 0.5, "grid",
                              S, T, 5)
    C, C_np = _setup(inst)
    gpu, ref = both_swarms(C_np, C, inst.tags, S, 1234 + n)
    gpu.step(T)
    ref.run(T)
    assert_same_state(gpu.state(), ref, f"grid n={n}")


def test_swarm_of_one_and_three_viewpoints():
    inst = inputs.random_instance(3, 0, 2)
    C, C_np = _setup(inst)
    gpu, ref = both_swarms(C_np, C, inst.tags, 1, 3)
    gpu.step(5)
    ref.run(5)
    assert_same_state(gpu.state(), ref, "n=3 S=1")


@pytest.mark.parametrize("name", ["facade", "bridge"])
def test_full_size_init_bitwise(name):
    inst = inputs.CONFIGS[name]()
    C, C_np = _setup(inst)
    gpu, ref = both_swarms(C_np, C, inst.tags, inst.swarm, inst.seed)
    assert_same_state(gpu.state(), ref, f"{name} init")


@pytest.mark.parametrize("name", ["facade", "bridge"])
def test_full_size_first_generation(name):
    """Generation 1 at full size: the particle update of every particle exactly,
    the edge exchange exactly for sampled particles, properties for the rest."""
    inst = inputs.CONFIGS[name]()
    C, C_np = _setup(inst)
    S, n = inst.swarm, inst.n
    # (a) without the edge exchange every particle is compared
    gpu, ref = both_swarms(C_np, C, inst.tags, S, inst.seed,
                           flags=F.FLAG_DET_INIT | F.FLAG_MUTATION)
    gpu.step(1)
    ref.run(1)
    assert_same_state(gpu.state(), ref, f"{name} generation 1 without 2-opt")
    gpu.close()
    # (b) with it: the oracle runs the exchange on a sample of particles only
    gpu = dpso.Swarm(C, n, inst.tags, dpso.default_params(swarm=S), inst.seed)
    gpu.step(1)
    gs = gpu.state()
    ref = oracle.Swarm(C_np, inst.tags, swarm=S, seed=inst.seed)
    gf0 = ref.gf
    ref.move(1)
    ref.gbest()
    ran = not ref.gf < gf0       # the exchange runs when gbest did not strictly improve
    assert gs["runs"] == int(ran)
    sample = [0, S // 2, S - 1] if name == "facade" else [1, S - 1]
    if ran:
        ref.two_opt(sample)
    rs = ref.state()
    for p in sample:
        for key in ("X", "P"):
            assert np.array_equal(gs[key][p], rs[key][p]), (name, key, p)
        assert gs["F"][p] == rs["F"][p] and gs["PF"][p] == rs["PF"][p], (name, p)
    assert np.array_equal(gs["V"], rs["V"])          # the exchange leaves velocities alone
    # properties of every particle
    for p in range(S):
        assert np.array_equal(np.sort(gs["X"][p]), np.arange(n))
    chk = np.random.default_rng(0).choice(S, 16, replace=False)
    for p in chk:
        assert gs["F"][p] == oracle.fitness(C_np, gs["X"][p])
        assert gs["PF"][p] == oracle.fitness(C_np, gs["P"][p]) <= gs["F"][p]
    assert gs["gf"] == gs["PF"].min() == oracle.fitness(C_np, gs["G"])
    assert gs["history"][0] == gs["gf"]


def test_checkpoint_resume_is_bit_exact():
    inst = inputs.random_instance(60, 3, 8)
    C, C_np = _setup(inst)
    p = dpso.default_params(swarm=40)
    a = dpso.Swarm(C, inst.n, inst.tags, p, 55)
    a.step(7)
    blob = a.state_bytes()
    a.step(8)
    end_a = a.state()
    b = dpso.Swarm(C, inst.n, inst.tags, p, 55)
    b.set_state_bytes(blob)
    b.step(8)
    end_b = b.state()
    for key in ("X", "V", "P", "G", "F", "PF", "history"):
        assert np.array_equal(end_a[key], end_b[key]), key
    ref = oracle.Swarm(C_np, inst.tags, swarm=40, seed=55)
    ref.run(15)
    assert_same_state(end_b, ref, "resumed")
    c = dpso.Swarm(C, inst.n, inst.tags, dpso.default_params(swarm=41), 55)
    with pytest.raises(dpso.DpsoError):
        c.set_state_bytes(blob)


def test_plan_from_host_buffers():
    inst = inputs.tiny()
    tour, cost = dpso.dpso_plan(inst.xyz, inst.boxes, inst.tags, dpso.default_cost_params(),
                                dpso.default_params(swarm=inst.swarm), inst.seed, inst.iterations)
    C_np, _ = oracle.cost_matrix(inst.xyz, inst.boxes)
    ref = oracle.Swarm(C_np, inst.tags, swarm=inst.swarm, seed=inst.seed)
    ref.run(inst.iterations)
    assert cost == ref.gf == 30_000
    assert np.array_equal(tour, ref.state()["G"])
    assert oracle.fitness(C_np, tour) == cost


def test_init_rejects_bad_arguments():
    inst = inputs.random_instance(12, 1, 9)
    C, C_np = _setup(inst)
    for kw in (dict(swarm=0), dict(w=1.5), dict(phi2=-0.1), dict(mut_period=0),
               dict(two_opt_trigger=2), dict(flags=16)):
        with pytest.raises(dpso.DpsoError) as e:
            dpso.Swarm(C, inst.n, inst.tags, dpso.default_params(**kw), 1)
        assert e.value.status == dpso.ERR_ARG, kw
    dup = inst.tags.copy()
    dup[3] = dup[4]
    with pytest.raises(dpso.DpsoError) as e:
        dpso.Swarm(C, inst.n, dup, dpso.default_params(swarm=4), 1)
    assert e.value.status == dpso.ERR_ARG
    asym = C_np.copy()
    asym[2, 5] += 3
    with pytest.raises(dpso.DpsoError) as e:
        dpso.Swarm(torch.from_numpy(asym).to(DEV), inst.n, inst.tags, dpso.default_params(), 1)
    assert e.value.status == dpso.ERR_ARG
    with pytest.raises(dpso.DpsoError) as e:
        dpso.Swarm(C, 2, None, dpso.default_params(), 1)
    assert e.value.status == dpso.ERR_ARG


@pytest.mark.parametrize("name,count,sample", [("facade", 256, [0, 101, 255]),
                                               ("bridge", 64, [9, 63])])
def test_full_size_two_opt_from_initial_tours(name, count, sample):
    """The edge exchange at full size from random starting tours: the GPU runs
    it on `count` initial particles, the oracle on a sample of them (both sides
    build their own initial swarm; test_full_size_init_bitwise shows they agree)."""
    inst = inputs.CONFIGS[name]()
    C, C_np = _setup(inst)
    S, n = inst.swarm, inst.n
    gpu = dpso.Swarm(C, n, inst.tags, dpso.default_params(swarm=S), inst.seed)
    X0 = gpu.state()["X"]
    gpu.close()
    first = S - count                     # random (not back-and-forth) particles
    T = torch.from_numpy(X0[first:].view(np.int16).copy()).to(DEV)
    cost = torch.empty(count, dtype=torch.int64, device=DEV)
    pairs, moves = dpso.dpso_two_opt(C, n, T, count, cost)
    got = T.cpu().numpy().view(np.uint16)
    got_c = cost.cpu().numpy()
    ref = oracle.Swarm(C_np, inst.tags, swarm=S, seed=inst.seed)
    X0_ref = ref.state()["X"]
    for k in sample:
        y, f, mv, pr = oracle.two_opt(C_np, X0_ref[first + k])
        assert np.array_equal(got[k], y), (name, k)
        assert got_c[k] == f and mv > n // 4, (name, k, mv)
    assert moves > count * (n // 4) and pairs % (n * (n - 3) // 2) == 0
    for k in range(count):
        assert np.array_equal(np.sort(got[k]), np.arange(n))
    for k in range(0, count, max(1, count // 8)):
        assert got_c[k] == oracle.fitness(C_np, got[k])


def test_side_stream_matches_default_stream():
    """A swarm created, stepped and checkpointed on a non-blocking stream
    follows the same trajectory as one on the legacy default stream (every
    zero-fill and upload of the library is ordered on the caller's stream)."""
    inst = inputs.planar_grid(1367, 1.0, np.zeros((0, 6)), "grid1367", 96, 4, 0)
    C = cost_matrix_gpu(inst)
    p = dpso.default_params(swarm=inst.swarm)
    ref = dpso.Swarm(C, inst.n, inst.tags, p, inst.seed)
    ref.step(inst.iterations)
    want = ref.state()
    side = torch.cuda.Stream()
    for _ in range(3):
        sw = dpso.Swarm(C, inst.n, inst.tags, p, inst.seed, side)
        sw.step(2, side)
        blob = sw.state_bytes()
        sw.set_state_bytes(blob)
        sw.step(inst.iterations - 2, side)
        got = sw.state()
        for key in ("X", "V", "P", "G", "F", "PF", "history"):
            assert np.array_equal(got[key], want[key]), key
        sw.close()
    tour, cost = dpso.dpso_plan(inst.xyz, inst.boxes, inst.tags, dpso.default_cost_params(), p,
                                inst.seed, inst.iterations)
    assert cost == want["gf"] and np.array_equal(tour, want["G"].astype(np.int32))
    ref.close()


@pytest.mark.parametrize("n", [60, 300])
def test_two_opt_evaluated_pair_count(n):
    """The exchange kernels' evaluated-pair count: each tour's first pass in a
    generation scans all n(n-3)/2 pairs and later passes only the rows and
    columns the previous move changed, so runs*S*n(n-3)/2 <= evaluated <=
    pairs (the plain scan's count, which the oracle reproduces); the node
    swap rescans every pair."""
    inst = inputs.random_instance(n, 3, 900 + n)
    C = cost_matrix_gpu(inst)
    S, T = 64, 4
    sw = dpso.Swarm(C, n, inst.tags, dpso.default_params(swarm=S), 3)
    sw.step(T)
    st = sw.stats()
    first_passes = st["two_opt_runs"] * S * (n * (n - 3) // 2)
    assert st["two_opt_moves"] > 0
    assert first_passes <= st["two_opt_evaluated"] < st["two_opt_pairs"]
    sw.close()
    ns = dpso.Swarm(C, n, inst.tags,
                    dpso.default_params(swarm=S, flags=dpso.FLAGS_ALL | dpso.FLAG_NODE_SWAP), 3)
    ns.step(T)
    st = ns.stats()
    assert st["two_opt_evaluated"] == st["two_opt_pairs"] > 0
    ns.close()
