"""Snapshot replay at the full facade and bridge sizes (the configurations
the benchmark times): the GPU runs the swarm to generation t0, its state is
loaded into the oracle, and both run generation t0 + 1 from it.

Without the edge exchange every particle's update, mutation (the sort,
duplicate test and ranking over the whole swarm, Sec. 3.2.2), pbest, gbest
and history entry are compared bit-exactly.  With it (Sec. 3.2.3), the
facade's whole generation is compared (the oracle exchanges every particle,
on several host threads); on the bridge the oracle exchanges a sample of
particles, compared exactly, and the others are checked for validity,
fitness and 2-optimality.
"""
import functools

import numpy as np
import pytest

from gpu_helpers import (DEV, checkpoint_with_flags, cost_matrix_gpu,  # noqa: F401
                         host_threads, torch)
import oracle
from paper_1706_04399_gb300 import dpso, inputs

pytestmark = pytest.mark.gpu

NO_EXCHANGE = dpso.FLAG_DET_INIT | dpso.FLAG_MUTATION
STOPS = {"facade": (2, 8, 10), "bridge": (2, 5)}


@functools.lru_cache(maxsize=None)
def _instance(name):
    inst = inputs.CONFIGS[name]()
    C = cost_matrix_gpu(inst)
    C_np, st = oracle.cost_matrix(inst.xyz, inst.boxes)
    assert st == 0 and np.array_equal(C.cpu().numpy(), C_np)
    return inst, C, C_np


@functools.lru_cache(maxsize=None)
def _trajectory(name):
    """GPU checkpoints of the full swarm at each stop generation t0 and the
    GPU state one generation later."""
    inst, C, _ = _instance(name)
    sw = dpso.Swarm(C, inst.n, inst.tags, dpso.default_params(swarm=inst.swarm), inst.seed)
    out = {}
    t = 0
    for t0 in STOPS[name]:
        sw.step(t0 - t)
        blob = sw.state_bytes()
        sw.step(1)
        out[t0] = (blob, sw.state(), sw.stats())
        sw.set_state_bytes(blob)          # back to t0, then on to the next stop
        t = t0
    sw.close()
    return out


def _compare(gs, rs, what, particles=None):
    keys = ("X", "P", "V", "F", "PF")
    for key in keys:
        a, b = gs[key], rs[key]
        if particles is not None and key != "V":
            a, b = a[particles], b[particles]
        if not np.array_equal(a, b):
            bad = np.argwhere(a != b)
            raise AssertionError(f"{what}: {key} differs at {bad[:5].tolist()} ({len(bad)})")


CASES = [(name, t0) for name in STOPS for t0 in STOPS[name]]


@pytest.mark.parametrize("name,t0", CASES)
def test_replay_generation_without_exchange(name, t0):
    """Every particle of the full swarm through one generation from a GPU
    steady state (tours already exchanged, duplicates present), the edge
    exchange switched off on both sides: particle update, fitness, pbest,
    mutation when t0 + 1 is a multiple of 3, gbest and history."""
    inst, C, C_np = _instance(name)
    blob, _, _ = _trajectory(name)[t0]
    gpu = dpso.Swarm(C, inst.n, inst.tags,
                     dpso.default_params(swarm=inst.swarm, flags=NO_EXCHANGE), inst.seed)
    gpu.set_state_bytes(checkpoint_with_flags(blob, NO_EXCHANGE))
    start = gpu.state()
    assert start["t"] == t0
    ref = oracle.Swarm(C_np, inst.tags, swarm=inst.swarm, seed=inst.seed, flags=NO_EXCHANGE)
    ref.load_state(start)
    gpu.step(1)
    ref.iterate()
    gs, rs = gpu.state(), ref.state()
    gpu.close()
    what = f"{name} t={t0}->{t0 + 1} without exchange"
    _compare(gs, rs, what)
    assert np.array_equal(gs["G"], rs["G"]) and gs["gf"] == rs["gf"], what
    assert np.array_equal(gs["history"], rs["history"]), what
    assert (gs["t"], gs["stall"]) == (rs["t"], rs["stall"]), what
    if (t0 + 1) % 3 == 0:
        # the mutation really disturbed particles: at least S - ceil(S/3) tours moved
        moved = np.any(gs["X"] != start["X"], axis=1).sum()
        assert moved >= inst.swarm - (inst.swarm + 2) // 3, (what, moved)


@pytest.mark.parametrize("name,t0", CASES)
def test_replay_generation_with_exchange(name, t0):
    """One whole generation, edge exchange included, from the GPU's state at
    t0.  Facade: the oracle exchanges every particle (threads over disjoint
    particles) and the whole state, history and counters must match.  Bridge:
    a sample of particles is exchanged by the oracle and compared exactly;
    every other particle is checked for validity, its cost, and (a subset)
    2-optimality; velocities (which the exchange leaves alone) are compared
    for every particle."""
    inst, C, C_np = _instance(name)
    blob, gs, gstats = _trajectory(name)[t0]
    S, n = inst.swarm, inst.n
    ref = oracle.Swarm(C_np, inst.tags, swarm=S, seed=inst.seed)
    start = dpso.Swarm(C, n, inst.tags, dpso.default_params(swarm=S), inst.seed)
    start.set_state_bytes(blob)
    ref.load_state(start.state())
    start.close()
    what = f"{name} t={t0}->{t0 + 1}"
    if name == "facade":
        ran = ref.iterate_threaded(host_threads())
        rs = ref.state()
        assert gs["runs"] == rs["runs"], what
        _compare(gs, rs, what)
        assert np.array_equal(gs["G"], rs["G"]) and gs["gf"] == rs["gf"], what
        assert np.array_equal(gs["history"], rs["history"]), what
        assert (gs["pairs"], gs["moves"]) == (rs["pairs"], rs["moves"]), what
        assert gstats["two_opt_pairs"] == rs["pairs"]
        return
    sample = np.array([0, 1, 409, 410, S // 3, S // 2, S - 2, S - 1]
                      + list(np.random.default_rng(t0).choice(S, 8, replace=False)), np.int32)
    sample = np.unique(sample)
    ran = ref.iterate_threaded(host_threads(), sample=sample)
    rs = ref.state()
    assert gs["runs"] - start_runs(blob) == int(ran), what
    if not ran:                           # gbest improved: no exchange, all comparable
        _compare(gs, rs, what)
        assert np.array_equal(gs["history"], rs["history"]) and gs["gf"] == rs["gf"], what
        return
    _compare(gs, rs, what, particles=sample)
    for p in range(S):
        assert np.array_equal(np.sort(gs["X"][p]), np.arange(n)), (what, p)
    chk = np.random.default_rng(100 + t0).choice(S, 48, replace=False)
    for p in chk:
        assert gs["F"][p] == oracle.fitness(C_np, gs["X"][p]), (what, p)
        assert gs["PF"][p] == oracle.fitness(C_np, gs["P"][p]) <= gs["F"][p], (what, p)
        if ran:
            _, _, mv, _ = oracle.two_opt(C_np, gs["X"][p], max_moves=1)
            assert mv == 0, (what, p, "not 2-optimal")
    assert gs["gf"] == gs["PF"].min() == oracle.fitness(C_np, gs["G"]), what
    assert gs["history"][-1] == gs["gf"] and len(gs["history"]) == t0 + 1, what
    assert np.array_equal(gs["history"][:t0], rs["history"][:t0]), what


def start_runs(blob):
    """Exchange runs recorded in a checkpoint's header."""
    return int(np.frombuffer(blob, np.int64, 1, 56)[0])


def test_facade_full_swarm_trajectory_from_both_initial_swarms():
    """Independent of any GPU state: the GPU and the oracle each build the
    facade's 1024-particle swarm from the same inputs and run generations
    1..4 (generation 3 mutates, Sec. 3.2.2; the edge exchange runs in every
    generation whose gbest did not improve, Sec. 3.2.3); after every
    generation the whole state, history and exchange counters must agree.
    The oracle runs each particle's exchange on one of the host threads."""
    inst, C, C_np = _instance("facade")
    S = inst.swarm
    gpu = dpso.Swarm(C, inst.n, inst.tags, dpso.default_params(swarm=S), inst.seed)
    ref = oracle.Swarm(C_np, inst.tags, swarm=S, seed=inst.seed)
    threads = host_threads()
    for t in range(1, 5):
        gpu.step(1)
        ref.iterate_threaded(threads)
        gs, rs = gpu.state(), ref.state()
        what = f"facade generation {t}"
        _compare(gs, rs, what)
        assert np.array_equal(gs["G"], rs["G"]) and gs["gf"] == rs["gf"], what
        assert np.array_equal(gs["history"], rs["history"]), what
        assert (gs["pairs"], gs["moves"], gs["runs"]) == (rs["pairs"], rs["moves"],
                                                          rs["runs"]), what
    gpu.close()
