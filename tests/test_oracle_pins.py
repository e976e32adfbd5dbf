"""Pins for the CPU oracle against facts fixed outside the oracle itself.

Each test checks the oracle against one of: a published known-answer vector,
the paper's worked example (Sec. 3.1), an exact closed form, an independent
algorithm (exact rational separating-axis test, exact integer square roots,
brute force over all tours), or an invariant the paper's definitions imply.
"""
import itertools
import math
from fractions import Fraction

import numpy as np
import pytest

from conftest import read_golden
from paper_1706_04399_gb300 import inputs


# --------------------------------------------------------------------- Philox

def test_philox_known_answers(oracle_mod):
    for row in read_golden("philox4x32_10_kat.txt"):
        vals = [int(v, 16) for v in row]
        out = oracle_mod.philox4x32_10(vals[:4], vals[4:6])
        assert [int(v) for v in out] == vals[6:10]


def test_philox_draw_layout(oracle_mod):
    # draw d of (seed, phase, iteration, particle) is word d%4 of counter
    # (d//4, particle, iteration, phase) under key (seed lo, seed hi)
    seed = 0x0123456789ABCDEF
    for d in range(9):
        blk = oracle_mod.philox4x32_10([d // 4, 5, 7, 3], [seed & 0xFFFFFFFF, seed >> 32])
        assert oracle_mod.draw(seed, 3, 7, 5, d) == int(blk[d % 4])


def test_philox_bounded_uniformity(oracle_mod):
    # chi-square of 64 bins over 2^14 bounded draws: a gross-bias screen
    counts = np.zeros(64)
    for d in range(1 << 14):
        u = oracle_mod.draw(11, 1, 0, d >> 8, d & 255)
        counts[(u * 64) >> 32] += 1
    exp = (1 << 14) / 64
    chi2 = float(((counts - exp) ** 2 / exp).sum())
    assert 20 < chi2 < 120  # 63 dof


# ------------------------------------------------------------ Sec. 3.1 algebra

def test_worked_example_addition(oracle_mod):
    rows = {r[0]: [int(v) for v in r[1:]] for r in read_golden("sec3_1_worked_example.txt")}
    x = np.array(rows["x"]) - 1
    v = (np.array(rows["v"]) - 1).reshape(-1, 2)
    assert list(oracle_mod.apply(x, v[:1]) + 1) == rows["after1"]
    assert list(oracle_mod.apply(x, v) + 1) == rows["after2"]


def _label_cycles(x2, x1):
    """Cycles of the label map s with s(x1[k]) = x2[k], counted by walking."""
    n = len(x1)
    s = np.empty(n, np.int64)
    s[np.asarray(x1, np.int64)] = np.asarray(x2, np.int64)
    seen = np.zeros(n, bool)
    cyc = 0
    for a in range(n):
        if not seen[a]:
            cyc += 1
            b = a
            while not seen[b]:
                seen[b] = True
                b = s[b]
    return cyc


def test_subtraction_definition_and_minimality(oracle_mod):
    rng = np.random.default_rng(5)
    for _ in range(2000):
        n = int(rng.integers(3, 61))
        x1 = rng.permutation(n).astype(np.uint16)
        x2 = rng.permutation(n).astype(np.uint16)
        v = oracle_mod.subtract(x2, x1)
        assert np.array_equal(oracle_mod.apply(x1, v), x2)      # x1 + (x2 - x1) = x2
        assert len(v) == n - _label_cycles(x2, x1)               # minimal length
    x = rng.permutation(17).astype(np.uint16)
    assert len(oracle_mod.subtract(x, x)) == 0


def test_velocity_concatenation(oracle_mod):
    rng = np.random.default_rng(6)
    for _ in range(500):
        n = int(rng.integers(3, 40))
        x = rng.permutation(n)
        v1 = rng.integers(0, n, size=(int(rng.integers(0, 20)), 2))
        v2 = rng.integers(0, n, size=(int(rng.integers(0, 20)), 2))
        both = np.concatenate([v1, v2]) if len(v1) + len(v2) else np.zeros((0, 2), int)
        assert np.array_equal(oracle_mod.apply(x, both),
                              oracle_mod.apply(oracle_mod.apply(x, v1), v2))


def test_scalar_multiplication_counts(oracle_mod):
    # c.v keeps the first floor(c |v|) transpositions, c = phi * u / 2^32
    assert oracle_mod.scaled_count(0.0, 0xFFFFFFFF, 1000) == 0
    assert oracle_mod.scaled_count(0.4, 0, 1000) == 0
    assert oracle_mod.scaled_count(1.0, 0xFFFFFFFF, 1000) == 999
    rng = np.random.default_rng(7)
    for _ in range(5000):
        phi = float(rng.uniform(0, 1))
        u = int(rng.integers(0, 1 << 32))
        ln = int(rng.integers(0, 70000))
        k = oracle_mod.scaled_count(phi, u, ln)
        c = Fraction(phi) * Fraction(u, 1 << 32)
        assert 0 <= k <= ln
        assert abs(Fraction(k) - c * ln) <= 1


# ----------------------------------------------------------------- cost matrix

def _nearest_mm(k2: int) -> int:
    """Integer nearest to 1000*sqrt(k2), exactly (no floating point)."""
    t = 1_000_000 * k2
    m = math.isqrt(t)
    # choose m+1 when sqrt(t) > m + 1/2, i.e. 4t > (2m+1)^2 (ties impossible)
    return m + 1 if 4 * t > (2 * m + 1) ** 2 else m


def _sat_blocked(p, q, box):
    """Closed segment vs closed box by the separating-axis theorem, exactly."""
    p = [Fraction(v) for v in p]
    q = [Fraction(v) for v in q]
    lo = [Fraction(v) for v in box[:3]]
    hi = [Fraction(v) for v in box[3:]]
    c = [(a + b) / 2 for a, b in zip(lo, hi)]
    e = [(b - a) / 2 for a, b in zip(lo, hi)]
    m = [(p[i] + q[i]) / 2 - c[i] for i in range(3)]
    h = [(q[i] - p[i]) / 2 for i in range(3)]
    for i in range(3):
        if abs(m[i]) > e[i] + abs(h[i]):
            return False
    for i in range(3):
        j, k = (i + 1) % 3, (i + 2) % 3
        if abs(m[j] * h[k] - m[k] * h[j]) > e[j] * abs(h[k]) + e[k] * abs(h[j]):
            return False
    return True


def test_tiny_costs_exact(oracle_mod):
    inst = inputs.tiny()
    C, st = oracle_mod.cost_matrix(inst.xyz, inst.boxes)
    assert st == 0
    golden = {(int(a), int(b)): int(c) for a, b, c in read_golden("tiny_grid_costs.txt")}
    pts = inst.xyz.astype(int)
    seen = 0
    for i in range(inst.n):
        for j in range(inst.n):
            dx, dy = abs(pts[i, 0] - pts[j, 0]), abs(pts[i, 1] - pts[j, 1])
            if i == j:
                assert C[i, j] == 0
                continue
            blocked = _sat_blocked(inst.xyz[i], inst.xyz[j], inst.boxes[0])
            base = _nearest_mm(dx * dx + dy * dy)
            assert C[i, j] == base + (1_000_000 if blocked else 0), (i, j)
            if (dx, dy) in golden:
                assert base == golden[(dx, dy)]
                seen += 1
    assert seen > 0


def test_tiny_blocked_set(oracle_mod):
    inst = inputs.tiny()
    C, _ = oracle_mod.cost_matrix(inst.xyz, inst.boxes)
    node = {(int(x), int(y)): k for k, (x, y, _z) in enumerate(inst.xyz)}
    for a, b in [((2, 2), (3, 2)), ((2, 3), (3, 3)), ((2, 1), (3, 2)), ((0, 0), (5, 4))]:
        assert C[node[a], node[b]] >= 1_000_000
    for a, b in [((2, 1), (3, 1)), ((2, 4), (3, 4)), ((2, 0), (3, 0)), ((2, 2), (2, 3))]:
        assert C[node[a], node[b]] == 1000
    # a comb cycle of 30 unit edges that avoids the box: the optimum, 30 000 mm
    cyc = [(0, y) for y in range(5)] + [(1, y) for y in range(4, 0, -1)] + \
          [(2, y) for y in range(1, 5)] + [(3, y) for y in range(4, 0, -1)] + \
          [(4, y) for y in range(1, 5)] + [(5, y) for y in range(4, -1, -1)] + \
          [(x, 0) for x in range(4, 0, -1)]
    tour = np.array([node[c] for c in cyc], np.uint16)
    assert sorted(tour.tolist()) == list(range(30))
    assert oracle_mod.fitness(C, tour) == 30_000


def test_blocked_random_against_sat(oracle_mod):
    rng = np.random.default_rng(9)
    hits = 0
    for _ in range(3000):
        # small dyadic coordinates: differences are exact and the correctly
        # rounded slab quotients keep every comparison of the exact rationals
        # (distinct quotients differ by far more than an ulp), so the FP64 slab
        # test must agree with the exact separating-axis test, touching included
        p = rng.integers(-16, 17, size=3) / 4
        q = rng.integers(-16, 17, size=3) / 4
        lo = rng.integers(-12, 8, size=3) / 4
        hi = lo + rng.integers(0, 9, size=3) / 4
        box = np.concatenate([lo, hi])
        got = oracle_mod.segment_blocked(p, q, box)
        assert got == _sat_blocked(p, q, box), (p, q, box)
        hits += got
    assert 100 < hits < 2900


def test_cost_matrix_properties(oracle_mod):
    for inst in (inputs.facade(), inputs.random_instance(150, 6, 3)):
        C, st = oracle_mod.cost_matrix(inst.xyz, inst.boxes)
        assert st == 0
        assert np.array_equal(C, C.T)
        assert np.all(np.diag(C) == 0)
        off = C[~np.eye(inst.n, dtype=bool)]
        assert off.min() > 0 and off.max() <= (1 << 29)


def test_cost_matrix_radius_and_inside_point(oracle_mod):
    # segment 0->3 is y = 0.28 x: over x in [4, 5] it stays at y >= 1.12, above
    # the box (y <= 0.5); grown by r it is hit iff 0.28 (4 - r) <= 0.5 + r,
    # i.e. r >= 0.484...
    xyz = np.array([[0, 0, 0], [10, 0, 0], [5, 5, 0], [5, 1.4, 0]], float)
    box = np.array([[4, -0.5, -0.5, 6, 0.5, 0.5]], float)
    C0, _ = oracle_mod.cost_matrix(xyz, box, radius=0.0)
    assert C0[0, 1] == 10_000 + 1_000_000        # straight through the box
    assert C0[0, 3] < 1_000_000                  # passes above it
    C1, _ = oracle_mod.cost_matrix(xyz, box, radius=0.2)
    assert C1[0, 3] < 1_000_000
    C2, _ = oracle_mod.cost_matrix(xyz, box, radius=0.5)
    assert C2[0, 3] >= 1_000_000                 # the grown box now meets it
    inside = np.array([[5, 0, 0], [0, 9, 0], [9, 9, 0]], float)
    C3, _ = oracle_mod.cost_matrix(inside, box)
    assert C3[0, 1] >= 1_000_000 and C3[0, 2] >= 1_000_000 and C3[1, 2] < 1_000_000


def test_cost_matrix_range_error(oracle_mod):
    xyz = np.array([[0, 0, 0], [600_000, 0, 0], [0, 1, 0]], float)  # 600 km > 2^29 mm
    _, st = oracle_mod.cost_matrix(xyz, np.zeros((0, 6)))
    assert st == oracle_mod.ERR_RANGE


# ---------------------------------------------------- tours, brute force, grids

def _brute_force(C):
    n = C.shape[0]
    best = None
    for perm in itertools.permutations(range(1, n)):
        if perm[0] > perm[-1]:
            continue  # each cycle once per direction
        tour = (0,) + perm
        cost = sum(int(C[tour[k], tour[(k + 1) % n]]) for k in range(n))
        best = cost if best is None else min(best, cost)
    return best


@pytest.mark.parametrize("n,seed", [(5, 1), (6, 2), (7, 3), (8, 4), (9, 5)])
def test_brute_force_bounds_solver(oracle_mod, n, seed):
    inst = inputs.random_instance(n, 2, seed, swarm=16)
    C, _ = oracle_mod.cost_matrix(inst.xyz, inst.boxes)
    opt = _brute_force(C)
    rng = np.random.default_rng(seed)
    for _ in range(20):
        _t, f, _m, _p = oracle_mod.two_opt(C, rng.permutation(n))
        assert f >= opt
    sw = oracle_mod.Swarm(C, inst.tags, swarm=16, seed=seed)
    sw.run(30)
    assert sw.gf >= opt
    assert sw.gf == opt            # small instances: the swarm reaches the optimum
    assert oracle_mod.fitness(C, sw.state()["G"]) == sw.gf


def test_even_grid_closed_form(oracle_mod):
    # obstacle-free m x n grid with m*n even: optimum = N * spacing
    inst = inputs.planar_grid(8, 1.5, np.zeros((0, 6)), "g8", 16, 30, 3)
    C, _ = oracle_mod.cost_matrix(inst.xyz, inst.boxes)
    assert _brute_force(C) == 8 * 1500
    inst = inputs.planar_grid(16, 1.0, np.zeros((0, 6)), "g16", 32, 40, 4)
    C, _ = oracle_mod.cost_matrix(inst.xyz, inst.boxes)
    sw = oracle_mod.Swarm(C, inst.tags, swarm=32, seed=4)
    sw.run(40)
    assert sw.gf == 16 * 1000


def test_tiny_reaches_closed_form_optimum(oracle_mod):
    inst = inputs.tiny()
    C, _ = oracle_mod.cost_matrix(inst.xyz, inst.boxes)
    sw = oracle_mod.Swarm(C, inst.tags, swarm=inst.swarm, seed=inst.seed)
    sw.run(inst.iterations)
    assert sw.gf == 30_000
    assert sw.t == inst.iterations


# --------------------------------------------------- deterministic initialisation

def test_boustrophedon_closed_forms(oracle_mod):
    inst = inputs.tiny()
    C, _ = oracle_mod.cost_matrix(inst.xyz, inst.boxes)
    for s in range(8):
        order, st = oracle_mod.boustrophedon(inst.tags, s)
        assert st == 0 and sorted(order.tolist()) == list(range(30))
        f = oracle_mod.fitness(C, order)
        if s & 1:
            # column snake: 24 in-column + 5 between-column unit edges, 5 m closing edge
            assert f == 29 * 1000 + 5000
        else:
            # row snake over 5 rows ends at (5,4); two row edges cross the box and
            # the closing edge (5,4)->(0,0) passes through it: 3 penalties
            assert f == 29 * 1000 + _nearest_mm(41) + 3 * 1_000_000
    # consecutive nodes of a snake are grid neighbours except at the seam
    order, _ = oracle_mod.boustrophedon(inst.tags, 1)
    steps = np.abs(np.diff(inst.xyz[order.astype(int)], axis=0)).sum(axis=1)
    assert np.all(steps == 1.0)


def test_boustrophedon_rejects_duplicate_tags(oracle_mod):
    tags = np.array([[0, 0, 0], [0, 0, 1], [0, 0, 1]], np.int32)
    _, st = oracle_mod.boustrophedon(tags, 0)
    assert st == oracle_mod.ERR_ARG


def test_init_layout(oracle_mod):
    inst = inputs.tiny()
    C, _ = oracle_mod.cost_matrix(inst.xyz, inst.boxes)
    sw = oracle_mod.Swarm(C, inst.tags, swarm=32, seed=1)
    st = sw.state()
    # n_det = max(1, floor(32 * 10 / 100)) = 3 back-and-forth particles
    for p in range(3):
        order, _ = oracle_mod.boustrophedon(inst.tags, p % 8)
        assert np.array_equal(st["X"][p], np.roll(order, -(p // 8)))
    for p in range(32):
        assert sorted(st["X"][p].tolist()) == list(range(30))
        assert st["F"][p] == oracle_mod.fitness(C, st["X"][p]) == st["PF"][p]
    assert np.array_equal(st["X"], st["P"])
    assert np.all(st["V"] == np.arange(30))       # empty velocities
    assert st["gf"] == st["F"].min() == 34_000     # a column snake is the best seed


# ------------------------------------------------------------------- 2-opt

def _deltas(C, x):
    n = len(x)
    x = np.asarray(x, np.int64)
    nxt = np.roll(x, -1)
    D = (C[x[:, None], x[None, :]].astype(np.int64) + C[nxt[:, None], nxt[None, :]]
         - C[x, nxt][:, None] - C[x, nxt][None, :])
    i, j = np.indices((n, n))
    valid = (j >= i + 2) & ~((i == 0) & (j == n - 1))
    return np.where(valid, D, np.iinfo(np.int64).max)


@pytest.mark.parametrize("n", [3, 4, 5, 10, 37, 64])
def test_two_opt_optimality_and_moves(oracle_mod, n):
    C = inputs.random_cost_matrix(n, 100 + n)
    rng = np.random.default_rng(n)
    for _ in range(3):
        x = rng.permutation(n).astype(np.uint16)
        y, f, moves, pairs = oracle_mod.two_opt(C, x)
        assert sorted(y.tolist()) == list(range(n))
        assert f == oracle_mod.fitness(C, y)
        assert _deltas(C, y).min(initial=0) >= 0            # 2-optimal
        assert pairs == (moves + 1) * (n * (n - 3) // 2)
        # one move at a time: each is the lexicographic argmin of the deltas
        cur = x.copy()
        for _k in range(moves):
            D = _deltas(C, cur)
            flat = int(np.argmin(D))
            i, j = divmod(flat, n)
            nxt, f2, m1, _ = oracle_mod.two_opt(C, cur, max_moves=1)
            assert m1 == 1 and D[i, j] < 0
            assert f2 - oracle_mod.fitness(C, cur) == D[i, j]
            exp = cur.copy()
            exp[i + 1:j + 1] = exp[i + 1:j + 1][::-1]
            assert np.array_equal(nxt, exp)
            cur = nxt
        assert np.array_equal(cur, y)


def _swap_deltas_brute(oracle_mod, C, x):
    """Change of the full recomputed tour length for swapping positions i < j."""
    n = len(x)
    f0 = oracle_mod.fitness(C, x)
    D = np.full((n, n), np.iinfo(np.int64).max, np.int64)
    for i in range(n):
        for j in range(i + 1, n):
            y = x.copy()
            y[i], y[j] = y[j], y[i]
            D[i, j] = oracle_mod.fitness(C, y) - f0
    return D


@pytest.mark.parametrize("n", [3, 4, 5, 6, 9, 23])
def test_node_swap_optimality_and_moves(oracle_mod, n):
    """Node-swap exchange: every applied swap is the lexicographic argmin of the
    brute-force swap deltas (adjacent pairs and the wrap pair (0, n-1)
    included), the output admits no improving swap, and each pass evaluates
    n(n-1)/2 pairs."""
    C = inputs.random_cost_matrix(n, 300 + n)
    rng = np.random.default_rng(7 * n)
    for _ in range(3):
        x = rng.permutation(n).astype(np.uint16)
        y, f, moves, pairs = oracle_mod.node_swap(C, x)
        assert sorted(y.tolist()) == list(range(n))
        assert f == oracle_mod.fitness(C, y)
        assert _swap_deltas_brute(oracle_mod, C, y).min() >= 0
        assert pairs == (moves + 1) * (n * (n - 1) // 2)
        if n == 3:
            assert moves == 0  # a swap only reverses a 3-cycle
        cur = x.copy()
        for _k in range(moves):
            D = _swap_deltas_brute(oracle_mod, C, cur)
            i, j = divmod(int(np.argmin(D)), n)
            nxt, f2, m1, _ = oracle_mod.node_swap(C, cur, max_moves=1)
            assert m1 == 1 and D[i, j] < 0
            assert f2 - oracle_mod.fitness(C, cur) == D[i, j]
            exp = cur.copy()
            exp[i], exp[j] = exp[j], exp[i]
            assert np.array_equal(nxt, exp)
            cur = nxt
        assert np.array_equal(cur, y)


def test_node_swap_wrap_and_adjacent_pairs(oracle_mod):
    """Points on a circle visited in order except two neighbours exchanged: the
    only improving swap restores the order, whether the exchanged pair sits in
    the middle of the array (adjacent positions) or at its two ends (the wrap
    pair (0, n-1))."""
    n = 12
    ang = 2 * np.pi * np.arange(n) / n
    xyz = np.stack([10 * np.cos(ang), 10 * np.sin(ang), np.zeros(n)], axis=1)
    C, _ = oracle_mod.cost_matrix(xyz, np.zeros((0, 6)))
    opt = oracle_mod.fitness(C, np.arange(n, dtype=np.uint16))
    for i, j in ((4, 5), (0, n - 1)):
        x = np.arange(n, dtype=np.uint16)
        x[i], x[j] = x[j], x[i]
        y, f, moves, _ = oracle_mod.node_swap(C, x, max_moves=1)
        assert moves == 1 and f == opt
        assert oracle_mod.fitness(C, y) == opt


# ---------------------------------------------------------------- mutation

def test_mutation_keeps_best_third_unchanged(oracle_mod):
    inst = inputs.random_instance(40, 3, 21)
    C, _ = oracle_mod.cost_matrix(inst.xyz, inst.boxes)
    S = 31
    sw = oracle_mod.Swarm(C, inst.tags, swarm=S, seed=5, flags=oracle_mod.DET_INIT)
    sw.run(2)
    before = sw.state()
    kept = sw.mutate(3)
    after = sw.state()
    uniq = len(np.unique(before["X"], axis=0))
    K = -(-S // 3)
    assert kept.sum() == min(K, uniq)
    assert np.array_equal(after["X"][kept], before["X"][kept])
    order = np.lexsort((np.arange(S), before["F"]))
    # kept are the first K distinct tours in (fitness, index) order
    exp, seen = [], set()
    for p in order:
        key = before["X"][p].tobytes()
        if key not in seen:
            seen.add(key)
            if len(exp) < K:
                exp.append(p)
    assert sorted(exp) == sorted(np.nonzero(kept)[0].tolist())
    for p in np.nonzero(~kept)[0]:
        assert sorted(after["X"][p].tolist()) == list(range(40))
        assert np.count_nonzero(after["X"][p] != before["X"][p]) <= 4   # 2 swaps
        assert sw.vel_len(int(p)) == 0
        assert after["F"][p] == oracle_mod.fitness(C, after["X"][p])


def test_mutation_duplicates_are_disturbed(oracle_mod):
    # one row of 4 viewpoints: the 8 back-and-forth variants collapse to two
    # distinct arrays, so 8 particles hold only 2 distinct tours
    inst = inputs.planar_grid(4, 1.0, np.zeros((0, 6)), "row", 8, 1, 1)
    inst.tags[:, 1] = 0
    inst.tags[:, 2] = np.arange(4)
    C, _ = oracle_mod.cost_matrix(inst.xyz, inst.boxes)
    sw = oracle_mod.Swarm(C, inst.tags, swarm=8, det_frac_pct=100, seed=2,
                          flags=oracle_mod.DET_INIT)
    st = sw.state()
    uniq = len(np.unique(st["X"], axis=0))
    assert uniq < 8
    kept = sw.mutate(3)
    assert kept.sum() == min(3, uniq)


# ------------------------------------------------------------------ the loop

@pytest.mark.parametrize("w", [1.0, 0.5, 0.0])
def test_loop_invariants(oracle_mod, w):
    inst = inputs.random_instance(30, 3, 31)
    C, _ = oracle_mod.cost_matrix(inst.xyz, inst.boxes)
    sw = oracle_mod.Swarm(C, inst.tags, swarm=24, w=w, seed=3)
    ran_two_opt = False
    for _ in range(15):
        sw.iterate()
        st = sw.state()
        for p in range(24):
            assert sorted(st["X"][p].tolist()) == list(range(30))
            assert sorted(st["P"][p].tolist()) == list(range(30))
            assert st["F"][p] == oracle_mod.fitness(C, st["X"][p])
            assert st["PF"][p] == oracle_mod.fitness(C, st["P"][p])
            assert st["PF"][p] <= st["F"][p]
        assert st["gf"] == st["PF"].min() == oracle_mod.fitness(C, st["G"])
        if sw.last_two_opt:
            ran_two_opt = True
            for p in range(24):
                assert _deltas(C, st["X"][p]).min(initial=0) >= 0
    h = sw.history()
    assert len(h) == 15 and np.all(np.diff(h) <= 0)
    assert ran_two_opt


def test_velocity_list_matches_permutation(oracle_mod):
    # with w = 1 the list is never truncated, so x_{k+1} = V o x_k exactly
    inst = inputs.random_instance(25, 2, 41)
    C, _ = oracle_mod.cost_matrix(inst.xyz, inst.boxes)
    sw = oracle_mod.Swarm(C, inst.tags, swarm=8, seed=9, flags=0)
    for t in range(1, 6):
        x0 = sw.state()["X"]
        sw.move(t)
        st = sw.state()
        for p in range(8):
            assert np.array_equal(st["V"][p][x0[p].astype(int)], st["X"][p])


def test_stall_limit_and_trigger(oracle_mod):
    inst = inputs.tiny()
    C, _ = oracle_mod.cost_matrix(inst.xyz, inst.boxes)
    sw = oracle_mod.Swarm(C, inst.tags, swarm=32, stall_limit=4, seed=1)
    sw.run(200)
    assert sw.done and sw.t < 200 and sw.stall == 4
    sw = oracle_mod.Swarm(C, inst.tags, swarm=32, trigger=1, seed=1)
    ran = []
    for t in range(1, 13):
        sw.iterate()
        if sw.last_two_opt:
            ran.append(t)
    assert ran and all(t % 3 == 0 for t in ran)   # only in mutation generations


def test_swarm_rejects_bad_arguments(oracle_mod):
    C = inputs.random_cost_matrix(5, 1)
    for kw in ({"swarm": 0}, {"w": 1.5}, {"phi1": -0.1}, {"mut_period": 0}, {"trigger": 2}):
        with pytest.raises(ValueError):
            oracle_mod.Swarm(C, None, **kw)
    with pytest.raises(ValueError):
        oracle_mod.Swarm(inputs.random_cost_matrix(2, 1), None)


def test_costs_exact_3d_integer_points(oracle_mod):
    # integer coordinates in metres: the cost is the integer nearest to
    # 1000 * sqrt(dx^2 + dy^2 + dz^2), computed here with exact integer roots
    rng = np.random.default_rng(12)
    pts = rng.integers(-40, 41, size=(60, 3)).astype(float)
    C, st = oracle_mod.cost_matrix(pts, np.zeros((0, 6)))
    assert st == 0
    for i in range(60):
        for j in range(60):
            d2 = int(((pts[i] - pts[j]) ** 2).sum())
            assert C[i, j] == (_nearest_mm(d2) if i != j else 0)


def test_loop_invariants_without_edge_exchange(oracle_mod):
    inst = inputs.random_instance(30, 3, 33)
    C, _ = oracle_mod.cost_matrix(inst.xyz, inst.boxes)
    sw = oracle_mod.Swarm(C, inst.tags, swarm=24, seed=4,
                          flags=oracle_mod.DET_INIT | oracle_mod.MUTATION)
    prev_G, prev_gf = sw.state()["G"], sw.gf
    for _ in range(12):
        sw.iterate()
        st = sw.state()
        assert st["gf"] == st["PF"].min() == oracle_mod.fitness(C, st["G"])
        if st["gf"] == prev_gf:
            assert np.array_equal(st["G"], prev_G)     # replaced only on strict improvement
        else:
            best = int(np.flatnonzero(st["PF"] == st["PF"].min())[0])
            assert np.array_equal(st["G"], st["P"][best])
        prev_G, prev_gf = st["G"], st["gf"]


def test_move_equation_wiring(oracle_mod):
    # Eq. (velocity): phi1 r1 scales (P - x) with draw 0, phi2 r2 scales (G - x)
    # with draw 1; at t=1 every pbest equals its position, so P - x is empty
    inst = inputs.random_instance(40, 2, 51)
    C, _ = oracle_mod.cost_matrix(inst.xyz, inst.boxes)
    seed = 77
    sw = oracle_mod.Swarm(C, None, swarm=6, phi1=0.9, phi2=0.3, seed=seed, flags=0)
    s0 = sw.state()
    sw.move(1)
    s1 = sw.state()
    for p in range(6):
        b = oracle_mod.subtract(s0["G"], s0["X"][p])
        kb = oracle_mod.scaled_count(0.3, oracle_mod.draw(seed, 2, 1, p, 1), len(b))
        assert sw.vel_len(p) == kb
        assert np.array_equal(s1["X"][p], oracle_mod.apply(s0["X"][p], b[:kb]))
    # t=2: v2 = v1 (+) a (+) b, both against x1; x2 = x1 + v2 (w = 1)
    sw.move(2)
    s2 = sw.state()
    nonempty = 0
    for p in range(6):
        b1 = oracle_mod.subtract(s0["G"], s0["X"][p])
        v1 = b1[:oracle_mod.scaled_count(0.3, oracle_mod.draw(seed, 2, 1, p, 1), len(b1))]
        a = oracle_mod.subtract(s1["P"][p], s1["X"][p])
        ka = oracle_mod.scaled_count(0.9, oracle_mod.draw(seed, 2, 2, p, 0), len(a))
        b = oracle_mod.subtract(s1["G"], s1["X"][p])
        kb = oracle_mod.scaled_count(0.3, oracle_mod.draw(seed, 2, 2, p, 1), len(b))
        nonempty += ka > 0
        v2 = np.concatenate([v1, a[:ka], b[:kb]])
        assert sw.vel_len(p) == len(v2)
        assert np.array_equal(s2["X"][p], oracle_mod.apply(s1["X"][p], v2))
    assert nonempty > 0


@pytest.mark.parametrize("w", [0.0, 0.5])
def test_inertia_truncates_canonical_velocity(oracle_mod, w):
    # w.v keeps the first floor(w |v|) transpositions of the velocity's
    # canonical list (identity + v) - identity; w = 0 drops it entirely
    inst = inputs.random_instance(40, 2, 52)
    C, _ = oracle_mod.cost_matrix(inst.xyz, inst.boxes)
    seed = 78
    sw = oracle_mod.Swarm(C, None, swarm=6, w=w, phi1=0.9, phi2=0.3, seed=seed, flags=0)
    sw.move(1)
    s1 = sw.state()
    lens1 = [sw.vel_len(p) for p in range(6)]
    sw.move(2)
    s2 = sw.state()
    ident = np.arange(40)
    for p in range(6):
        canon = oracle_mod.subtract(s1["V"][p], ident)
        assert len(canon) <= lens1[p]
        keep = int(np.floor(w * len(canon)))
        a = oracle_mod.subtract(s1["P"][p], s1["X"][p])
        ka = oracle_mod.scaled_count(0.9, oracle_mod.draw(seed, 2, 2, p, 0), len(a))
        b = oracle_mod.subtract(s1["G"], s1["X"][p])
        kb = oracle_mod.scaled_count(0.3, oracle_mod.draw(seed, 2, 2, p, 1), len(b))
        assert sw.vel_len(p) == keep + ka + kb
        v2 = np.concatenate([canon[:keep], a[:ka], b[:kb]])
        assert np.array_equal(s2["X"][p], oracle_mod.apply(s1["X"][p], v2))


# ------------------------------------------------------------ A* edge costs

def _grid_graph(occ, weights):
    """Sparse 26-neighbour graph of the free voxels (for scipy's Dijkstra)."""
    from scipy.sparse import coo_matrix
    nz, ny, nx = occ.shape
    rows, cols, vals = [], [], []
    idx = np.arange(nx * ny * nz).reshape(nz, ny, nx)
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                if not (dx or dy or dz):
                    continue
                zs = slice(max(0, -dz), nz - max(0, dz))
                ys = slice(max(0, -dy), ny - max(0, dy))
                xs = slice(max(0, -dx), nx - max(0, dx))
                zt = slice(max(0, dz), nz - max(0, -dz))
                yt = slice(max(0, dy), ny - max(0, -dy))
                xt = slice(max(0, dx), nx - max(0, -dx))
                ok = (occ[zs, ys, xs] == 0) & (occ[zt, yt, xt] == 0)
                rows.append(idx[zs, ys, xs][ok])
                cols.append(idx[zt, yt, xt][ok])
                w = weights[0] * dx * dx + weights[1] * dy * dy + weights[2] * dz * dz
                vals.append(np.full(int(ok.sum()), w, np.float64))
    n = nx * ny * nz
    return coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(n, n)).tocsr()


def test_voxel_occupancy_hand_case(oracle_mod):
    """Two voxel centres in a closed box (one face touching), then the
    6-neighbour shell for an inflation radius of one voxel."""
    dims = (6, 5, 3)
    box = [(1.2, 1.0, 0.5, 2.8, 1.9, 0.5)]  # centres (1.5|2.5, 1.5, 0.5): z on the face
    occ = oracle_mod.voxel_occupancy((0, 0, 0), 1.0, dims, box, 0)
    core = {(1, 1, 0), (2, 1, 0)}
    assert {tuple(v[::-1]) for v in np.argwhere(occ)} == core
    occ1 = oracle_mod.voxel_occupancy((0, 0, 0), 1.0, dims, box, 1)
    shell = {(0, 1, 0), (1, 0, 0), (1, 2, 0), (1, 1, 1), (3, 1, 0), (2, 0, 0), (2, 2, 0), (2, 1, 1)}
    assert {tuple(v[::-1]) for v in np.argwhere(occ1)} == core | shell


def test_astar_single_axis_corridors_pin_the_weights(oracle_mod):
    """In a one-voxel-wide corridor along an axis the only path is straight:
    cost = that axis' weight x the voxel count (pins the weight of each axis)."""
    weights = (2, 3, 5)
    for axis in range(3):
        dims = [1, 1, 1]
        dims[axis] = 9
        xyz = np.zeros((2, 3))
        xyz[0, axis], xyz[1, axis] = 0.5, 7.5
        occ = np.zeros(dims[::-1], np.uint8)
        C, st = oracle_mod.cost_matrix_astar(xyz, occ, (0, 0, 0), 1.0, dims, weights, unit_mm=1)
        assert st == 0 and C[0, 1] == C[1, 0] == 7 * weights[axis]


def test_astar_empty_grid_unit_weights_is_manhattan(oracle_mod):
    """Unit weights on an empty grid: every step moving toward the goal costs
    the number of axes it moves, so the cost is the Manhattan distance."""
    dims = (9, 8, 7)
    rng = np.random.default_rng(3)
    pts = rng.integers(0, dims, size=(12, 3)) + 0.5
    occ = np.zeros(dims[::-1], np.uint8)
    C, st = oracle_mod.cost_matrix_astar(pts, occ, (0, 0, 0), 1.0, dims, (1, 1, 1), unit_mm=1)
    man = np.abs(pts[:, None, :] - pts[None, :, :]).sum(axis=2)
    assert st == 0 and np.array_equal(C, man.astype(np.int32))


@pytest.mark.parametrize("weights", [(1, 1, 1), (1, 2, 3)])
def test_astar_cost_is_at_least_the_shortest_path(oracle_mod, weights):
    """The heuristic is the squared distance (not admissible), so A* may miss
    the shortest path but never beats it: compare with scipy's Dijkstra on
    the same voxel graph; unreachable goals get the blocked cost."""
    from scipy.sparse.csgraph import dijkstra
    dims = (10, 9, 4)
    rng = np.random.default_rng(sum(weights))
    boxes = []
    for _ in range(6):
        lo = rng.uniform(0, (10, 9, 4))
        boxes.append(tuple(lo) + tuple(lo + rng.uniform(0.5, 3.0, 3)))
    occ = oracle_mod.voxel_occupancy((0, 0, 0), 1.0, dims, boxes, 0)
    free = np.argwhere(occ == 0)
    pick = free[rng.choice(len(free), 14, replace=False)]
    pts = pick[:, ::-1] + 0.5
    C, st = oracle_mod.cost_matrix_astar(pts, occ, (0, 0, 0), 1.0, dims, weights, unit_mm=1,
                                         blocked_cost=10 ** 6)
    G = _grid_graph(occ, weights)
    src = [(int(z) * 9 + int(y)) * 10 + int(x) for z, y, x in pick]
    D = dijkstra(G, indices=src)[:, src]
    for i in range(len(src)):
        for j in range(i + 1, len(src)):
            if np.isinf(D[i, j]):
                assert C[i, j] == 10 ** 6
            else:
                assert C[i, j] >= D[i, j]


def test_astar_blocked_cases(oracle_mod):
    dims = (7, 7, 3)
    # the goal voxel (3, 3, 1) is walled in on all 26 sides
    boxes = [(2.0, 2.0, 0.0, 5.0, 5.0, 3.0)]
    occ = oracle_mod.voxel_occupancy((0, 0, 0), 1.0, dims, boxes, 0)
    occ[1, 3, 3] = 0
    pts = np.array([[0.5, 0.5, 0.5], [3.5, 3.5, 1.5], [6.5, 6.5, 2.5], [9.0, 1.0, 1.0]])
    C, st = oracle_mod.cost_matrix_astar(pts, occ, (0, 0, 0), 1.0, dims, unit_mm=1,
                                         blocked_cost=777)
    assert C[0, 1] == C[1, 2] == 777          # enclosed goal
    assert C[0, 3] == C[3, 2] == 777          # outside the grid
    assert C[0, 2] not in (0, 777)
    # an expansion cap of zero reaches only the start voxel itself
    C0, _ = oracle_mod.cost_matrix_astar(pts[[0, 0, 2]], occ, (0, 0, 0), 1.0, dims, unit_mm=1,
                                         blocked_cost=777, max_expansions=0)
    assert C0[0, 1] == 0 and C0[0, 2] == 777


def test_astar_squared_heuristic_trap(oracle_mod):
    """The squared heuristic is not admissible: on a 5 x 4 grid with one
    obstacle at (1, 2), from (3, 3) to (0, 2) the shortest path costs 4 (two
    face steps and a diagonal), but the search, traced by hand, pops (2, 2)
    (f = 2 + 4), then (1, 1) (f = 4 + 2, before (1, 3) by index), from which
    the goal enters the open list at g = 6 with h = 0 and is popped first."""
    occ = np.zeros((1, 4, 5), np.uint8)
    occ[0, 2, 1] = 1
    pts = np.array([[3.5, 3.5, 0.5], [0.5, 2.5, 0.5]])
    C, st = oracle_mod.cost_matrix_astar(pts, occ, (0, 0, 0), 1.0, (5, 4, 1), unit_mm=1)
    assert st == 0 and C[0, 1] == 6


def test_fitness_sums_past_the_int32_range(oracle_mod):
    # Eq. (min) over a complete graph whose off-diagonal costs are all K: any
    # tour costs exactly n*K, here far past 2^31 (the sum must be 64-bit)
    n, K = 400, 1 << 29
    C = np.full((n, n), K, dtype=np.int32)
    np.fill_diagonal(C, 0)
    rng = np.random.default_rng(3)
    for _ in range(3):
        x = rng.permutation(n).astype(np.uint16)
        assert oracle_mod.fitness(C, x) == n * K
    # one cheaper edge pair on the tour lowers the cost by exactly its saving
    x = np.arange(n, dtype=np.uint16)
    C[5, 6] = C[6, 5] = 7
    assert oracle_mod.fitness(C, x) == (n - 1) * K + 7


# ------------------------------------------------------------- snapshot replay

IMPORT_CASES = {
    "default": {},
    "w_half": dict(w=0.5),
    "w_zero": dict(w=0.0, phi1=0.7, phi2=0.9),
    "trigger1": dict(trigger=1),
    "period2_swaps5": dict(mut_period=2, mut_swaps=5, det_frac_pct=40),
    "stall": dict(stall_limit=3),
    "node_swap": dict(flags=7 | 8),
    "max_moves": dict(max_moves=2),
}


@pytest.mark.parametrize("case", list(IMPORT_CASES))
def test_import_continues_an_uninterrupted_run(oracle_mod, case):
    """A state exported at generation k and imported into a fresh swarm
    continues exactly as the run it came from (every array, the history, the
    loop state and the exchange counters), for every generation kind."""
    inst = inputs.random_instance(33, 3, 61)
    C, _ = oracle_mod.cost_matrix(inst.xyz, inst.boxes)
    kw = IMPORT_CASES[case]
    for k in (0, 1, 2, 3, 7):
        a = oracle_mod.Swarm(C, inst.tags, swarm=21, seed=17, **kw)
        a.run(k)
        b = oracle_mod.Swarm(C, inst.tags, swarm=21, seed=17, **kw)
        b.load_state(a.state())
        for _ in range(6):
            a.iterate()
            b.iterate()
            sa, sb = a.state(), b.state()
            for key in sa:
                assert np.array_equal(sa[key], sb[key]), (case, k, key, sa["t"])


def test_import_stores_minimal_velocities(oracle_mod):
    """An imported velocity becomes the subtraction's list for its
    permutation: n - cycles transpositions (Sec. 3.1: x1 + (x2 - x1) = x2),
    and with w = 1 the next position is that permutation applied after the
    two new terms' transpositions: x' = V' o x for the new velocity V'."""
    inst = inputs.random_instance(29, 2, 62)
    C, _ = oracle_mod.cost_matrix(inst.xyz, inst.boxes)
    sw = oracle_mod.Swarm(C, inst.tags, swarm=12, seed=3, flags=0)
    st = sw.state()
    rng = np.random.default_rng(11)
    ident = np.arange(29, dtype=np.uint16)
    st["V"] = np.stack([rng.permutation(29) for _ in range(12)]).astype(np.uint16)
    sw.load_state(st)
    for p in range(12):
        assert sw.vel_len(p) == 29 - _label_cycles(st["V"][p], ident)
    x0 = sw.state()["X"]
    sw.move(1)
    after = sw.state()
    for p in range(12):
        assert np.array_equal(after["V"][p][x0[p].astype(int)], after["X"][p])


def test_import_rejects_non_permutations(oracle_mod):
    inst = inputs.random_instance(15, 1, 63)
    C, _ = oracle_mod.cost_matrix(inst.xyz, inst.boxes)
    sw = oracle_mod.Swarm(C, inst.tags, swarm=6, seed=2)
    sw.run(2)
    good = sw.state()
    for key in ("X", "P", "V"):
        bad = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in good.items()}
        bad[key][3, 4] = bad[key][3, 5]
        with pytest.raises(ValueError):
            sw.load_state(bad)
    bad = dict(good, G=np.zeros(15, np.uint16))
    with pytest.raises(ValueError):
        sw.load_state(bad)
    after = sw.state()                    # a rejected import leaves the swarm alone
    for key in good:
        assert np.array_equal(good[key], after[key]), key


def test_threaded_exchange_equals_serial_generation(oracle_mod):
    """The generation split around the exchange, with the exchange run by
    several threads on disjoint particles, equals iterate()."""
    inst = inputs.random_instance(48, 3, 64)
    C, _ = oracle_mod.cost_matrix(inst.xyz, inst.boxes)
    a = oracle_mod.Swarm(C, inst.tags, swarm=30, seed=8)
    b = oracle_mod.Swarm(C, inst.tags, swarm=30, seed=8)
    ran = 0
    for _ in range(8):
        a.iterate()
        ran += b.iterate_threaded(threads=4)
        sa, sb = a.state(), b.state()
        for key in sa:
            assert np.array_equal(sa[key], sb[key]), (key, sa["t"])
    assert ran > 0
    # with a sample only those particles are exchanged and the generation stays open
    c = oracle_mod.Swarm(C, inst.tags, swarm=30, seed=8)
    c.load_state(a.state())
    a.iterate()
    if c.iterate_threaded(threads=3, sample=[2, 17, 29]):
        sa, sc = a.state(), c.state()
        for p in (2, 17, 29):
            assert np.array_equal(sa["X"][p], sc["X"][p]) and sa["F"][p] == sc["F"][p]
        with pytest.raises(RuntimeError):
            c.iterate_begin()             # still open
