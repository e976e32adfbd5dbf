"""GPU parity of the standalone kernels against the CPU oracle, through the C ABI.

Integer and index results must be bit-exact (the cost matrix included: the
FP64 steps are IEEE round-to-nearest on both sides).
"""
import numpy as np
import pytest

from gpu_helpers import DEV, cost_matrix_gpu, torch  # noqa: F401
import oracle
from paper_1706_04399_gb300 import dpso, inputs

pytestmark = pytest.mark.gpu


# -------------------------------------------------------------------- Philox

@pytest.mark.parametrize("seed,phase,it,part", [(1, 1, 0, 0), (2, 2, 7, 1023),
                                                 (0xFFFFFFFFFFFFFFFF, 3, 123456, 65534),
                                                 (0x0123456789ABCDEF, 2, 1, 5)])
def test_philox_stream_matches_oracle(seed, phase, it, part):
    count = 1 << 18
    out = torch.empty(count, dtype=torch.int32, device=DEV)
    dpso.dpso_philox_draws(seed, phase, it, part, count, out)
    torch.cuda.synchronize()
    got = out.cpu().numpy().view(np.uint32)
    assert np.array_equal(got, oracle.draws(seed, phase, it, part, count))


# ---------------------------------------------------------------- cost matrix

@pytest.mark.parametrize("name", ["tiny", "facade", "bridge"])
def test_cost_matrix_bitwise(name):
    inst = inputs.CONFIGS[name]()
    C = cost_matrix_gpu(inst).cpu().numpy()
    ref, st = oracle.cost_matrix(inst.xyz, inst.boxes)
    assert st == 0
    assert np.array_equal(C, ref)


@pytest.mark.parametrize("n,m,radius", [(1, 0, 0.0), (2, 1, 0.0), (3, 0, 0.0), (33, 4, 0.3),
                                        (257, 300, 0.0), (700, 12, 0.25)])
def test_cost_matrix_random_bitwise(n, m, radius):
    inst = inputs.random_instance(n, m, 1000 + n)
    C = cost_matrix_gpu(inst, radius=radius).cpu().numpy()
    ref, st = oracle.cost_matrix(inst.xyz, inst.boxes, radius=radius)
    assert st == 0
    assert np.array_equal(C, ref)


def test_cost_matrix_dyadic_touching_bitwise():
    # segments that graze faces, edges and corners exactly
    rng = np.random.default_rng(4)
    pts = rng.integers(-8, 9, size=(300, 3)) / 4.0
    boxes = []
    for _ in range(40):
        lo = rng.integers(-6, 6, size=3) / 4.0
        boxes.append(np.concatenate([lo, lo + rng.integers(0, 5, size=3) / 4.0]))
    inst = inputs.Instance("dyadic", pts, np.zeros((300, 3), np.int32), np.array(boxes), 1, 1, 1)
    C = cost_matrix_gpu(inst).cpu().numpy()
    ref, _ = oracle.cost_matrix(inst.xyz, inst.boxes)
    assert np.array_equal(C, ref)


def test_cost_matrix_errors():
    inst = inputs.random_instance(10, 2, 3)
    bad = inst.xyz.copy()
    bad[3, 1] = np.nan
    xyz = torch.from_numpy(bad).to(DEV)
    boxes = torch.from_numpy(inst.boxes).to(DEV)
    C = torch.empty((10, 10), dtype=torch.int32, device=DEV)
    cp = dpso.default_cost_params()
    with pytest.raises(dpso.DpsoError) as e:
        dpso.dpso_cost_matrix(xyz, 10, boxes, 2, cp, C)
    assert e.value.status == dpso.ERR_ARG
    inv = inst.boxes.copy()
    inv[0, 0], inv[0, 3] = inv[0, 3], inv[0, 0] - 1
    with pytest.raises(dpso.DpsoError) as e:
        dpso.dpso_cost_matrix(torch.from_numpy(inst.xyz).to(DEV), 10,
                              torch.from_numpy(inv).to(DEV), 2, cp, C)
    assert e.value.status == dpso.ERR_ARG
    far = np.array([[0, 0, 0], [600_000, 0, 0], [0, 1, 0]], float)
    C3 = torch.empty((3, 3), dtype=torch.int32, device=DEV)
    with pytest.raises(dpso.DpsoError) as e:
        dpso.dpso_cost_matrix(torch.from_numpy(far).to(DEV), 3, None, 0, cp, C3)
    assert e.value.status == dpso.ERR_RANGE
    ref, _ = oracle.cost_matrix(far, np.zeros((0, 6)))
    assert np.array_equal(C3.cpu().numpy(), ref)           # clamped identically
    with pytest.raises(dpso.DpsoError):
        dpso.dpso_cost_matrix(xyz, dpso.MAX_N + 1, None, 0, cp, C)


# -------------------------------------------------------------------- fitness

@pytest.mark.parametrize("n", [3, 31, 32, 33, 255, 256, 257, 400, 513, 1992])
def test_fitness_bitwise(n):
    C_np = inputs.random_cost_matrix(n, n, hi=dpso.COST_MAX)
    tours = inputs.random_tours(n, 37, n + 1)
    C = torch.from_numpy(C_np).to(DEV)
    T = torch.from_numpy(tours.view(np.int16)).to(DEV)
    out = torch.empty(37, dtype=torch.int64, device=DEV)
    dpso.dpso_fitness(C, n, T, 37, out)
    got = out.cpu().numpy()
    assert np.array_equal(got, [oracle.fitness(C_np, t) for t in tours])


def test_fitness_skips_labels_outside_the_tour_range():
    # dpso_fitness's contract: an edge with a label outside [0, n) adds nothing
    # (and never indexes C); the others add their cost as usual
    n = 300
    C_np = inputs.random_cost_matrix(n, 11)
    tours = inputs.random_tours(n, 5, 12)
    tours[1, 0] = n
    tours[2, 299] = 65535
    tours[3, 100:140] = n + 7
    tours[4, :] = n
    C = torch.from_numpy(C_np).to(DEV)
    T = torch.from_numpy(tours.view(np.int16)).to(DEV)
    out = torch.empty(5, dtype=torch.int64, device=DEV)
    dpso.dpso_fitness(C, n, T, 5, out)
    want = []
    for t in tours.astype(np.int64):
        nxt = np.roll(t, -1)
        ok = (t < n) & (nxt < n)
        want.append(int(C_np[t[ok], nxt[ok]].astype(np.int64).sum()))
    assert np.array_equal(out.cpu().numpy(), want)
    assert want[0] == oracle.fitness(C_np, tours[0])


def test_gather_probe_reports_a_rate():
    g = dpso.dpso_probe_l2_gather_gbs(8 << 20, 4)
    assert 1.0 < g < 1e6


# ---------------------------------------------------------------------- 2-opt

def _two_opt_case(C_np, tours, max_moves=0):
    n = C_np.shape[0]
    C = torch.from_numpy(C_np).to(DEV)
    T = torch.from_numpy(tours.view(np.int16).copy()).to(DEV)
    cost = torch.empty(len(tours), dtype=torch.int64, device=DEV)
    pairs, moves = dpso.dpso_two_opt(C, n, T, len(tours), cost, max_moves)
    got_t = T.cpu().numpy().view(np.uint16)
    got_c = cost.cpu().numpy()
    tot_p = tot_m = 0
    for k, x in enumerate(tours):
        y, f, mv, pr = oracle.two_opt(C_np, x, max_moves)
        assert np.array_equal(got_t[k], y), (n, k)
        assert got_c[k] == f, (n, k)
        tot_p += pr
        tot_m += mv
    assert (pairs, moves) == (tot_p, tot_m)


@pytest.mark.parametrize("n,count", [(3, 4), (4, 5), (5, 9), (6, 3), (33, 20), (34, 7),
                                     (35, 6), (64, 16), (65, 16), (100, 40), (257, 6), (400, 4),
                                     (600, 2), (820, 2)])
def test_two_opt_to_convergence_bitwise(n, count):
    C_np = inputs.random_cost_matrix(n, 7 * n)
    _two_opt_case(C_np, inputs.random_tours(n, count, 3 * n))


def test_two_opt_grid_ties_bitwise():
    # integer grid costs have many equal deltas: exercises the (delta, i, j) tie order
    inst = inputs.planar_grid(144, 1.0, np.zeros((0, 6)), "g144", 1, 1, 1)
    C_np, _ = oracle.cost_matrix(inst.xyz, inst.boxes)
    _two_opt_case(C_np, inputs.random_tours(144, 12, 5))


@pytest.mark.parametrize("n,moves", [(1500, 12), (1700, 8), (2300, 6), (3500, 4), (6600, 2),
                                     (8192, 1)])
def test_two_opt_large_tiles_capped_bitwise(n, moves):
    # tiled kernel with 32 / 24 / 16 / 8-row tiles, then the general kernel
    # (6600, 8192); capped move counts keep the oracle fast while still
    # checking each pass exactly
    C_np = inputs.random_cost_matrix(n, n, hi=1_000_000)
    _two_opt_case(C_np, inputs.random_tours(n, 3, n), max_moves=moves)


def test_two_opt_long_tours_two_per_cta_bitwise():
    # 1904 <= n <= 2049 with at least two tours per SM takes 8-row tiles, one
    # tour per CTA and four lane groups per warp by default; capped moves keep
    # the oracle to a few passes per tour
    n, count = 1992, 320
    C_np = inputs.random_cost_matrix(n, 19, hi=1_000_000)
    _two_opt_case(C_np, inputs.random_tours(n, count, 20), max_moves=2)


@pytest.mark.parametrize("n", [37, 101, 403])
def test_two_opt_extreme_costs_bitwise(n):
    # entries at the top of the allowed range: the padding columns past n must
    # neither wrap nor look improving
    rng = np.random.default_rng(n)
    top = rng.integers(dpso.COST_MAX - 3, dpso.COST_MAX + 1, size=(n, n))
    top = np.triu(top, 1)
    C_np = np.ascontiguousarray((top + top.T).astype(np.int32))
    _two_opt_case(C_np, inputs.random_tours(n, 5, n + 7))
    _two_opt_case(inputs.random_cost_matrix(n, n + 9, hi=dpso.COST_MAX),
                  inputs.random_tours(n, 5, n + 8))


def test_two_opt_already_optimal_and_max_moves():
    n = 50
    C_np = inputs.random_cost_matrix(n, 11)
    x = inputs.random_tours(n, 2, 12)
    y0, _, _, _ = oracle.two_opt(C_np, x[0])
    _two_opt_case(C_np, np.stack([y0, x[1]]))
    _two_opt_case(C_np, x, max_moves=1)
    _two_opt_case(C_np, x, max_moves=3)


def test_two_opt_rejects_bad_input():
    n = 20
    C_np = inputs.random_cost_matrix(n, 2)
    C = torch.from_numpy(C_np).to(DEV)
    cost = torch.empty(1, dtype=torch.int64, device=DEV)
    bad = inputs.random_tours(n, 1, 3)
    bad[0, 4] = bad[0, 5]
    T = torch.from_numpy(bad.view(np.int16)).to(DEV)
    with pytest.raises(dpso.DpsoError) as e:
        dpso.dpso_two_opt(C, n, T, 1, cost)
    assert e.value.status == dpso.ERR_ARG
    asym = C_np.copy()
    asym[1, 2] += 1
    good = torch.from_numpy(inputs.random_tours(n, 1, 4).view(np.int16)).to(DEV)
    with pytest.raises(dpso.DpsoError) as e:
        dpso.dpso_two_opt(torch.from_numpy(asym).to(DEV), n, good, 1, cost)
    assert e.value.status == dpso.ERR_ARG
