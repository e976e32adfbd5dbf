"""A* edge costs on the GPU against the oracle: inflated occupancy and the
cost matrix, bit for bit, including searches that need the second pass,
blocked pairs and expansion caps."""
import numpy as np
import pytest

from gpu_helpers import DEV, torch  # noqa: F401
import oracle
from paper_1706_04399_gb300 import dpso, inputs

pytestmark = pytest.mark.gpu


def _occupancy_gpu(boxes, origin, voxel, dims, r2):
    ap = dpso.astar_params(origin, voxel, dims, inflate_r2=r2)
    occ = torch.empty(int(np.prod(dims)), dtype=torch.uint8, device=DEV)
    b = np.asarray(boxes, np.float64).reshape(-1, 6)
    bd = torch.from_numpy(b).to(DEV) if len(b) else None
    dpso.dpso_voxel_occupancy(bd, len(b), ap, occ)
    return occ


def _astar_both(xyz, boxes, origin, voxel, dims, r2=0, weights=(1, 1, 1), unit_mm=500,
                blocked=10 ** 8, max_exp=20000):
    occ_ref = oracle.voxel_occupancy(origin, voxel, dims, boxes, r2)
    occ = _occupancy_gpu(boxes, origin, voxel, dims, r2)
    assert np.array_equal(occ.cpu().numpy().reshape(occ_ref.shape), occ_ref)
    want, st = oracle.cost_matrix_astar(xyz, occ_ref, origin, voxel, dims, weights, unit_mm,
                                        blocked, max_exp)
    n = len(xyz)
    ap = dpso.astar_params(origin, voxel, dims, inflate_r2=r2, weights=weights, unit_mm=unit_mm,
                           blocked_cost=blocked, max_expansions=max_exp)
    C = torch.empty((n, n), dtype=torch.int32, device=DEV)
    dpso.dpso_cost_matrix_astar(torch.from_numpy(np.ascontiguousarray(xyz)).to(DEV), n, occ, ap, C)
    got = C.cpu().numpy()
    bad = np.argwhere(got != want)
    assert not len(bad), (bad[:5].tolist(), got[tuple(bad[0])], want[tuple(bad[0])])
    return got


@pytest.mark.parametrize("r2", [0, 1, 2, 4, 9])
def test_occupancy_bitwise(r2):
    inst = inputs.random_instance(10, 6, 11 + r2, extent=8.0)
    origin, dims = inputs.voxel_grid(inst, 0.5)
    occ_ref = oracle.voxel_occupancy(origin, 0.5, dims, inst.boxes, r2)
    occ = _occupancy_gpu(inst.boxes, origin, 0.5, dims, r2)
    assert np.array_equal(occ.cpu().numpy().reshape(occ_ref.shape), occ_ref)
    assert occ_ref.any() and not occ_ref.all()


@pytest.mark.parametrize("n,m,weights,r2", [(24, 4, (1, 1, 1), 0), (31, 8, (1, 2, 3), 1),
                                            (40, 10, (2, 2, 1), 2)])
def test_cost_matrix_bitwise(n, m, weights, r2):
    inst = inputs.random_instance(n, m, 70 + n, extent=10.0)
    origin, dims = inputs.voxel_grid(inst, 0.5)
    C = _astar_both(inst.xyz, inst.boxes, origin, 0.5, dims, r2=r2, weights=weights)
    assert (np.diag(C) == 0).all() and np.array_equal(C, C.T)


def test_second_pass_and_caps_bitwise():
    """Walls with narrow gaps force long searches (the second pass); small
    caps turn searches into blocked pairs; a cap below the first pass's room
    finishes in one pass."""
    dims = (40, 30, 3)
    boxes = [(9.0, 0.0, 0.0, 10.0, 27.0, 3.0), (19.0, 3.0, 0.0, 20.0, 30.0, 3.0),
             (29.0, 0.0, 0.0, 30.0, 27.0, 3.0)]
    rng = np.random.default_rng(5)
    xyz = np.column_stack([rng.uniform(0, 40, 18), rng.uniform(0, 30, 18), rng.uniform(0, 3, 18)])
    full = _astar_both(xyz, boxes, (0, 0, 0), 1.0, dims, max_exp=20000, blocked=999)
    capped = _astar_both(xyz, boxes, (0, 0, 0), 1.0, dims, max_exp=300, blocked=999)
    small = _astar_both(xyz, boxes, (0, 0, 0), 1.0, dims, max_exp=40, blocked=999)
    assert (capped == 999).sum() > (full == 999).sum()
    assert (small == 999).sum() >= (capped == 999).sum()


def test_blocked_viewpoints_bitwise():
    dims = (12, 10, 4)
    boxes = [(3.0, 3.0, 0.0, 6.0, 6.0, 4.0)]
    xyz = np.array([[0.5, 0.5, 0.5], [4.5, 4.5, 1.5], [11.5, 9.5, 3.5], [20.0, 1.0, 1.0],
                    [2.5, 8.5, 2.5], [-0.1, 4.0, 1.0]])
    C = _astar_both(xyz, boxes, (0, 0, 0), 1.0, dims, r2=1, blocked=4242)
    assert (C[1, [0, 2, 4]] == 4242).all() and (C[3, [0, 1, 2, 4]] == 4242).all()


def test_facade_grid_bitwise():
    """The facade workload's viewpoints on a 0.5 m grid with its boxes."""
    inst = inputs.facade()
    sub = inst.xyz[::5]  # 80 viewpoints
    origin, dims = inputs.voxel_grid(inst, 0.5)
    r2 = inputs.inflate_r2(0.5, 0.5)
    _astar_both(sub, inst.boxes, origin, 0.5, dims, r2=r2)


def test_astar_rejects_bad_parameters():
    occ = torch.zeros(8, dtype=torch.uint8, device=DEV)
    C = torch.empty((2, 2), dtype=torch.int32, device=DEV)
    xyz = torch.zeros((2, 3), dtype=torch.float64, device=DEV)
    for kw, status in ((dict(voxel_m=0.0), dpso.ERR_ARG), (dict(dims=(5000, 1, 1)), dpso.ERR_RANGE),
                       (dict(max_expansions=10 ** 6), dpso.ERR_RANGE)):
        args = dict(origin=(0, 0, 0), voxel_m=1.0, dims=(2, 2, 2))
        args.update(kw)
        ap = dpso.astar_params(**args)
        with pytest.raises(dpso.DpsoError) as e:
            dpso.dpso_cost_matrix_astar(xyz, 2, occ, ap, C)
        assert e.value.status == status


def test_search_outgrowing_the_warp_pass_bitwise():
    """A wall with one gap at its far end: the search between the two sides
    floods about 1960 voxels, more than the one-warp pass keeps in shared
    memory, so it is searched again by the thread pass; the other pairs stay
    in the warp pass."""
    dims = (64, 64, 1)
    boxes = [(32.0, 0.0, 0.0, 33.0, 62.0, 1.0)]
    xyz = np.array([[10.5, 5.5, 0.5], [50.5, 5.5, 0.5], [5.5, 60.5, 0.5], [60.5, 30.5, 0.5],
                    [20.5, 40.5, 0.5], [40.5, 63.5, 0.5]])
    C = _astar_both(xyz, boxes, (0, 0, 0), 1.0, dims, blocked=999)
    assert C[0, 1] == 77000 and (C != 999).all()


def test_large_weights_take_the_thread_pass_bitwise():
    """Step weights of about 1000 make f too wide for the warp pass's packed
    keys; the thread pass then takes every pair (256 expansions, then the cap)."""
    inst = inputs.random_instance(30, 5, 321, extent=10.0)
    origin, dims = inputs.voxel_grid(inst, 0.5)
    _astar_both(inst.xyz, inst.boxes, origin, 0.5, dims, r2=1, weights=(1000, 999, 998),
                unit_mm=1, blocked=10 ** 8)


def test_bridge_grid_bitwise():
    """Viewpoints of the bridge workload on its 0.5 m grid with its boxes."""
    inst = inputs.bridge()
    sub = inst.xyz[::33]  # 61 viewpoints
    origin, dims = inputs.voxel_grid(inst, 0.5)
    _astar_both(sub, inst.boxes, origin, 0.5, dims, r2=inputs.inflate_r2(0.5, 0.5))


def test_grid_wider_than_256_takes_the_thread_pass_bitwise():
    """A grid dimension above 256 does not fit the warp pass's packed voxel
    coordinates; the thread pass takes every pair."""
    dims = (300, 4, 3)
    boxes = [(100.0, 0.0, 0.0, 101.0, 3.0, 3.0), (200.0, 1.0, 0.0, 201.0, 4.0, 3.0)]
    rng = np.random.default_rng(8)
    xyz = np.column_stack([rng.uniform(0, 300, 12), rng.uniform(0, 4, 12), rng.uniform(0, 3, 12)])
    C = _astar_both(xyz, boxes, (0, 0, 0), 1.0, dims, blocked=777)
    assert (C == 777).sum() < C.size - 12
