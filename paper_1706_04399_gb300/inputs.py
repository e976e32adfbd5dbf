"""Seeded synthetic inputs for the inspection-path DPSO.

The paper's office-floor and bridge laser scans (Sec. 4) are not available, so
these generators build viewpoint sets of the same kind: grids of camera
positions on working planes at a stand-off from planar surfaces (Sec. 2.1),
tagged with (face, row, col) so that the deterministic back-and-forth
initialisation (Sec. 3.2.1) can be formed, plus axis-aligned box obstacles
(Sec. 2.2-2.3).

This module holds no arithmetic of the method itself: it only draws numbers.
Both the CPU oracle and the CUDA path consume exactly the arrays it returns.
Every generator is driven by ``numpy.random.default_rng(gen_seed)``.

Array conventions (shared with the C ABI):
  xyz   float64 [N, 3]  viewpoint positions in metres
  tags  int32   [N, 3]  (face, row, col) grid tags, unique per viewpoint
  boxes float64 [M, 6]  (lo_x, lo_y, lo_z, hi_x, hi_y, hi_z) in metres
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


@dataclasses.dataclass
class Instance:
    """One planning problem: viewpoints, their grid tags and obstacles."""

    name: str
    xyz: np.ndarray
    tags: np.ndarray
    boxes: np.ndarray
    swarm: int
    iterations: int
    seed: int

    @property
    def n(self) -> int:
        return int(self.xyz.shape[0])

    @property
    def m(self) -> int:
        return int(self.boxes.shape[0])


def _pack(name, pts, tags, boxes, swarm, iterations, seed) -> Instance:
    xyz = np.ascontiguousarray(np.asarray(pts, dtype=np.float64).reshape(-1, 3))
    tg = np.ascontiguousarray(np.asarray(tags, dtype=np.int32).reshape(-1, 3))
    bx = np.ascontiguousarray(np.asarray(boxes, dtype=np.float64).reshape(-1, 6))
    return Instance(name, xyz, tg, bx, int(swarm), int(iterations), int(seed))


def _random_boxes(rng, count, lo, hi, side_lo=1.0, side_hi=4.0):
    """Boxes with centres uniform in [lo, hi] and sides uniform in [side_lo, side_hi]."""
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    out = np.zeros((count, 6), dtype=np.float64)
    for b in range(count):
        c = rng.uniform(lo, hi)
        s = rng.uniform(side_lo, side_hi, size=3)
        out[b, :3] = c - s / 2
        out[b, 3:] = c + s / 2
    return out


def tiny() -> Instance:
    """6x5 planar grid at integer points, 1.0 m spacing, z=0, one box.

    The box is dyadic so the blocked set is exact: it cuts the unit edges
    (2,2)-(3,2) and (2,3)-(3,3) but a 30-edge Hamiltonian cycle of unit edges
    avoids it, so the optimum tour costs 30 000 mm.
    """
    pts, tags = [], []
    for y in range(5):
        for x in range(6):
            pts.append((float(x), float(y), 0.0))
            tags.append((0, y, x))
    boxes = [(2.25, 1.25, -0.5, 2.75, 3.75, 0.5)]
    return _pack("tiny", pts, tags, boxes, swarm=32, iterations=200, seed=1)


def facade(gen_seed: int = 2) -> Instance:
    """Office-facade-shaped set: 20x20 cells over a 40 m x 30 m wall.

    Wall plane y=0, cells of 2.0 m (x) by 1.5 m (z); viewpoints 3 m out at
    y=-3 over the cell centres, jittered by U[-0.2, 0.2] m on each axis;
    5 boxes with sides U[1,4] m and centres uniform over the viewpoints'
    bounding box grown by 1 m.
    """
    rng = np.random.default_rng(gen_seed)
    pts, tags = [], []
    for r in range(20):
        for c in range(20):
            pts.append((1.0 + 2.0 * c, -3.0, 0.75 + 1.5 * r))
            tags.append((0, r, c))
    pts = np.asarray(pts) + rng.uniform(-0.2, 0.2, size=(400, 3))
    lo = pts.min(axis=0) - 1.0
    hi = pts.max(axis=0) + 1.0
    boxes = _random_boxes(rng, 5, lo, hi)
    return _pack("facade", pts, tags, boxes, swarm=1024, iterations=1000, seed=2)


def bridge(gen_seed: int = 3) -> Instance:
    """Bridge-shaped set: 7 planar faces at 1 m cells with 2 m stand-off.

    Deck underside 100x12 m at z=12 (viewpoints at z=10, 1200 points); two
    deck sides 100x3 m at y=0 and y=12 (deck z in [12,15]; viewpoints at y=-2
    and y=14, 300 points each); four pier faces 4 m (y in [4,8]) x 12 m
    (z in [0,12]) at x = 32.5, 33.5, 66.5, 67.5 (two 1 m thick piers),
    viewpoints 2 m out (48 points each).  N = 1992.  Obstacles: the deck slab,
    the two pier bodies and 17 random clutter boxes near the structure.
    """
    rng = np.random.default_rng(gen_seed)
    pts, tags = [], []
    for j in range(12):
        for i in range(100):
            pts.append((0.5 + i, 0.5 + j, 10.0))
            tags.append((0, j, i))
    for face, yv in ((1, -2.0), (2, 14.0)):
        for k in range(3):
            for i in range(100):
                pts.append((0.5 + i, yv, 12.5 + k))
                tags.append((face, k, i))
    for face, xv in ((3, 30.5), (4, 35.5), (5, 64.5), (6, 69.5)):
        for k in range(12):
            for j in range(4):
                pts.append((xv, 4.5 + j, 0.5 + k))
                tags.append((face, k, j))
    boxes = [
        (0.0, 0.0, 12.0, 100.0, 12.0, 15.0),
        (32.5, 4.0, 0.0, 33.5, 8.0, 12.0),
        (66.5, 4.0, 0.0, 67.5, 8.0, 12.0),
    ]
    clutter = _random_boxes(rng, 17, (0.0, -4.0, 0.0), (100.0, 16.0, 10.0))
    boxes = np.concatenate([np.asarray(boxes), clutter], axis=0)
    return _pack("bridge", pts, tags, boxes, swarm=4096, iterations=2000, seed=3)


def planar_grid(n: int, spacing: float, boxes: np.ndarray, name: str,
                swarm: int, iterations: int, seed: int) -> Instance:
    """First n cells, row-major, of a floor(sqrt(n)) x ceil(n/rows) grid at z=0."""
    rows = max(1, int(math.isqrt(n)))
    cols = -(-n // rows)
    pts, tags = [], []
    for k in range(n):
        r, c = divmod(k, cols)
        pts.append((c * spacing, r * spacing, 0.0))
        tags.append((0, r, c))
    return _pack(name, pts, tags, boxes, swarm, iterations, seed)


def batched(gen_seed: int = 4, count: int = 256) -> list[Instance]:
    """Independent instances: N log-uniform in [50,1500], swarm in [256,2048]."""
    rng = np.random.default_rng(gen_seed)
    out = []
    for i in range(count):
        n = int(round(math.exp(rng.uniform(math.log(50), math.log(1500)))))
        spacing = float(rng.uniform(0.5, 2.0))
        rows = max(1, int(math.isqrt(n)))
        cols = -(-n // rows)
        nb = int(rng.integers(0, 11))
        ext = np.array([cols * spacing, rows * spacing, 0.0])
        bx = _random_boxes(rng, nb, (0.0, 0.0, -0.5), ext + np.array([0, 0, 0.5]),
                           side_lo=0.5 * spacing, side_hi=2.0 * spacing)
        s = int(round(math.exp(rng.uniform(math.log(256), math.log(2048)))))
        out.append(planar_grid(n, spacing, bx, f"batched{i}", s, 500, 1000 + i))
    return out


def serving(gen_seed: int = 5, count: int = 2000, rate_hz: float = 200.0):
    """Poisson stream of re-planning requests: (arrival_s, Instance) pairs."""
    rng = np.random.default_rng(gen_seed)
    t = 0.0
    out = []
    for rid in range(count):
        t += float(rng.exponential(1.0 / rate_hz))
        n = int(round(math.exp(rng.uniform(math.log(50), math.log(3000)))))
        spacing = float(rng.uniform(0.5, 2.0))
        rows = max(1, int(math.isqrt(n)))
        cols = -(-n // rows)
        nb = int(rng.integers(0, 21))
        ext = np.array([cols * spacing, rows * spacing, 0.0])
        bx = _random_boxes(rng, nb, (0.0, 0.0, -0.5), ext + np.array([0, 0, 0.5]),
                           side_lo=0.5 * spacing, side_hi=2.0 * spacing)
        out.append((t, planar_grid(n, spacing, bx, f"req{rid}", 512, 300, rid)))
    return out


def random_instance(n: int, m: int, gen_seed: int, extent: float = 20.0,
                    swarm: int = 32, iterations: int = 20, seed: int = 7) -> Instance:
    """Uniform random viewpoints in a cube with random boxes; tags on a pseudo-grid."""
    rng = np.random.default_rng(gen_seed)
    pts = rng.uniform(0.0, extent, size=(n, 3))
    side = max(1, int(math.isqrt(n)))
    tags = [(0, k // side, k % side) for k in range(n)]
    boxes = _random_boxes(rng, m, (0.0, 0.0, 0.0), (extent, extent, extent))
    return _pack(f"random{n}", pts, tags, boxes, swarm, iterations, seed)


def random_tours(n: int, count: int, gen_seed: int) -> np.ndarray:
    """`count` uniformly random permutations of 0..n-1 as uint16 [count, n]."""
    rng = np.random.default_rng(gen_seed)
    return np.stack([rng.permutation(n) for _ in range(count)]).astype(np.uint16)


def random_cost_matrix(n: int, gen_seed: int, hi: int = 100000) -> np.ndarray:
    """Symmetric int32 matrix with zero diagonal and entries in [1, hi]."""
    rng = np.random.default_rng(gen_seed)
    a = rng.integers(1, hi + 1, size=(n, n), dtype=np.int64)
    c = np.triu(a, 1)
    c = c + c.T
    return np.ascontiguousarray(c.astype(np.int32))


def voxel_grid(inst: Instance, voxel_m: float, margin: int = 2):
    """A voxel grid spec covering the viewpoints and boxes with `margin` voxels
    to spare: (origin (3,), dims (3,)) with the origin on multiples of voxel_m."""
    pts = [inst.xyz]
    if inst.m:
        pts += [inst.boxes[:, :3], inst.boxes[:, 3:]]
    allp = np.concatenate(pts)
    lo = np.floor(allp.min(axis=0) / voxel_m) * voxel_m - margin * voxel_m
    hi = allp.max(axis=0) + margin * voxel_m
    dims = np.ceil((hi - lo) / voxel_m).astype(np.int32) + 1
    return lo.astype(np.float64), dims


def inflate_r2(radius_m: float, voxel_m: float) -> int:
    """The UAV sphere as an integer squared radius in voxel units."""
    return int(math.floor((radius_m / voxel_m) ** 2 + 1e-9))


CONFIGS = {"tiny": tiny, "facade": facade, "bridge": bridge}
