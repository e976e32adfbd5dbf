"""ctypes binding of the C ABI in include/dpso.h (argument marshalling only).

Every function keeps the C name.  Device buffers may be passed as torch CUDA
tensors (their data_ptr() is used), raw integer device addresses, or None.
Host buffers are numpy arrays.  Non-zero status codes raise DpsoError.
The library is loaded on first use; a missing library raises immediately.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

OK = 0
ERR_ARG = -1
ERR_RANGE = -2
ERR_NO_MEMORY = -3
ERR_CUDA = -4
ERR_TIMEOUT = -5
ERR_INTERNAL = -6

MAX_N = 8192
MAX_SWARM = 65535
COST_MAX = 1 << 29

FLAG_DET_INIT = 1
FLAG_MUTATION = 2
FLAG_TWO_OPT = 4
FLAG_NODE_SWAP = 8   # with FLAG_TWO_OPT: the exchange swaps nodes instead of edges
FLAGS_ALL = FLAG_DET_INIT | FLAG_MUTATION | FLAG_TWO_OPT
NODE_SWAP_COST_MAX = 1 << 28


class DpsoError(RuntimeError):
    def __init__(self, status: int, where: str):
        super().__init__(f"{where}: {status_string(status)} ({status})")
        self.status = status


class dpso_params(ctypes.Structure):
    _fields_ = [("w", ctypes.c_double), ("phi1", ctypes.c_double), ("phi2", ctypes.c_double),
                ("swarm", ctypes.c_int32), ("mut_period", ctypes.c_int32),
                ("mut_swaps", ctypes.c_int32), ("det_frac_pct", ctypes.c_int32),
                ("stall_limit", ctypes.c_int32), ("flags", ctypes.c_int32),
                ("two_opt_trigger", ctypes.c_int32), ("max_moves", ctypes.c_int32)]


class dpso_cost_params(ctypes.Structure):
    _fields_ = [("uav_radius_m", ctypes.c_double), ("blocked_penalty_mm", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class dpso_stats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int32), ("stalled", ctypes.c_int32),
                ("gbest_cost", ctypes.c_int64), ("two_opt_pairs", ctypes.c_int64),
                ("two_opt_moves", ctypes.c_int64), ("two_opt_runs", ctypes.c_int64),
                ("device_status", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("two_opt_evaluated", ctypes.c_int64)]


PHASES = ("move", "mutation", "gbest", "two_opt")


class dpso_timing(ctypes.Structure):
    _fields_ = [("ms", ctypes.c_double * 4), ("launches", ctypes.c_int64 * 4),
                ("generations", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class dpso_two_opt_shape(ctypes.Structure):
    _fields_ = [("rows", ctypes.c_int32), ("tours_per_cta", ctypes.c_int32),
                ("tiles_in_flight", ctypes.c_int32)]


SERVE_ARRIVAL_ORDER = 0
SERVE_SHORTEST_FIRST = 1


class dpso_astar_params(ctypes.Structure):
    _fields_ = [("origin", ctypes.c_double * 3), ("voxel_m", ctypes.c_double),
                ("dims", ctypes.c_int32 * 3), ("inflate_r2", ctypes.c_int32),
                ("weights", ctypes.c_int32 * 3), ("unit_mm", ctypes.c_int32),
                ("blocked_cost", ctypes.c_int32), ("max_expansions", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class dpso_server_params(ctypes.Structure):
    _fields_ = [("memory_budget_bytes", ctypes.c_uint64), ("max_active", ctypes.c_int32),
                ("generations_per_tick", ctypes.c_int32), ("policy", ctypes.c_int32),
                ("lanes", ctypes.c_int32)]


class dpso_request(ctypes.Structure):
    _fields_ = [("xyz_host", ctypes.c_void_p), ("boxes_host", ctypes.c_void_p),
                ("tags_host", ctypes.c_void_p), ("n", ctypes.c_int32), ("m", ctypes.c_int32),
                ("iterations", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("seed", ctypes.c_uint64), ("cost", dpso_cost_params), ("params", dpso_params)]


class dpso_server_stats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64),
                ("failed", ctypes.c_int64), ("ticks", ctypes.c_int64),
                ("particle_iterations", ctypes.c_int64), ("memory_used_bytes", ctypes.c_uint64),
                ("peak_active", ctypes.c_int32), ("queued", ctypes.c_int32),
                ("elapsed_s", ctypes.c_double)]


_lib = None
_vp = ctypes.c_void_p
_i32 = ctypes.c_int32
_i64p = ctypes.POINTER(ctypes.c_int64)
_i32p = ctypes.POINTER(ctypes.c_int32)


def library_path() -> str:
    return _build.LIB


def lib():
    """Loads libdpso_gb300.so; raises if it has not been built."""
    global _lib
    if _lib is None:
        path = library_path()
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: build it with paper_1706_04399_gb300.build")
        L = ctypes.CDLL(path)
        sig = {
            "dpso_default_params": (None, [ctypes.POINTER(dpso_params)]),
            "dpso_default_cost_params": (None, [ctypes.POINTER(dpso_cost_params)]),
            "dpso_status_string": (ctypes.c_char_p, [ctypes.c_int]),
            "dpso_cost_matrix": (ctypes.c_int, [_vp, _i32, _vp, _i32,
                                                ctypes.POINTER(dpso_cost_params), _vp, _vp]),
            "dpso_fitness": (ctypes.c_int, [_vp, _i32, _vp, _i32, _vp, _vp]),
            "dpso_two_opt_default_shape": (ctypes.c_int, [_i32, _i32, _i32,
                                                          ctypes.POINTER(dpso_two_opt_shape)]),
            "dpso_probe_l2_gather_gbs": (ctypes.c_int, [ctypes.c_size_t, _i32,
                                                        ctypes.POINTER(ctypes.c_double), _vp]),
            "dpso_two_opt": (ctypes.c_int, [_vp, _i32, _vp, _i32, _vp, _i32, _i64p, _i64p, _vp]),
            "dpso_default_astar_params": (None, [ctypes.POINTER(dpso_astar_params)]),
            "dpso_voxel_occupancy": (ctypes.c_int, [_vp, _i32, ctypes.POINTER(dpso_astar_params),
                                                    _vp, _vp]),
            "dpso_cost_matrix_astar": (ctypes.c_int, [_vp, _i32, _vp,
                                                      ctypes.POINTER(dpso_astar_params), _vp,
                                                      _vp]),
            "dpso_node_swap": (ctypes.c_int, [_vp, _i32, _vp, _i32, _vp, _i32, _i64p, _i64p, _vp]),
            "dpso_two_opt_noalloc": (ctypes.c_int, [_vp, _i32, _vp, _i32, _vp, _i32, _i64p, _i64p,
                                                    _vp]),
            "dpso_init": (ctypes.c_int, [ctypes.POINTER(_vp), _vp, _i32, _vp,
                                         ctypes.POINTER(dpso_params), ctypes.c_uint64, _vp]),
            "dpso_step": (ctypes.c_int, [_vp, _i32, _vp]),
            "dpso_get_best": (ctypes.c_int, [_vp, _i32p, _i64p]),
            "dpso_get_history": (ctypes.c_int, [_vp, _i64p, _i32, _i32p]),
            "dpso_get_stats": (ctypes.c_int, [_vp, ctypes.POINTER(dpso_stats)]),
            "dpso_set_timing": (ctypes.c_int, [_vp, ctypes.c_int]),
            "dpso_get_timing": (ctypes.c_int, [_vp, ctypes.POINTER(dpso_timing)]),
            "dpso_get_state": (ctypes.c_int, [_vp, _vp, ctypes.POINTER(ctypes.c_size_t)]),
            "dpso_set_state": (ctypes.c_int, [_vp, _vp, ctypes.c_size_t]),
            "dpso_destroy": (None, [_vp]),
            "dpso_plan": (ctypes.c_int, [_vp, _i32, _vp, _i32, _vp,
                                         ctypes.POINTER(dpso_cost_params),
                                         ctypes.POINTER(dpso_params), ctypes.c_uint64, _i32,
                                         _i32p, _i64p]),
            "dpso_batch_create": (ctypes.c_int, [ctypes.POINTER(_vp), ctypes.POINTER(_vp), _i32,
                                                 _vp]),
            "dpso_batch_step": (ctypes.c_int, [_vp, _i32, _vp]),
            "dpso_batch_autotune": (ctypes.c_int, [_vp, ctypes.POINTER(dpso_two_opt_shape), _vp]),
            "dpso_batch_set_two_opt_shape": (ctypes.c_int, [_vp,
                                                            ctypes.POINTER(dpso_two_opt_shape)]),
            "dpso_batch_destroy": (None, [_vp]),
            "dpso_probe_l2_read_gbs": (ctypes.c_int, [ctypes.c_size_t, _i32,
                                                      ctypes.POINTER(ctypes.c_double), _vp]),
            "dpso_default_server_params": (None, [ctypes.POINTER(dpso_server_params)]),
            "dpso_server_create": (ctypes.c_int, [ctypes.POINTER(_vp),
                                                  ctypes.POINTER(dpso_server_params)]),
            "dpso_server_submit": (ctypes.c_int, [_vp, ctypes.POINTER(dpso_request), _i64p]),
            "dpso_server_footprint": (ctypes.c_int, [ctypes.POINTER(dpso_request),
                                                     ctypes.POINTER(ctypes.c_uint64)]),
            "dpso_server_poll": (ctypes.c_int, [_vp, ctypes.c_int64, _i32p, _i32p, _i32, _i64p,
                                                ctypes.POINTER(ctypes.c_double)]),
            "dpso_server_wait": (ctypes.c_int, [_vp, ctypes.c_int64, ctypes.c_double, _i32p]),
            "dpso_server_stats_get": (ctypes.c_int, [_vp, ctypes.POINTER(dpso_server_stats)]),
            "dpso_server_destroy": (None, [_vp]),
            "dpso_philox_draws": (ctypes.c_int, [ctypes.c_uint64, ctypes.c_uint32,
                                                 ctypes.c_uint32, ctypes.c_uint32, _i32, _vp, _vp]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _dev(t):
    """Device address of a torch tensor, an int address, or None."""
    if t is None:
        return None
    if isinstance(t, int):
        return t
    return t.data_ptr()


def _stream(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _check(status: int, where: str):
    if status != OK:
        raise DpsoError(status, where)


def status_string(status: int) -> str:
    return lib().dpso_status_string(status).decode()


def default_params(**overrides) -> dpso_params:
    p = dpso_params()
    lib().dpso_default_params(ctypes.byref(p))
    for k, v in overrides.items():
        setattr(p, k, v)
    return p


def default_cost_params(**overrides) -> dpso_cost_params:
    p = dpso_cost_params()
    lib().dpso_default_cost_params(ctypes.byref(p))
    for k, v in overrides.items():
        setattr(p, k, v)
    return p


# ---------------------------------------------------------------- entry points

def dpso_cost_matrix(xyz_dev, n: int, boxes_dev, m: int, cp: dpso_cost_params, C_dev,
                     stream=None) -> None:
    _check(lib().dpso_cost_matrix(_dev(xyz_dev), n, _dev(boxes_dev), m, ctypes.byref(cp),
                                  _dev(C_dev), _stream(stream)), "dpso_cost_matrix")


def dpso_fitness(C_dev, n: int, tours_dev, count: int, cost_dev, stream=None) -> None:
    _check(lib().dpso_fitness(_dev(C_dev), n, _dev(tours_dev), count, _dev(cost_dev),
                              _stream(stream)), "dpso_fitness")


def dpso_two_opt(C_dev, n: int, tours_dev, count: int, cost_dev, max_moves: int = 0,
                 stream=None) -> tuple[int, int]:
    pairs = ctypes.c_int64(0)
    moves = ctypes.c_int64(0)
    _check(lib().dpso_two_opt(_dev(C_dev), n, _dev(tours_dev), count, _dev(cost_dev), max_moves,
                              ctypes.byref(pairs), ctypes.byref(moves), _stream(stream)),
           "dpso_two_opt")
    return pairs.value, moves.value


def dpso_node_swap(C_dev, n: int, tours_dev, count: int, cost_dev, max_moves: int = 0,
                   stream=None) -> tuple[int, int]:
    pairs = ctypes.c_int64(0)
    moves = ctypes.c_int64(0)
    _check(lib().dpso_node_swap(_dev(C_dev), n, _dev(tours_dev), count, _dev(cost_dev), max_moves,
                                ctypes.byref(pairs), ctypes.byref(moves), _stream(stream)),
           "dpso_node_swap")
    return pairs.value, moves.value


def astar_params(origin, voxel_m: float, dims, inflate_r2: int = 0, weights=(1, 1, 1),
                 unit_mm: int = 500, blocked_cost: int = 100_000_000,
                 max_expansions: int = 20000) -> dpso_astar_params:
    p = dpso_astar_params()
    lib().dpso_default_astar_params(ctypes.byref(p))
    p.origin[:] = [float(v) for v in origin]
    p.voxel_m = voxel_m
    p.dims[:] = [int(v) for v in dims]
    p.inflate_r2 = inflate_r2
    p.weights[:] = [int(v) for v in weights]
    p.unit_mm = unit_mm
    p.blocked_cost = blocked_cost
    p.max_expansions = max_expansions
    return p


def dpso_voxel_occupancy(boxes_dev, m: int, ap: dpso_astar_params, occ_dev, stream=None) -> None:
    _check(lib().dpso_voxel_occupancy(_dev(boxes_dev), m, ctypes.byref(ap), _dev(occ_dev),
                                      _stream(stream)), "dpso_voxel_occupancy")


def dpso_cost_matrix_astar(xyz_dev, n: int, occ_dev, ap: dpso_astar_params, C_dev,
                           stream=None) -> None:
    _check(lib().dpso_cost_matrix_astar(_dev(xyz_dev), n, _dev(occ_dev), ctypes.byref(ap),
                                        _dev(C_dev), _stream(stream)), "dpso_cost_matrix_astar")


def dpso_probe_l2_read_gbs(nbytes: int = 24 << 20, reps: int = 40, stream=None) -> float:
    """Measured L2 read bandwidth (GB/s) of the current device."""
    out = ctypes.c_double(0.0)
    _check(lib().dpso_probe_l2_read_gbs(nbytes, reps, ctypes.byref(out), _stream(stream)),
           "dpso_probe_l2_read_gbs")
    return out.value


def dpso_two_opt_default_shape(n: int, count: int, num_sms: int) -> tuple[int, int, int]:
    """(tile rows, tours per CTA, tiles in flight) a launch over `count` tours
    of n viewpoints takes when no shape is pinned; (0, 0, 0): the general kernel."""
    sh = dpso_two_opt_shape()
    _check(lib().dpso_two_opt_default_shape(n, count, num_sms, ctypes.byref(sh)),
           "dpso_two_opt_default_shape")
    return sh.rows, sh.tours_per_cta, sh.tiles_in_flight


def dpso_probe_l2_gather_gbs(nbytes: int = 16 << 20, reps: int = 64, stream=None) -> float:
    """Measured rate (GB/s of 4-byte words) of random gathers from an L2-resident buffer."""
    out = ctypes.c_double(0.0)
    _check(lib().dpso_probe_l2_gather_gbs(nbytes, reps, ctypes.byref(out), _stream(stream)),
           "dpso_probe_l2_gather_gbs")
    return out.value


NOALLOC_MAX_TOURS = 16350


def dpso_two_opt_noalloc(C_dev, n: int, tours_dev, count: int, cost_dev, max_moves: int = 0,
                         stream=None) -> tuple[int, int]:
    """dpso_two_opt whose scratch is a fixed array in the library (no allocation)."""
    pairs = ctypes.c_int64(0)
    moves = ctypes.c_int64(0)
    _check(lib().dpso_two_opt_noalloc(_dev(C_dev), n, _dev(tours_dev), count, _dev(cost_dev),
                                      max_moves, ctypes.byref(pairs), ctypes.byref(moves),
                                      _stream(stream)), "dpso_two_opt_noalloc")
    return pairs.value, moves.value


def dpso_philox_draws(seed: int, phase: int, iteration: int, particle: int, count: int, out_dev,
                      stream=None) -> None:
    _check(lib().dpso_philox_draws(seed, phase, iteration, particle, count, _dev(out_dev),
                                   _stream(stream)), "dpso_philox_draws")


def dpso_plan(xyz: np.ndarray, boxes: np.ndarray, tags, cp: dpso_cost_params,
              p: dpso_params, seed: int, iterations: int):
    xyz = np.ascontiguousarray(xyz, dtype=np.float64)
    boxes = np.ascontiguousarray(boxes, dtype=np.float64).reshape(-1, 6)
    n, m = xyz.shape[0], boxes.shape[0]
    tg = None if tags is None else np.ascontiguousarray(tags, dtype=np.int32)
    tour = np.zeros(n, np.int32)
    cost = ctypes.c_int64(0)
    _check(lib().dpso_plan(xyz.ctypes.data, n, boxes.ctypes.data if m else None, m,
                           None if tg is None else tg.ctypes.data, ctypes.byref(cp),
                           ctypes.byref(p), seed, iterations,
                           tour.ctypes.data_as(_i32p), ctypes.byref(cost)), "dpso_plan")
    return tour, cost.value


class Swarm:
    """Owns a dpso_swarm handle: dpso_init / dpso_step / dpso_get_* / dpso_destroy."""

    def __init__(self, C_dev, n: int, tags, p: dpso_params, seed: int, stream=None):
        self.n = n
        self.p = p
        h = _vp()
        tg = None if tags is None else np.ascontiguousarray(tags, dtype=np.int32)
        _check(lib().dpso_init(ctypes.byref(h), _dev(C_dev), n,
                               None if tg is None else tg.ctypes.data, ctypes.byref(p), seed,
                               _stream(stream)), "dpso_init")
        self._h = h

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            lib().dpso_destroy(self._h)
            self._h = _vp()

    __del__ = close

    def step(self, iterations: int, stream=None):
        _check(lib().dpso_step(self._h, iterations, _stream(stream)), "dpso_step")

    def best(self):
        tour = np.zeros(self.n, np.int32)
        cost = ctypes.c_int64(0)
        _check(lib().dpso_get_best(self._h, tour.ctypes.data_as(_i32p), ctypes.byref(cost)),
               "dpso_get_best")
        return tour, cost.value

    def history(self) -> np.ndarray:
        ln = ctypes.c_int32(0)
        _check(lib().dpso_get_history(self._h, None, 0, ctypes.byref(ln)), "dpso_get_history")
        out = np.zeros(max(ln.value, 1), np.int64)
        _check(lib().dpso_get_history(self._h, out.ctypes.data_as(_i64p), ln.value,
                                      ctypes.byref(ln)), "dpso_get_history")
        return out[:ln.value]

    def stats(self) -> dict:
        st = dpso_stats()
        _check(lib().dpso_get_stats(self._h, ctypes.byref(st)), "dpso_get_stats")
        return {k: getattr(st, k) for k, _ in dpso_stats._fields_ if k != "reserved"}

    def set_timing(self, on: bool):
        _check(lib().dpso_set_timing(self._h, 1 if on else 0), "dpso_set_timing")

    def timing(self) -> dict:
        t = dpso_timing()
        _check(lib().dpso_get_timing(self._h, ctypes.byref(t)), "dpso_get_timing")
        return {"ms": dict(zip(PHASES, list(t.ms))),
                "launches": dict(zip(PHASES, list(t.launches))),
                "generations": t.generations}

    def state_bytes(self) -> bytes:
        nb = ctypes.c_size_t(0)
        _check(lib().dpso_get_state(self._h, None, ctypes.byref(nb)), "dpso_get_state")
        buf = ctypes.create_string_buffer(nb.value)
        _check(lib().dpso_get_state(self._h, buf, ctypes.byref(nb)), "dpso_get_state")
        return buf.raw[:nb.value]

    def set_state_bytes(self, blob: bytes):
        buf = ctypes.create_string_buffer(blob, len(blob))
        _check(lib().dpso_set_state(self._h, buf, len(blob)), "dpso_set_state")

    def state(self) -> dict:
        """Decoded checkpoint: X, V, P (S x n), G, F, PF, history, counters."""
        blob = self.state_bytes()
        hdr = np.frombuffer(blob, dtype=np.uint8, count=_HDR_SIZE)
        magic, version, n, S, t, stall, done, n_det = np.frombuffer(hdr, np.int32, 8, 0)
        gf, pairs, moves, runs = np.frombuffer(hdr, np.int64, 4, 32)
        off = _HDR_SIZE
        out = {"n": int(n), "S": int(S), "t": int(t), "stall": int(stall), "done": bool(done),
               "n_det": int(n_det), "gf": int(gf), "pairs": int(pairs), "moves": int(moves),
               "runs": int(runs)}
        for name in ("X", "V", "P"):
            out[name] = np.frombuffer(blob, np.uint16, S * n, off).reshape(S, n).copy()
            off += 2 * S * n
        out["G"] = np.frombuffer(blob, np.uint16, n, off).copy()
        off += 2 * n
        out["F"] = np.frombuffer(blob, np.int64, S, off).copy()
        off += 8 * S
        out["PF"] = np.frombuffer(blob, np.int64, S, off).copy()
        off += 8 * S
        out["history"] = np.frombuffer(blob, np.int64, t, off).copy()
        return out


# StateHeader: 2 uint32 + 6 int32 + int64 + 3 uint64 + uint64 seed + dpso_params
_HDR_SIZE = 8 + 24 + 8 + 24 + 8 + ctypes.sizeof(dpso_params)


class Batch:
    """Owns a dpso_batch over existing Swarm objects (kept alive by the batch)."""

    def __init__(self, swarms, stream=None):
        self.swarms = list(swarms)
        arr = (_vp * len(self.swarms))(*[sw._h.value for sw in self.swarms])
        h = _vp()
        _check(lib().dpso_batch_create(ctypes.byref(h), arr, len(self.swarms), _stream(stream)),
               "dpso_batch_create")
        self._h = h

    def step(self, iterations: int, stream=None):
        _check(lib().dpso_batch_step(self._h, iterations, _stream(stream)), "dpso_batch_step")

    def autotune(self, stream=None) -> tuple[int, int, int]:
        """Chosen 2-opt launch shape: (tile height, tours per CTA, tiles in flight)."""
        sh = dpso_two_opt_shape()
        _check(lib().dpso_batch_autotune(self._h, ctypes.byref(sh), _stream(stream)),
               "dpso_batch_autotune")
        return sh.rows, sh.tours_per_cta, sh.tiles_in_flight

    def set_two_opt_shape(self, rows: int, tpc: int, tiles_in_flight: int = 1):
        sh = dpso_two_opt_shape(rows, tpc, tiles_in_flight)
        _check(lib().dpso_batch_set_two_opt_shape(self._h, ctypes.byref(sh)),
               "dpso_batch_set_two_opt_shape")

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            lib().dpso_batch_destroy(self._h)
            self._h = _vp()

    __del__ = close


def default_server_params(**overrides) -> dpso_server_params:
    p = dpso_server_params()
    lib().dpso_default_server_params(ctypes.byref(p))
    for k, v in overrides.items():
        setattr(p, k, v)
    return p


def make_request(xyz: np.ndarray, boxes: np.ndarray, tags, cp: dpso_cost_params,
                 p: dpso_params, seed: int, iterations: int):
    """A dpso_request and the contiguous arrays it points into (keep them alive)."""
    xyz = np.ascontiguousarray(xyz, dtype=np.float64)
    boxes = np.ascontiguousarray(boxes, dtype=np.float64).reshape(-1, 6)
    tg = None if tags is None else np.ascontiguousarray(tags, dtype=np.int32)
    r = dpso_request()
    r.xyz_host = xyz.ctypes.data
    r.boxes_host = boxes.ctypes.data if boxes.shape[0] else None
    r.tags_host = None if tg is None else tg.ctypes.data
    r.n, r.m = xyz.shape[0], boxes.shape[0]
    r.iterations = iterations
    r.seed = seed
    r.cost = cp
    r.params = p
    return r, (xyz, boxes, tg)


def dpso_server_footprint(xyz, boxes, tags, cp, p, seed, iterations) -> int:
    r, _keep = make_request(xyz, boxes, tags, cp, p, seed, iterations)
    out = ctypes.c_uint64(0)
    _check(lib().dpso_server_footprint(ctypes.byref(r), ctypes.byref(out)),
           "dpso_server_footprint")
    return out.value


class Server:
    """Owns a dpso_server: submit / poll / wait / stats / close."""

    def __init__(self, params: dpso_server_params | None = None):
        p = params if params is not None else default_server_params()
        h = _vp()
        _check(lib().dpso_server_create(ctypes.byref(h), ctypes.byref(p)), "dpso_server_create")
        self._h = h
        self._n = {}

    def submit(self, xyz: np.ndarray, boxes: np.ndarray, tags, cp: dpso_cost_params,
               p: dpso_params, seed: int, iterations: int) -> int:
        r, keep = make_request(xyz, boxes, tags, cp, p, seed, iterations)
        rid = ctypes.c_int64(0)
        _check(lib().dpso_server_submit(self._h, ctypes.byref(r), ctypes.byref(rid)),
               "dpso_server_submit")
        self._n[rid.value] = keep[0].shape[0]
        return rid.value

    def poll(self, rid: int):
        """(state, tour or None, cost or None, latency_s); state 0 pending, 1 done, < 0 failed."""
        n = self._n.get(rid, 0)
        tour = np.zeros(max(n, 1), np.int32)
        state = ctypes.c_int32(0)
        cost = ctypes.c_int64(0)
        lat = ctypes.c_double(0.0)
        _check(lib().dpso_server_poll(self._h, rid, ctypes.byref(state),
                                      tour.ctypes.data_as(_i32p), n, ctypes.byref(cost),
                                      ctypes.byref(lat)), "dpso_server_poll")
        if state.value == 1:
            return 1, tour, cost.value, lat.value
        return state.value, None, None, lat.value

    def wait(self, rid: int, timeout_s: float = 600.0) -> int:
        state = ctypes.c_int32(0)
        st = lib().dpso_server_wait(self._h, rid, timeout_s, ctypes.byref(state))
        if st not in (OK, ERR_TIMEOUT):
            _check(st, "dpso_server_wait")
        return state.value

    def stats(self) -> dict:
        st = dpso_server_stats()
        _check(lib().dpso_server_stats_get(self._h, ctypes.byref(st)), "dpso_server_stats_get")
        return {k: getattr(st, k) for k, _ in dpso_server_stats._fields_}

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            lib().dpso_server_destroy(self._h)
            self._h = _vp()

    __del__ = close
