"""CPU oracle for the enhanced DPSO (arXiv:1706.04399): ctypes wrapper.

TEST INFRASTRUCTURE ONLY: the plain single-threaded C implementation in
``dpso_oracle.c`` that the CUDA library is checked against.  Only the tests,
``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg may use it.
It shares no code with the CUDA path and imports nothing from it.

See ``dpso_oracle.c`` for the paper passages each function follows and for
which parts are pinned.
"""
from __future__ import annotations

import ctypes
import os
import platform
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dpso_oracle.c")
_LIB = os.path.join(_HERE, "liboracle_dpso.so")
_STAMP = _LIB + ".machine"

DET_INIT = 1
MUTATION = 2
TWO_OPT = 4
NODE_SWAP = 8   # with TWO_OPT: the exchange swaps two nodes instead of two edges
ALL = DET_INIT | MUTATION | TWO_OPT

ERR_ARG = -1
ERR_RANGE = -2


def build(force: bool = False) -> str:
    """Compile the oracle with strict IEEE semantics (no contraction, no fast-math)."""
    try:
        with open(_STAMP) as fh:
            same_machine = fh.read().strip() == platform.machine()
    except OSError:
        same_machine = False
    if (force or not same_machine or not os.path.exists(_LIB)
            or os.path.getmtime(_LIB) < os.path.getmtime(_SRC)):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call([
            "gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math",
            "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
        with open(_STAMP, "w") as fh:
            fh.write(platform.machine() + "\n")
    return _LIB


_lib = None

_u16p = ctypes.POINTER(ctypes.c_uint16)
_i32p = ctypes.POINTER(ctypes.c_int32)
_i64p = ctypes.POINTER(ctypes.c_int64)
_u32p = ctypes.POINTER(ctypes.c_uint32)
_f64p = ctypes.POINTER(ctypes.c_double)
_u8p = ctypes.POINTER(ctypes.c_uint8)


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        L.orc_philox4x32_10.argtypes = [_u32p, _u32p, _u32p]
        L.orc_draw.argtypes = [ctypes.c_uint64] + [ctypes.c_uint32] * 4
        L.orc_draw.restype = ctypes.c_uint32
        L.orc_draws.argtypes = [ctypes.c_uint64] + [ctypes.c_uint32] * 3 + [ctypes.c_int32, _u32p]
        L.orc_segment_blocked.argtypes = [_f64p, _f64p, _f64p, ctypes.c_double]
        L.orc_cost_matrix.argtypes = [_f64p, ctypes.c_int32, _f64p, ctypes.c_int32,
                                      ctypes.c_double, ctypes.c_int32, _i32p]
        L.orc_fitness.argtypes = [_i32p, ctypes.c_int32, _u16p]
        L.orc_fitness.restype = ctypes.c_int64
        L.orc_apply.argtypes = [_u16p, ctypes.c_int32, _u16p, ctypes.c_int64]
        L.orc_subtract.argtypes = [_u16p, _u16p, ctypes.c_int32, _u16p]
        L.orc_subtract.restype = ctypes.c_int64
        L.orc_scaled_count.argtypes = [ctypes.c_double, ctypes.c_uint32, ctypes.c_int64]
        L.orc_scaled_count.restype = ctypes.c_int64
        L.orc_boustrophedon.argtypes = [_i32p, ctypes.c_int32, ctypes.c_int32, _u16p]
        L.orc_two_opt.argtypes = [_i32p, ctypes.c_int32, _u16p, _i64p, ctypes.c_int32, _i64p]
        L.orc_two_opt.restype = ctypes.c_int64
        L.orc_node_swap.argtypes = [_i32p, ctypes.c_int32, _u16p, _i64p, ctypes.c_int32, _i64p]
        L.orc_node_swap.restype = ctypes.c_int64
        L.orc_voxel_occupancy.argtypes = [_f64p, ctypes.c_double, _i32p, _f64p, ctypes.c_int32,
                                          ctypes.c_int32, _u8p]
        L.orc_voxel_occupancy.restype = ctypes.c_int
        L.orc_cost_matrix_astar.argtypes = [_f64p, ctypes.c_int32, _u8p, _f64p, ctypes.c_double,
                                            _i32p, _i32p, ctypes.c_int32, ctypes.c_int32,
                                            ctypes.c_int32, _i32p]
        L.orc_cost_matrix_astar.restype = ctypes.c_int
        L.orc_swarm_new.argtypes = [
            _i32p, ctypes.c_int32, _i32p, ctypes.c_int32, ctypes.c_double, ctypes.c_double,
            ctypes.c_double, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
            ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_uint64, _i32p]
        L.orc_swarm_new.restype = ctypes.c_void_p
        L.orc_swarm_free.argtypes = [ctypes.c_void_p]
        for name in ("orc_swarm_move",):
            getattr(L, name).argtypes = [ctypes.c_void_p, ctypes.c_int32]
        L.orc_swarm_mutate.argtypes = [ctypes.c_void_p, ctypes.c_int32, _i32p]
        L.orc_swarm_gbest.argtypes = [ctypes.c_void_p]
        L.orc_swarm_two_opt.argtypes = [ctypes.c_void_p, _i32p, ctypes.c_int32]
        L.orc_swarm_iterate.argtypes = [ctypes.c_void_p]
        L.orc_swarm_iterate_begin.argtypes = [ctypes.c_void_p, _i32p]
        L.orc_swarm_iterate_end.argtypes = [ctypes.c_void_p]
        L.orc_swarm_two_opt_part.argtypes = [ctypes.c_void_p, _i32p, ctypes.c_int32, _i64p]
        L.orc_swarm_add_counters.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64]
        L.orc_swarm_import.argtypes = [ctypes.c_void_p, _u16p, _u16p, _u16p, _i64p, _i64p, _u16p,
                                       ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
                                       ctypes.c_int32, _i64p, _i64p]
        L.orc_swarm_run.argtypes = [ctypes.c_void_p, ctypes.c_int32]
        for name in ("orc_swarm_n", "orc_swarm_size", "orc_swarm_t", "orc_swarm_done",
                     "orc_swarm_stall", "orc_swarm_last_two_opt", "orc_swarm_last_improved"):
            getattr(L, name).argtypes = [ctypes.c_void_p]
            getattr(L, name).restype = ctypes.c_int32
        L.orc_swarm_gf.argtypes = [ctypes.c_void_p]
        L.orc_swarm_gf.restype = ctypes.c_int64
        L.orc_swarm_counters.argtypes = [ctypes.c_void_p, _i64p]
        L.orc_swarm_export.argtypes = [ctypes.c_void_p, _u16p, _u16p, _u16p, _i64p, _i64p, _u16p]
        L.orc_swarm_vel_len.argtypes = [ctypes.c_void_p, ctypes.c_int32]
        L.orc_swarm_vel_len.restype = ctypes.c_int64
        L.orc_swarm_history.argtypes = [ctypes.c_void_p, _i64p, ctypes.c_int32]
        L.orc_swarm_history.restype = ctypes.c_int32
        _lib = L
    return _lib


def _p(a, t):
    return a.ctypes.data_as(t)


def _c(a, dtype):
    return np.ascontiguousarray(np.asarray(a, dtype=dtype))


# ---------------------------------------------------------------- primitives

def philox4x32_10(ctr, key) -> np.ndarray:
    c = _c(ctr, np.uint32)
    k = _c(key, np.uint32)
    out = np.zeros(4, np.uint32)
    lib().orc_philox4x32_10(_p(c, _u32p), _p(k, _u32p), _p(out, _u32p))
    return out


def draw(seed: int, phase: int, iteration: int, particle: int, d: int) -> int:
    return int(lib().orc_draw(seed, phase, iteration, particle, d))


def draws(seed: int, phase: int, iteration: int, particle: int, count: int) -> np.ndarray:
    out = np.zeros(count, np.uint32)
    lib().orc_draws(seed, phase, iteration, particle, count, _p(out, _u32p))
    return out


def segment_blocked(p, q, box, radius: float = 0.0) -> bool:
    p = _c(p, np.float64)
    q = _c(q, np.float64)
    b = _c(box, np.float64)
    return bool(lib().orc_segment_blocked(_p(p, _f64p), _p(q, _f64p), _p(b, _f64p), radius))


def cost_matrix(xyz, boxes, radius: float = 0.0, penalty: int = 1_000_000):
    """Returns (C int32 [n,n], status)."""
    xyz = _c(xyz, np.float64).reshape(-1, 3)
    boxes = _c(boxes, np.float64).reshape(-1, 6)
    n = xyz.shape[0]
    C = np.zeros((n, n), np.int32)
    st = lib().orc_cost_matrix(_p(xyz, _f64p), n, _p(boxes, _f64p), boxes.shape[0],
                               radius, penalty, _p(C, _i32p))
    return C, int(st)


def fitness(C, x) -> int:
    C = _c(C, np.int32)
    x = _c(x, np.uint16)
    return int(lib().orc_fitness(_p(C, _i32p), C.shape[0], _p(x, _u16p)))


def apply(x, v):
    """x + v for a list v of (a, b) label transpositions; returns a new array."""
    y = _c(x, np.uint16).copy()
    vv = _c(np.asarray(v, dtype=np.int64).reshape(-1, 2), np.uint16)
    lib().orc_apply(_p(y, _u16p), y.shape[0], _p(vv, _u16p), vv.shape[0])
    return y


def subtract(x2, x1):
    """x2 - x1 as an [len, 2] uint16 array of label transpositions."""
    a = _c(x2, np.uint16)
    b = _c(x1, np.uint16)
    n = a.shape[0]
    out = np.zeros((max(n - 1, 1), 2), np.uint16)
    ln = lib().orc_subtract(_p(a, _u16p), _p(b, _u16p), n, _p(out, _u16p))
    return out[:ln].copy()


def scaled_count(phi: float, u: int, length: int) -> int:
    """Number of transpositions kept by (phi * u / 2^32) . v when |v| = length."""
    return int(lib().orc_scaled_count(phi, u, length))


def boustrophedon(tags, variant: int):
    tags = _c(tags, np.int32).reshape(-1, 3)
    out = np.zeros(tags.shape[0], np.uint16)
    st = lib().orc_boustrophedon(_p(tags, _i32p), tags.shape[0], variant, _p(out, _u16p))
    return out, int(st)


def two_opt(C, x, max_moves: int = 0):
    """2-opt to convergence (best improvement). Returns (tour, cost, moves, pairs)."""
    C = _c(C, np.int32)
    y = _c(x, np.uint16).copy()
    f = np.array([fitness(C, y)], np.int64)
    pairs = np.zeros(1, np.int64)
    mv = lib().orc_two_opt(_p(C, _i32p), C.shape[0], _p(y, _u16p), _p(f, _i64p),
                           max_moves, _p(pairs, _i64p))
    return y, int(f[0]), int(mv), int(pairs[0])


def voxel_occupancy(origin, voxel: float, dims, boxes, r2: int):
    """Inflated occupancy of the voxel grid (Sec. 2.2): uint8 [nz, ny, nx]."""
    o = _c(origin, np.float64)
    d = _c(dims, np.int32)
    b = _c(np.asarray(boxes, np.float64).reshape(-1, 6), np.float64)
    occ = np.zeros((int(d[2]), int(d[1]), int(d[0])), np.uint8)
    st = lib().orc_voxel_occupancy(_p(o, ctypes.POINTER(ctypes.c_double)), voxel, _p(d, _i32p),
                                   _p(b, ctypes.POINTER(ctypes.c_double)), b.shape[0], r2,
                                   _p(occ, ctypes.POINTER(ctypes.c_uint8)))
    if st:
        raise ValueError(f"voxel_occupancy rejected its arguments ({st})")
    return occ


def cost_matrix_astar(xyz, occ, origin, voxel: float, dims, weights=(1, 1, 1), unit_mm: int = 500,
                      blocked_cost: int = 100_000_000, max_expansions: int = 100_000):
    """A* edge costs (Sec. 2.2) over an occupancy grid; returns (C int32 [n, n], status)."""
    x = _c(np.asarray(xyz, np.float64).reshape(-1, 3), np.float64)
    n = x.shape[0]
    oc = _c(occ, np.uint8)
    o = _c(origin, np.float64)
    d = _c(dims, np.int32)
    a = _c(weights, np.int32)
    C = np.zeros((n, n), np.int32)
    f64 = ctypes.POINTER(ctypes.c_double)
    st = lib().orc_cost_matrix_astar(_p(x, f64), n, _p(oc, ctypes.POINTER(ctypes.c_uint8)),
                                     _p(o, f64), voxel, _p(d, _i32p), _p(a, _i32p), unit_mm,
                                     blocked_cost, max_expansions, _p(C, _i32p))
    if st == ERR_ARG:
        raise ValueError("cost_matrix_astar rejected its arguments")
    return C, int(st)


def node_swap(C, x, max_moves: int = 0):
    """Node-swap exchange to convergence (best improvement). Returns (tour, cost, moves, pairs)."""
    C = _c(C, np.int32)
    y = _c(x, np.uint16).copy()
    f = np.array([fitness(C, y)], np.int64)
    pairs = np.zeros(1, np.int64)
    mv = lib().orc_node_swap(_p(C, _i32p), C.shape[0], _p(y, _u16p), _p(f, _i64p),
                             max_moves, _p(pairs, _i64p))
    return y, int(f[0]), int(mv), int(pairs[0])


# --------------------------------------------------------------------- swarm

class Swarm:
    """Oracle swarm: the loop of Fig. "pseudocode", one generation per iterate()."""

    def __init__(self, C, tags=None, swarm: int = 32, w: float = 1.0, phi1: float = 0.4,
                 phi2: float = 0.4, mut_period: int = 3, mut_swaps: int = 2,
                 det_frac_pct: int = 10, stall_limit: int = 0, flags: int = ALL,
                 trigger: int = 0, max_moves: int = 0, seed: int = 1):
        self.C = _c(C, np.int32)
        self.n = self.C.shape[0]
        self.S = int(swarm)
        tg = None if tags is None else _c(tags, np.int32).reshape(-1, 3)
        st = np.zeros(1, np.int32)
        self._h = lib().orc_swarm_new(
            _p(self.C, _i32p), self.n, None if tg is None else _p(tg, _i32p), self.S, w, phi1,
            phi2, mut_period, mut_swaps, det_frac_pct, stall_limit, flags, trigger, max_moves,
            seed, _p(st, _i32p))
        self.status = int(st[0])
        if not self._h:
            raise ValueError(f"oracle swarm rejected its arguments (status {self.status})")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().orc_swarm_free(h)
            self._h = None

    # phases
    def move(self, t: int):
        return lib().orc_swarm_move(self._h, t)

    def mutate(self, t: int):
        kept = np.zeros(self.S, np.int32)
        lib().orc_swarm_mutate(self._h, t, _p(kept, _i32p))
        return kept.astype(bool)

    def gbest(self):
        lib().orc_swarm_gbest(self._h)

    def two_opt(self, idx=None):
        if idx is None:
            lib().orc_swarm_two_opt(self._h, None, 0)
        else:
            ii = _c(idx, np.int32)
            lib().orc_swarm_two_opt(self._h, _p(ii, _i32p), ii.shape[0])

    def iterate(self) -> int:
        return lib().orc_swarm_iterate(self._h)

    def iterate_begin(self) -> bool:
        """The generation up to the edge exchange; True when the exchange runs."""
        run = np.zeros(1, np.int32)
        st = lib().orc_swarm_iterate_begin(self._h, _p(run, _i32p))
        if st < 0:
            raise RuntimeError(f"oracle generation failed ({st})")
        return bool(run[0])

    def iterate_end(self):
        """The rest of the generation after the exchange (gbest, history, stall)."""
        if lib().orc_swarm_iterate_end(self._h) < 0:
            raise RuntimeError("iterate_end without iterate_begin")

    def two_opt_part(self, idx):
        """Exchange of the particles idx only; returns (pairs, moves) without
        adding them to the swarm's counters.  Calls on disjoint sets of
        particles may run in concurrent threads (ctypes releases the GIL)."""
        ii = _c(idx, np.int32)
        out = np.zeros(2, np.int64)
        lib().orc_swarm_two_opt_part(self._h, _p(ii, _i32p), ii.shape[0], _p(out, _i64p))
        return int(out[0]), int(out[1])

    def iterate_threaded(self, threads: int = 1, sample=None):
        """One generation whose edge exchange runs on `threads` host threads,
        each on its own particles (the exchange of a particle reads and writes
        only that particle, so the result is that of iterate()).  With `sample`
        (particle indices) only those particles are exchanged and the
        generation is left open: the gbest after the exchange would need every
        particle.  Returns whether the exchange ran."""
        from concurrent.futures import ThreadPoolExecutor
        run = self.iterate_begin()
        if run:
            idx = np.arange(self.S, dtype=np.int32) if sample is None else _c(sample, np.int32)
            # one particle per task, in index order, so long and short
            # exchanges spread over the threads
            chunks = [idx[k:k + 1] for k in range(idx.shape[0])]
            with ThreadPoolExecutor(max(1, threads)) as ex:
                got = list(ex.map(self.two_opt_part, chunks))
            lib().orc_swarm_add_counters(self._h, sum(g[0] for g in got), sum(g[1] for g in got))
        if sample is None or not run:
            self.iterate_end()
        return run

    def load_state(self, st: dict):
        """Snapshot replay: takes the state of another run (same instance and
        parameters) as a dict with X, P, V (S x n, V as permutations), G, F,
        PF, gf, t, stall, done, history and optionally pairs, moves, runs."""
        S, n = self.S, self.n
        X = _c(st["X"], np.uint16).reshape(S, n)
        P = _c(st["P"], np.uint16).reshape(S, n)
        V = _c(st["V"], np.uint16).reshape(S, n)
        G = _c(st["G"], np.uint16).reshape(n)
        F = _c(st["F"], np.int64).reshape(S)
        PF = _c(st["PF"], np.int64).reshape(S)
        t = int(st["t"])
        hist = _c(st["history"], np.int64).reshape(-1)
        if hist.shape[0] != t:
            raise ValueError("history length differs from t")
        hist1 = hist if t else np.zeros(1, np.int64)
        cnt = np.array([st.get("pairs", 0), st.get("moves", 0), st.get("runs", 0)], np.int64)
        rc = lib().orc_swarm_import(self._h, _p(X, _u16p), _p(P, _u16p), _p(G, _u16p),
                                    _p(F, _i64p), _p(PF, _i64p), _p(V, _u16p), int(st["gf"]), t,
                                    int(st.get("stall", 0)), int(bool(st.get("done", False))),
                                    _p(hist1, _i64p), _p(cnt, _i64p))
        if rc:
            raise ValueError(f"oracle rejected the imported state ({rc})")

    def run(self, iterations: int) -> int:
        return lib().orc_swarm_run(self._h, iterations)

    # state
    @property
    def t(self) -> int:
        return lib().orc_swarm_t(self._h)

    @property
    def done(self) -> bool:
        return bool(lib().orc_swarm_done(self._h))

    @property
    def stall(self) -> int:
        return lib().orc_swarm_stall(self._h)

    @property
    def gf(self) -> int:
        return int(lib().orc_swarm_gf(self._h))

    @property
    def last_two_opt(self) -> bool:
        return bool(lib().orc_swarm_last_two_opt(self._h))

    @property
    def last_improved(self) -> bool:
        return bool(lib().orc_swarm_last_improved(self._h))

    def counters(self):
        out = np.zeros(3, np.int64)
        lib().orc_swarm_counters(self._h, _p(out, _i64p))
        return {"pairs": int(out[0]), "moves": int(out[1]), "two_opt_runs": int(out[2])}

    def state(self):
        S, n = self.S, self.n
        X = np.zeros((S, n), np.uint16)
        P = np.zeros((S, n), np.uint16)
        G = np.zeros(n, np.uint16)
        F = np.zeros(S, np.int64)
        PF = np.zeros(S, np.int64)
        V = np.zeros((S, n), np.uint16)
        lib().orc_swarm_export(self._h, _p(X, _u16p), _p(P, _u16p), _p(G, _u16p),
                               _p(F, _i64p), _p(PF, _i64p), _p(V, _u16p))
        c = self.counters()
        return {"X": X, "P": P, "G": G, "F": F, "PF": PF, "V": V, "gf": self.gf, "t": self.t,
                "stall": self.stall, "done": self.done, "history": self.history(),
                "pairs": c["pairs"], "moves": c["moves"], "runs": c["two_opt_runs"]}

    def vel_len(self, p: int) -> int:
        return int(lib().orc_swarm_vel_len(self._h, p))

    def history(self) -> np.ndarray:
        ln = lib().orc_swarm_history(self._h, None, 0)
        out = np.zeros(max(ln, 1), np.int64)
        lib().orc_swarm_history(self._h, _p(out, _i64p), ln)
        return out[:ln]
