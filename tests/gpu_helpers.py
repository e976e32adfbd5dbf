"""Shared helpers of the GPU tests: build inputs on the device and run both sides."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_1706_04399_gb300 import dpso, inputs  # noqa: E402

DEV = "cuda:0"


def cost_matrix_gpu(inst: "inputs.Instance", radius: float = 0.0, penalty: int = 1_000_000):
    xyz = torch.from_numpy(inst.xyz).to(DEV)
    boxes = torch.from_numpy(inst.boxes.reshape(-1, 6)).to(DEV) if inst.m else None
    C = torch.empty((inst.n, inst.n), dtype=torch.int32, device=DEV)
    cp = dpso.default_cost_params(uav_radius_m=radius, blocked_penalty_mm=penalty)
    dpso.dpso_cost_matrix(xyz, inst.n, boxes, inst.m, cp, C)
    torch.cuda.synchronize()
    return C


ORACLE_KW = ("w", "phi1", "phi2", "mut_period", "mut_swaps", "det_frac_pct", "stall_limit",
             "trigger", "max_moves")


def both_swarms(C_np, C_dev, tags, swarm, seed, flags=dpso.FLAGS_ALL, **kw):
    """A GPU swarm and an oracle swarm with the same parameters."""
    p = dpso.default_params(swarm=swarm, flags=flags)
    for k, v in kw.items():
        setattr(p, "two_opt_trigger" if k == "trigger" else k, v)
    n = C_np.shape[0]
    gpu = dpso.Swarm(C_dev, n, tags, p, seed)
    ref = oracle.Swarm(C_np, tags, swarm=swarm, seed=seed, flags=flags, **kw)
    return gpu, ref


def assert_same_state(gpu_state, ref: "oracle.Swarm", what=""):
    rs = ref.state()
    for key in ("X", "P", "V", "G", "F", "PF"):
        a, b = gpu_state[key], rs[key]
        if not np.array_equal(a, b):
            bad = np.argwhere(a != b)
            raise AssertionError(f"{what}: {key} differs at {bad[:5].tolist()} "
                                 f"({len(bad)} entries)")
    assert gpu_state["gf"] == rs["gf"], (what, gpu_state["gf"], rs["gf"])
    assert gpu_state["t"] == rs["t"], (what, gpu_state["t"], rs["t"])
    assert np.array_equal(gpu_state["history"], ref.history()), what


def checkpoint_with_flags(blob: bytes, flags: int) -> bytes:
    """The checkpoint `blob` with its parameter block's flags replaced, so it
    can be loaded into a swarm created with those flags (dpso_set_state
    accepts only a checkpoint taken with the swarm's own parameters)."""
    import ctypes
    import struct
    off = dpso._HDR_SIZE - ctypes.sizeof(dpso.dpso_params) + dpso.dpso_params.flags.offset
    out = bytearray(blob)
    struct.pack_into("<i", out, off, flags)
    return bytes(out)


def host_threads() -> int:
    import os
    try:
        return max(1, len(os.sched_getaffinity(0)))
    except AttributeError:
        return max(1, os.cpu_count() or 1)
