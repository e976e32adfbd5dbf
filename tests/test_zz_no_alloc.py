"""dpso_two_opt_noalloc: the 2-opt entry point for callers that must not
allocate device memory (a start-up-reserved on-board planning loop, or a
process whose GPU memory belongs to another allocator).  Its scratch is a fixed
array inside the library; its results must equal dpso_two_opt's.

Kept in a file of its own, collected last.
"""
import numpy as np
import pytest

from gpu_helpers import DEV, torch  # noqa: F401
from paper_1706_04399_gb300 import dpso, inputs

pytestmark = pytest.mark.gpu


def _run(fn, C_np, tours, max_moves=0):
    n = C_np.shape[0]
    C = torch.from_numpy(C_np).to(DEV)
    T = torch.from_numpy(tours.view(np.int16).copy()).to(DEV)
    cost = torch.empty(len(tours), dtype=torch.int64, device=DEV)
    pairs, moves = fn(C, n, T, len(tours), cost, max_moves)
    return T.cpu().numpy().view(np.uint16), cost.cpu().numpy(), pairs, moves


def test_no_alloc_matches_allocating_entry_point_twice():
    # two calls in a row; the second is smaller, so stale per-tour counts of
    # the first call would show up in its totals if they were not cleared
    cases = [(inputs.random_cost_matrix(97, 3), inputs.random_tours(97, 40, 4), 0),
             (inputs.random_cost_matrix(61, 5), inputs.random_tours(61, 7, 6), 3)]
    for C_np, tours, cap in cases:
        want = _run(dpso.dpso_two_opt, C_np, tours, cap)
        got = _run(dpso.dpso_two_opt_noalloc, C_np, tours, cap)
        assert np.array_equal(got[0], want[0])          # tours, bit-exact
        assert np.array_equal(got[1], want[1])          # costs
        assert got[2:] == want[2:]                      # pairs evaluated, moves applied
        assert got[3] > 0


def test_no_alloc_call_leaves_device_memory_unchanged():
    # the property the entry point exists for: after a first call (which may
    # load the library's kernels on the device), a call takes no device
    # memory, neither from the driver nor from torch's caching allocator
    C_np, tours = inputs.random_cost_matrix(83, 8), inputs.random_tours(83, 33, 9)
    n = C_np.shape[0]
    C = torch.from_numpy(C_np).to(DEV)
    T0 = torch.from_numpy(tours.view(np.int16).copy()).to(DEV)
    T = T0.clone()
    cost = torch.empty(len(tours), dtype=torch.int64, device=DEV)
    dpso.dpso_two_opt_noalloc(C, n, T, len(tours), cost)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    alloc0, reserved0 = torch.cuda.memory_allocated(), torch.cuda.memory_reserved()
    for _ in range(3):
        T.copy_(T0)                     # no allocation inside the measured stretch
        dpso.dpso_two_opt_noalloc(C, n, T, len(tours), cost)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert (torch.cuda.memory_allocated(), torch.cuda.memory_reserved()) == (alloc0, reserved0)


def test_no_alloc_rejects_counts_beyond_its_array():
    n = 10
    C = torch.from_numpy(inputs.random_cost_matrix(n, 1)).to(DEV)
    T = torch.zeros((1, n), dtype=torch.int16, device=DEV)
    cost = torch.empty(1, dtype=torch.int64, device=DEV)
    with pytest.raises(dpso.DpsoError) as e:
        dpso.dpso_two_opt_noalloc(C, n, T, dpso.NOALLOC_MAX_TOURS + 1, cost)
    assert e.value.status == dpso.ERR_RANGE
