"""The allocation-free brick sort (mpm_sort_bricks_noalloc), for callers that
cannot allocate device memory while they run, against the sort that
mpm_substep performs with the context's own scratch.

Both order particles by the brick of their base cell; the order inside a brick
is not unique, so the test compares what is: the brick of every sorted slot
and the brick boundaries.  Two calls in a row on different inputs check that
the shared static scratch is reset between calls.  This file is collected last.
"""
import numpy as np
import pytest

import oracle
from paper_2502_18437_gb300 import mpm, workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def brick_keys(x, n):
    return oracle.sort_by_brick(n, x)[0]


def sorted_by_context(sc):
    # storage order after one substep = the substep's sort of the input positions
    with mpm.from_workload(sc) as sim:
        sim.substep(sc["dt"], 1)
        return sim.read_state(0, ("order",))["order"]


def noalloc_sort(x, n):
    N = len(x)
    xd = torch.tensor(x, device="cuda")
    perm = torch.full((N,), -1, dtype=torch.int32, device="cuda")
    start = torch.full(((n // 4) ** 3 + 1,), -1, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    status = mpm.mpm_sort_bricks_noalloc(n, N, xd.data_ptr(), perm.data_ptr(), start.data_ptr(), stream)
    assert status == 0, mpm.mpm_status_string(status)
    torch.cuda.synchronize()
    return perm.cpu().numpy(), start.cpu().numpy()


def test_noalloc_sort_matches_context_sort_on_two_calls():
    cases = [W.tissue_block(N=65536, n=64), W.tissue_slab(cells=(40, 8, 40), n=64, substeps=1, with_tools=False)]
    for sc in cases:  # two calls in a row, different sizes and layouts
        n = sc["n"]
        order = sorted_by_context(sc)
        perm, start = noalloc_sort(sc["x"], n)
        N = len(sc["x"])
        assert np.array_equal(np.sort(perm), np.arange(N))  # a permutation
        keys = brick_keys(sc["x"], n)
        assert np.array_equal(keys[perm], keys[order])  # same brick in every slot
        counts = np.bincount(keys, minlength=(n // 4) ** 3)
        assert np.array_equal(start, np.concatenate([[0], np.cumsum(counts)]))


def test_noalloc_sort_rejects_sizes_beyond_its_scratch():
    x = torch.zeros((4, 3), device="cuda")
    p = torch.zeros(4, dtype=torch.int32, device="cuda")
    assert mpm.mpm_sort_bricks_noalloc(512, 4, x.data_ptr(), p.data_ptr()) == -7
    assert mpm.mpm_sort_bricks_noalloc(64, (1 << 20) + 1, x.data_ptr(), p.data_ptr()) == -7
    assert mpm.mpm_sort_bricks_noalloc(30, 4, x.data_ptr(), p.data_ptr()) == -1


def test_noalloc_sort_at_its_limits_and_degenerate_calls():
    # The sizes the static scratch is built for (N = MPM_NOALLOC_MAX_PARTICLES on
    # a 256^3 grid: 262,144 bricks + the end offset), without brick_start, and
    # an empty input (every brick starts at 0).
    sc = W.tissue_block(N=1 << 20, n=256)
    n, N = sc["n"], len(sc["x"])
    keys = brick_keys(sc["x"], n)
    perm, start = noalloc_sort(sc["x"], n)
    assert np.array_equal(np.sort(perm), np.arange(N))
    assert np.all(np.diff(keys[perm]) >= 0)
    assert np.array_equal(start, np.concatenate([[0], np.cumsum(np.bincount(keys, minlength=(n // 4) ** 3))]))
    xd = torch.tensor(sc["x"], device="cuda")
    p2 = torch.full((N,), -1, dtype=torch.int32, device="cuda")
    assert mpm.mpm_sort_bricks_noalloc(n, N, xd.data_ptr(), p2.data_ptr(), None,
                                       torch.cuda.current_stream().cuda_stream) == 0
    torch.cuda.synchronize()
    assert np.array_equal(keys[p2.cpu().numpy()], keys[perm])
    start0 = torch.full(((64 // 4) ** 3 + 1,), -1, dtype=torch.int32, device="cuda")
    assert mpm.mpm_sort_bricks_noalloc(64, 0, None, None, start0.data_ptr(),
                                       torch.cuda.current_stream().cuda_stream) == 0
    torch.cuda.synchronize()
    assert not start0.cpu().numpy().any()
