"""amber_rank_noalloc: the ranking for callers that cannot allocate device memory.

Callers such as a plug-in inside a framework that owns the device pool, or a
real-time loop that must not reach cudaMalloc, rank through this entry point,
which keeps its working storage in a fixed array inside the library.  Its
result must be exactly amber_rank's (ranks are integers: bit-exact), call
after call, since every call reuses that one array.  This file is collected
last so a failure here does not stop the rest of the suite.
"""
import ctypes as C

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

MAX_CELLS = 1 << 20


@pytest.fixture(scope="module")
def B():
    import __graft_entry__ as g
    g.build()
    from paper_2109_10375_gb300 import binding
    return binding


def _keys(n, seed):
    g = np.random.default_rng(seed)
    J = g.normal(size=n).astype(np.float32)
    J[:: 5] = np.round(J[:: 5], 1)  # many exact ties
    return torch.from_numpy(J).cuda()


def test_rank_noalloc_matches_rank_on_consecutive_calls(B):
    stream = torch.cuda.current_stream()
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    with B.Context(MAX_CELLS) as ctx:
        for n, seed in [(777_777, 1), (MAX_CELLS, 2)]:  # two calls in a row on the shared array
            J = _keys(n, seed)
            ref = ctx.rank(J)
            out = torch.full((n,), -1, dtype=torch.int32, device="cuda")
            rc = B.lib.amber_rank_noalloc(C.c_void_p(J.data_ptr()), n, C.c_void_p(out.data_ptr()),
                                          C.c_void_p(status.data_ptr()), C.c_void_p(stream.cuda_stream))
            assert rc == B.AMBER_OK, B.status_string(rc)
            torch.cuda.synchronize()
            assert ctx.sync_status() == 0
            assert int(status.item()) == 0
            assert torch.equal(out, ref)


def test_rank_noalloc_rejects_more_cells_than_its_scratch(B):
    J = torch.zeros(8, device="cuda")
    out = torch.zeros(8, dtype=torch.int32, device="cuda")
    rc = B.lib.amber_rank_noalloc(C.c_void_p(J.data_ptr()), MAX_CELLS + 1, C.c_void_p(out.data_ptr()), None, None)
    assert rc == B.AMBER_ERR_CAPACITY


@pytest.mark.parametrize("n", [1, 4095, 4097])
def test_rank_noalloc_small_and_ragged_sizes_without_status_word(B, n):
    # fewer keys than one sort tile, and a ragged tail; no caller status word,
    # so device errors go to the array's own word (none are expected)
    stream = torch.cuda.current_stream()
    J = _keys(n, 10 + n)
    with B.Context(MAX_CELLS) as ctx:
        ref = ctx.rank(J)
        for _ in range(2):
            out = torch.full((n,), -1, dtype=torch.int32, device="cuda")
            rc = B.lib.amber_rank_noalloc(C.c_void_p(J.data_ptr()), n, C.c_void_p(out.data_ptr()), None,
                                          C.c_void_p(stream.cuda_stream))
            assert rc == B.AMBER_OK, B.status_string(rc)
            torch.cuda.synchronize()
            assert torch.equal(out, ref)


def test_rank_noalloc_view_off_a_16_byte_boundary(B):
    # J[1:] starts 4 bytes past an aligned allocation: the histogram reads it
    # element by element instead of 16 bytes at a time
    stream = torch.cuda.current_stream()
    base = _keys(300_001, 77)
    J = base[1:]
    assert J.data_ptr() % 16 != 0
    n = J.numel()
    with B.Context(MAX_CELLS) as ctx:
        ref = ctx.rank(J.clone())
        view = ctx.rank(J)
        out = torch.full((n,), -1, dtype=torch.int32, device="cuda")
        rc = B.lib.amber_rank_noalloc(C.c_void_p(J.data_ptr()), n, C.c_void_p(out.data_ptr()), None,
                                      C.c_void_p(stream.cuda_stream))
        assert rc == B.AMBER_OK
        torch.cuda.synchronize()
        assert ctx.sync_status() == 0
    assert torch.equal(view, ref)
    assert torch.equal(out, ref)
