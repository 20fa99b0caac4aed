"""lcs_partition_noalloc: the allocation-free partition for callers that may
not allocate device memory (inside graph capture, under a fixed memory
budget, in latency-critical loops).

Called through the C ABI with ctypes and compared, bit for bit (the result
is integer work), with lcs_partition -- the allocating entry point -- on two
calls in a row with different inputs, so that the second call runs on a
scratch array that still holds the first call's contents, and as a call
recorded into a CUDA graph and replayed on new keys.  This file is
collected last so that a stop at the first failure has run every other test.
"""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2604_11008_gb300 as lcs
    from paper_2604_11008_gb300 import build
    build.build()
    return torch, lcs


def noalloc(torch, lcs, keys_np, nbins):
    keys = torch.from_numpy(keys_np.astype(np.int32)).cuda()
    n = keys.numel()
    perm = torch.empty(max(n, 1), dtype=torch.int32, device="cuda")
    off = torch.empty(nbins + 1, dtype=torch.int64, device="cuda")
    status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = lcs.lib().lcs_partition_noalloc(C.c_void_p(keys.data_ptr()), n, nbins,
                                         C.c_void_p(perm.data_ptr()), C.c_void_p(off.data_ptr()),
                                         C.c_void_p(status.data_ptr()), stream)
    torch.cuda.synchronize()
    return rc, perm[:n].cpu().numpy(), off.cpu().numpy(), int(status.item())


def test_noalloc_matches_allocating_partition_on_two_calls(env):
    torch, lcs = env
    g = np.random.default_rng(2024)
    for n, nbins in ((lcs.PARTITION_NOALLOC_MAX_N, 1000), (77777, 2),
                     (lcs.PARTITION_NOALLOC_MAX_N, 65536), (0, 5), (1, 1)):
        keys = g.integers(0, nbins, n)
        rc, perm, off, status = noalloc(torch, lcs, keys, nbins)
        assert rc == lcs.LCS_OK
        ref_perm, ref_off, ref_status = lcs.partition(keys, nbins)
        assert np.array_equal(perm, ref_perm.cpu().numpy())
        assert np.array_equal(off, ref_off.cpu().numpy())
        assert status == int(ref_status.item()) == lcs.LCS_OK


def test_noalloc_rejects_sizes_beyond_its_scratch(env):
    torch, lcs = env
    keys = np.zeros(lcs.PARTITION_NOALLOC_MAX_N + 1, np.int32)
    rc, _, _, status = noalloc(torch, lcs, keys, 4)
    assert rc == lcs.LCS_ERR_ARG
    assert status == -1  # nothing was enqueued


def test_noalloc_recorded_in_a_cuda_graph_and_replayed(env):
    """The use case the header names: a call made while the stream is being
    captured into a CUDA graph (after one call outside capture, which looks
    up the scratch address), replayed on new keys written into the same
    input buffer; every replay equals lcs_partition on those keys."""
    torch, lcs = env
    n, nbins = 100000, 513
    g = np.random.default_rng(2025)
    keys = torch.from_numpy(g.integers(0, nbins, n).astype(np.int32)).cuda()
    perm = torch.empty(n, dtype=torch.int32, device="cuda")
    off = torch.empty(nbins + 1, dtype=torch.int64, device="cuda")
    status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    side = torch.cuda.Stream()

    def call(stream):
        return lcs.lib().lcs_partition_noalloc(
            C.c_void_p(keys.data_ptr()), n, nbins, C.c_void_p(perm.data_ptr()),
            C.c_void_p(off.data_ptr()), C.c_void_p(status.data_ptr()),
            C.c_void_p(stream.cuda_stream))

    with torch.cuda.stream(side):
        assert call(side) == lcs.LCS_OK  # outside capture: caches the scratch address
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=side):
        rc = call(side)
    assert rc == lcs.LCS_OK
    for _ in range(3):
        keys.copy_(torch.from_numpy(g.integers(0, nbins, n).astype(np.int32)))
        status.fill_(-1)
        torch.cuda.synchronize()
        graph.replay()
        torch.cuda.synchronize()
        ref_perm, ref_off, _ = lcs.partition(keys.cpu().numpy(), nbins)
        assert int(status.item()) == lcs.LCS_OK
        assert torch.equal(perm, ref_perm)
        assert torch.equal(off, ref_off)
