"""The allocation-free key sort (hv_sort_keys_noalloc) against the ordinary
one (hv_sort_keys) and the oracle's stable counting sort, through the C ABI.

Some callers cannot allocate device memory at the moment they sort (their
own pool owns the GPU, or the loop must not enter the CUDA allocator, which
can synchronise the device); the no-allocation variant serves them from a
static device array.  Two calls in a row with different sizes and keys must
each give exactly the ordinary sort's permutation and counts, and the
oracle's (integer work: bit-exact), so nothing left in the shared array by
the first call leaks into the second.  A call with an out-of-range key must
fail and the next in-range call must still be exact (the error flag in the
shared array is cleared per call).  This file is collected last; it must
pass both alone and after the other tests."""
import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hvmod():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2305_05600_gb300 import hv
    hv.lib()
    hv.hv_set_allocator(True)
    return hv


def noalloc(hvmod, keys_np, nkeys, with_counts=True):
    import torch
    n = keys_np.shape[0]
    keys = torch.from_numpy(keys_np.astype(np.int32)).cuda()
    perm = torch.full((max(n, 1),), -1, dtype=torch.int32, device="cuda")
    counts = torch.full((nkeys,), -1, dtype=torch.int32, device="cuda") if with_counts else None
    hvmod.hv_sort_keys_noalloc(keys, nkeys, perm, counts)
    return keys, perm[:n], counts


def test_noalloc_sort_matches_allocating_sort_and_oracle_twice(hvmod):
    import torch
    rng = np.random.default_rng(2024)
    for n, nkeys in ((300_001, 70_000), (123_457, 4_099)):
        k = rng.integers(0, nkeys, n)
        keys, perm, counts = noalloc(hvmod, k, nkeys)
        ref_perm, ref_counts = hvmod.hv_sort_keys(keys, nkeys)
        assert torch.equal(perm, ref_perm)
        assert torch.equal(counts, ref_counts)
        operm, ocounts, _ = O.sort_stable(k, nkeys)
        assert np.array_equal(perm.cpu().numpy().astype(np.int64), operm)
        assert np.array_equal(counts.cpu().numpy().astype(np.int64), ocounts)


def test_noalloc_sort_rejects_out_of_range_keys_then_recovers(hvmod):
    rng = np.random.default_rng(7)
    for bad in (5, -1):
        k = rng.integers(0, 5, 1000)
        k[313] = bad
        with pytest.raises(hvmod.HVError, match="out of range"):
            noalloc(hvmod, k, 5)
        good = rng.integers(0, 5, 777)
        _, perm, counts = noalloc(hvmod, good, 5)
        operm, ocounts, _ = O.sort_stable(good, 5)
        assert np.array_equal(perm.cpu().numpy().astype(np.int64), operm)
        assert np.array_equal(counts.cpu().numpy().astype(np.int64), ocounts)


def test_noalloc_sort_without_counts_and_empty(hvmod):
    rng = np.random.default_rng(8)
    k = rng.integers(0, 300, 4097)
    _, perm, counts = noalloc(hvmod, k, 300, with_counts=False)
    assert counts is None
    operm, _, _ = O.sort_stable(k, 300)
    assert np.array_equal(perm.cpu().numpy().astype(np.int64), operm)
    _, perm0, counts0 = noalloc(hvmod, np.zeros(0, np.int64), 3)
    assert perm0.numel() == 0
    assert counts0.cpu().numpy().tolist() == [0, 0, 0]


def test_noalloc_binding_checks_buffer_sizes(hvmod):
    import torch
    keys = torch.zeros(100, dtype=torch.int32, device="cuda")
    with pytest.raises(ValueError, match="perm"):
        hvmod.hv_sort_keys_noalloc(keys, 4, torch.empty(99, dtype=torch.int32, device="cuda"))
    with pytest.raises(ValueError, match="counts"):
        hvmod.hv_sort_keys_noalloc(keys, 4, torch.empty(100, dtype=torch.int32, device="cuda"),
                                   torch.empty(3, dtype=torch.int32, device="cuda"))
    with pytest.raises(TypeError):
        hvmod.hv_sort_keys_noalloc(keys, 4, torch.empty(100, dtype=torch.int64, device="cuda"))
    with pytest.raises(ValueError, match="contiguous"):
        hvmod.hv_sort_keys_noalloc(torch.zeros(200, dtype=torch.int32, device="cuda")[::2], 4,
                                   torch.empty(100, dtype=torch.int32, device="cuda"))


def test_noalloc_sort_rejects_too_many_keys(hvmod):
    import torch
    n = (1 << 20) + 1
    keys = torch.zeros(n, dtype=torch.int32, device="cuda")
    perm = torch.empty(n, dtype=torch.int32, device="cuda")
    with pytest.raises(hvmod.HVError, match="limit"):
        hvmod.hv_sort_keys_noalloc(keys, 4, perm)
