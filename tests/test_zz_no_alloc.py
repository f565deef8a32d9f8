"""The allocation-free key sort (hv_sort_keys_noalloc) against the ordinary
one (hv_sort_keys), through the C ABI.

Some callers cannot allocate device memory at the moment they sort (their
own pool owns the GPU, or the loop must not enter the CUDA allocator, which
can synchronise the device); the no-allocation variant serves them from a
static device array.  Two calls in a row with different sizes and keys must
each give exactly the ordinary sort's permutation and counts (integer work:
bit-exact), so nothing left in the shared array by the first call leaks
into the second.  This file is collected last; it must pass both alone and
after the other tests."""
import numpy as np
import pytest

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


def test_noalloc_sort_matches_allocating_sort_twice(hvmod):
    import torch
    rng = np.random.default_rng(2024)
    for n, nkeys in ((300_001, 70_000), (123_457, 4_099)):
        keys = torch.from_numpy(rng.integers(0, nkeys, n).astype(np.int32)).cuda()
        ref_perm, ref_counts = hvmod.hv_sort_keys(keys, nkeys)
        perm = torch.full((n,), -1, dtype=torch.int32, device="cuda")
        counts = torch.full((nkeys,), -1, dtype=torch.int32, device="cuda")
        hvmod.hv_sort_keys_noalloc(keys, nkeys, perm, counts)
        assert torch.equal(perm, ref_perm)
        assert torch.equal(counts, ref_counts)


def test_noalloc_sort_rejects_too_many_keys(hvmod):
    import torch
    n = (1 << 20) + 1
    keys = torch.zeros(n, dtype=torch.int32, device="cuda")
    perm = torch.empty(n, dtype=torch.int32, device="cuda")
    with pytest.raises(hvmod.HVError, match="limit"):
        hvmod.hv_sort_keys_noalloc(keys, 4, perm)
