"""The allocation-free sort entry point (vr_sort_u64_noalloc).

It serves callers that must not allocate device memory during a library call
(for example code working inside a fixed, pre-reserved device-memory budget),
so its scratch is a static device array of bounded size instead of memory
allocated per call.  These tests check, through the C ABI, that it returns
exactly what the allocating entry point vr_sort_u64 returns (integer keys:
bit-exact), on two calls in a row -- the second call reuses the array the
first one left behind -- and that sizes above its limit are refused.

The file name makes pytest collect it last.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def vr():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("a CUDA device is required for the gpu tests")
    from paper_2502_05063_b300 import vr as _vr
    return _vr


def _pair(seed, num, bits):
    import torch
    rng = np.random.default_rng(seed)
    keys = rng.integers(0, 2 ** 63, size=num, dtype=np.int64)
    if bits < 64:
        keys &= (1 << bits) - 1
    keys[: num // 4] = keys[num // 4: 2 * (num // 4)]  # equal keys: stability matters
    vals = np.arange(num, dtype=np.int64)
    return torch.from_numpy(keys).cuda(), torch.from_numpy(vals).cuda()


def test_noalloc_matches_allocating_sort_twice(vr):
    cases = [(11, 200000, 49), (12, 4097, 64)]  # two calls in a row, different sizes and widths
    for seed, num, bits in cases:
        k1, v1 = _pair(seed, num, bits)
        k2, v2 = k1.clone(), v1.clone()
        vr.sort_u64(k1, v1, bits)
        vr.sort_u64_noalloc(k2, v2, bits)
        assert k2.cpu().numpy().tolist() == k1.cpu().numpy().tolist()
        assert v2.cpu().numpy().tolist() == v1.cpu().numpy().tolist()


def test_noalloc_keys_only_and_limit(vr):
    import torch
    k1, _ = _pair(13, vr.VR_SORT_NOALLOC_MAX_KEYS, 40)
    k2 = k1.clone()
    vr.sort_u64(k1, None, 40)
    vr.sort_u64_noalloc(k2, None, 40)
    assert k2.cpu().numpy().tolist() == k1.cpu().numpy().tolist()
    big = torch.zeros(vr.VR_SORT_NOALLOC_MAX_KEYS + 1, dtype=torch.int64, device="cuda")
    with pytest.raises(vr.VRError) as e:
        vr.sort_u64_noalloc(big, None, 64)
    assert e.value.name == "VR_ERR_INVALID_ARG"
