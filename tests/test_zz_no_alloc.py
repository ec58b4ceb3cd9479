"""mpm_bin_static (the binning entry point whose sort scratch is a fixed device array) gives
the same keys and permutation as mpm_bin, bit for bit, on two calls in a row whose second
call is smaller than the first (so stale scratch contents from the first call would show),
allocates no device memory, and rejects sizes beyond its fixed maximum before launching.

Collected last on purpose: it must pass alone in a fresh process and after every other test.
"""
import numpy as np
import pytest

from paper_2412_12089_gb300 import mpm

pytestmark = pytest.mark.gpu


def positions(n, G, seed):
    rng = np.random.default_rng(seed)
    x = (0.05 + 0.9 * rng.random((n, 3))).astype(np.float32)
    k = min(n, 500)
    x[:k] = ((np.floor(x[:k] * G - 0.5) + 0.5) / G).astype(np.float32)  # on cell boundaries
    return x


def bin_both(x, G):
    import torch

    n = x.shape[0]
    xd = torch.as_tensor(x).cuda()
    k_ref = torch.empty(n, dtype=torch.int32, device="cuda")
    p_ref = torch.empty(n, dtype=torch.int32, device="cuda")
    k_st = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    p_st = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    mpm.mpm_bin(xd, n, G, k_ref, p_ref)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    mpm.mpm_bin_static(xd, n, G, k_st, p_st)
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    return k_ref.cpu().numpy(), p_ref.cpu().numpy(), k_st.cpu().numpy(), p_st.cpu().numpy(), free0 - free1


def test_static_bin_matches_bin_twice_in_a_row():
    cmax = mpm.mpm_bin_static_max()
    assert cmax == 1 << 18
    calls = [(200_003, 96, 11), (70_001, 48, 12)]
    for c, (n, G, seed) in enumerate(calls):
        assert n <= cmax
        k_ref, p_ref, k_st, p_st, grown = bin_both(positions(n, G, seed), G)
        assert np.array_equal(k_st, k_ref), (n, G)
        assert np.array_equal(p_st, p_ref), (n, G)
        assert np.array_equal(np.sort(p_st.view(np.uint32)), np.arange(n, dtype=np.uint32))
        if c == 0:
            # a first call in the process may load the module that holds the fixed array
            # (4 MiB + 64 KiB, placed in 2 MiB pages) when CUDA loads modules lazily
            assert grown <= 8 << 20, grown
        else:
            assert grown == 0, grown  # no device memory taken by the call


def test_static_bin_rejects_beyond_max():
    import torch

    n = mpm.mpm_bin_static_max() + 1
    xd = torch.full((n, 3), 0.5, dtype=torch.float32, device="cuda")
    keys = torch.zeros(n, dtype=torch.int32, device="cuda")
    perm = torch.zeros(n, dtype=torch.int32, device="cuda")
    with pytest.raises(mpm.MpmError) as ei:
        mpm.mpm_bin_static(xd, n, 32, keys, perm)
    assert ei.value.code == 1  # MPM_ERR_INVALID_ARG
    torch.cuda.synchronize()
    assert int(keys.abs().sum()) == 0 and int(perm.abs().sum()) == 0
