"""The allocation-free F half (nmfkl_sweep_F_noalloc) against the regular one.

Some callers cannot call cudaMalloc (another runtime owns the device memory
through its own pool, or the path cannot afford cudaMalloc's device-wide
synchronization, or must not hit out-of-memory after start-up). For them the
library offers an F half whose scratch is a fixed array inside the library.
This test calls it through the C ABI on caller-owned device buffers, twice in
a row (the second call runs on whatever the first left in the shared
scratch), and compares each result with the regular nmfkl_sweep_F on the
same start. Every column here has 65..128 nonzeros, so both paths run the
same kernel shape and must agree within the parity tests' per-entry bar.

This file is named so that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest

import paper_1604_04026_gb300 as nk
from paper_1604_04026_gb300 import _native, synth

from _util import within

pytestmark = pytest.mark.gpu


def _columns_65_to_128(n, m, seed):
    rng = np.random.default_rng(seed)
    lens = rng.integers(65, 129, size=m)
    colptr = np.zeros(m + 1, dtype=np.int64)
    colptr[1:] = np.cumsum(lens)
    rowidx = np.concatenate([np.sort(rng.choice(n, size=L, replace=False)) for L in lens]).astype(np.int32)
    val = rng.integers(1, 6, size=int(colptr[-1])).astype(np.float32)
    return synth.from_csc(n, m, colptr, rowidx, val)


def _unit_major(torch, M, ldr):
    """(r x cols) numpy -> (cols x ldr) CUDA tensor, padding zero."""
    r, cols = M.shape
    out = torch.zeros((cols, ldr), dtype=torch.float32)
    out[:, :r] = torch.from_numpy(np.ascontiguousarray(M.T))
    return out.cuda().contiguous()


def test_noalloc_matches_regular_twice():
    import torch

    V = _columns_65_to_128(4000, 3000, seed=5)
    r = 40
    ldr = (r + 3) // 4 * 4
    W0 = synth.uniform_init(r, V.n, 3, 0)
    F0 = synth.uniform_init(r, V.m, 3, 1)
    p = nk.default_params(r, seed=21, list_mode=1)

    with nk.NMFKL(V.n, V.m, params=p) as model:
        model.set_data(V)
        model.init(W0, F0)
        model.sweep_F(4)
        F_ref = model.get_F()
        assert {b["kernel"] for b in model.plan() if b["side"] == 0 and b["kernel"].startswith("sweep_")} == \
            {"sweep_warp_k4"}

    lib = _native.load()
    colptr = torch.from_numpy(V.colptr).cuda()
    rowidx = torch.from_numpy(V.rowidx).cuda()
    val = torch.from_numpy(V.val).cuda()
    Wt = _unit_major(torch, W0, ldr)
    max_len = int(np.diff(V.colptr).max())
    for call in range(2):
        Ft = _unit_major(torch, F0, ldr)
        st = lib.nmfkl_sweep_F_noalloc(ctypes.byref(p), V.n, V.m, max_len, colptr.data_ptr(),
                                       rowidx.data_ptr(), val.data_ptr(), Wt.data_ptr(), Ft.data_ptr(), 4, None)
        assert st == 0, (call, _native.STATUS_NAMES.get(st))
        F = Ft.cpu().numpy()[:, :r].T
        assert within(F, F_ref).all(), call
        assert np.array_equal(F, F_ref), call


def test_noalloc_rejects_sizes_beyond_its_limits():
    import torch

    lib = _native.load()
    V = _columns_65_to_128(500, 20, seed=1)
    p = nk.default_params(8)
    colptr = torch.from_numpy(V.colptr).cuda()
    rowidx = torch.from_numpy(V.rowidx).cuda()
    val = torch.from_numpy(V.val).cuda()
    # a nonzero start, so that a kernel writing into a refused column would show
    Wt = _unit_major(torch, synth.uniform_init(8, V.n, 7, 0), 8)
    Ft = _unit_major(torch, synth.uniform_init(8, V.m, 7, 1), 8)
    F_start = Ft.clone()
    args = (colptr.data_ptr(), rowidx.data_ptr(), val.data_ptr(), Wt.data_ptr(), Ft.data_ptr(), 0, None)
    # max_len above the 256 limit
    assert lib.nmfkl_sweep_F_noalloc(ctypes.byref(p), V.n, V.m, 300, *args) == 1
    # r above 256
    big = nk.default_params(8)
    big.r = 300
    assert lib.nmfkl_sweep_F_noalloc(ctypes.byref(big), V.n, V.m, 128, *args) == 1
    assert torch.equal(Ft, F_start)
    # factors off a 16-byte boundary are refused before any launch
    Wt_off = torch.zeros(Wt.numel() + 1, dtype=torch.float32, device="cuda")
    bad = (args[0], args[1], args[2], Wt_off.data_ptr() + 4, args[4], 0, None)
    assert lib.nmfkl_sweep_F_noalloc(ctypes.byref(p), V.n, V.m, 128, *bad) == 1
    assert torch.equal(Ft, F_start)
    # max_len 32 selects the kernel that holds 32 nonzeros per column; every
    # column here is longer, so each is refused after the launch and left as it was
    assert lib.nmfkl_sweep_F_noalloc(ctypes.byref(p), V.n, V.m, 32, *args) == 1
    assert torch.equal(Ft, F_start)
