"""The allocation-free loss/gradient entry point (for callers that cannot
allocate device memory while they run, e.g. inside a host framework that
owns the allocator) gives the same loss and gradient as the regular one, on
two calls in a row through the C ABI, while the library's allocation hook
would fail any allocation, and refuses batches beyond its fixed scratch. Collected last on purpose: it must pass alone in a fresh process
and after every other test."""
import ctypes

import numpy as np
import pytest
import torch

import paper_2607_20766_b300 as shp
from paper_2607_20766_b300 import _binding as B

pytestmark = pytest.mark.gpu


def _call(fn, params, x, target, rows, n, grad, loss):
    return fn(params.data_ptr(), x.data_ptr(), target.data_ptr(), None if rows is None else rows.data_ptr(), n,
              grad.data_ptr(), loss.data_ptr(), torch.cuda.current_stream().cuda_stream)


def test_noalloc_matches_regular_entry_point():
    lib = shp.load_library()
    rng = np.random.default_rng(3)
    dev = "cuda"
    for call in range(2):  # two calls in a row: the fixed scratch keeps the previous call's contents
        n_rows = 8192 if call == 0 else 777
        x = torch.tensor(rng.uniform(0, 2.5, (9000, B.MLP_IN)), dtype=torch.float32, device=dev)
        t = torch.tensor(rng.uniform(0.2, 1.0, 9000), dtype=torch.float32, device=dev)
        p = torch.tensor(rng.normal(scale=0.1, size=B.MLP_PARAMS), dtype=torch.float32, device=dev)
        rows = torch.tensor(rng.permutation(9000)[:n_rows], dtype=torch.int32, device=dev)
        g_ref = torch.empty(B.MLP_PARAMS, dtype=torch.float32, device=dev)
        l_ref = torch.empty(1, dtype=torch.float64, device=dev)
        g_new = torch.full((B.MLP_PARAMS,), float("nan"), dtype=torch.float32, device=dev)
        l_new = torch.full((1,), float("nan"), dtype=torch.float64, device=dev)
        assert _call(lib.mlp_loss_grad, p, x, t, rows, n_rows, g_ref, l_ref) == 0
        # arm the library's allocation hook: any allocation on this path would
        # now fail with SHP_ENOMEM, so success shows that the call allocates nothing
        assert lib.shp_fail_next_allocations(1000) == 0
        try:
            rc = _call(lib.mlp_loss_grad_noalloc, p, x, t, rows, n_rows, g_new, l_new)
        finally:
            assert lib.shp_fail_next_allocations(0) == 0
        assert rc == 0, lib.shp_last_error()
        torch.cuda.synchronize()
        # same kernels, same fixed-order reduction: the results agree to the
        # tolerance the other network tests use (they are in fact identical)
        torch.testing.assert_close(l_new, l_ref, rtol=1e-5, atol=0)
        g_ref_np, g_new_np = g_ref.cpu().numpy(), g_new.cpu().numpy()
        assert np.linalg.norm(g_new_np - g_ref_np) <= 1e-4 * np.linalg.norm(g_ref_np)


def test_noalloc_rejects_batches_beyond_its_scratch():
    lib = shp.load_library()
    dev = "cuda"
    x = torch.zeros((8193, B.MLP_IN), dtype=torch.float32, device=dev)
    t = torch.zeros(8193, dtype=torch.float32, device=dev)
    p = torch.zeros(B.MLP_PARAMS, dtype=torch.float32, device=dev)
    g = torch.empty(B.MLP_PARAMS, dtype=torch.float32, device=dev)
    loss = torch.empty(1, dtype=torch.float64, device=dev)
    assert _call(lib.mlp_loss_grad_noalloc, p, x, t, None, 8193, g, loss) == -4
    assert b"8192" in lib.shp_last_error()
