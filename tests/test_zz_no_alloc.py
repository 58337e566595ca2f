"""The allocation-free inner product, enp_inner_product_noalloc.

It serves callers that cannot call cudaMalloc (an application that owns all
device memory through its own pool, or a latency-critical loop): its partial
sums live in a fixed static device array instead of handle-allocated scratch.
Checked through the C ABI against the allocating entry point,
enp_inner_product, on two calls in a row with different sizes (the shared
array still holds the first call's partials when the second starts). Both
run the same reduction kernels on the same grid, so the results must agree
bit for bit. This file is collected last.
"""
import ctypes

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def test_noalloc_inner_product_matches_allocating_entry_point_on_two_calls():
    import torch
    import paper_2112_09271_gb300 as enp
    enp.build()
    lib = enp.load()
    stream = torch.cuda.current_stream()
    calls = [("channel_n2", 3, 11), ("cube_n3_p2", 1, 21)]  # larger first, then smaller
    for cfg, batch, seed in calls:
        P = W.config(cfg)
        op = enp.Operator(P, batch=batch, stream=stream)
        xs = [W.random_vector(P, seed + b) for b in range(batch)]
        ys = [W.random_vector(P, seed + 100 + b) for b in range(batch)]
        x = torch.tensor(np.concatenate(xs), device="cuda")
        y = torch.tensor(np.concatenate(ys), device="cuda")
        ref = op.inner_product(x, y)  # allocating entry point (host result)
        out = torch.full((batch,), np.nan, dtype=torch.float64, device="cuda")
        st = lib.enp_inner_product_noalloc(_ptr(x), _ptr(y), ctypes.c_longlong(P.n_dof), batch,
                                           _ptr(out), ctypes.c_void_p(stream.cuda_stream))
        assert st == enp.ENP_OK
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        for b in range(batch):
            assert got[b] == ref[b], (cfg, b, got[b], ref[b])


def test_noalloc_inner_product_rejects_batches_beyond_its_array():
    import torch
    import paper_2112_09271_gb300 as enp
    enp.build()
    lib = enp.load()
    x = torch.zeros(8, dtype=torch.float64, device="cuda")
    out = torch.zeros(enp.NOALLOC_MAX_BATCH + 1, dtype=torch.float64, device="cuda")
    st = lib.enp_inner_product_noalloc(_ptr(x), _ptr(x), ctypes.c_longlong(1),
                                       enp.NOALLOC_MAX_BATCH + 1, _ptr(out), None)
    assert st == enp.ENP_ERR_INVALID_ARG
