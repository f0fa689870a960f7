"""ripple_totals_noalloc: conserved totals for callers that cannot allocate.

A caller that has given all device memory to its own pool, or that must not
trigger the device synchronisation of cudaMalloc/cudaFree inside a
latency-bound loop, can still get the FP64 compensated totals of a state it
owns: this entry point keeps its scratch in a fixed array of the library image.
The test calls it through the C ABI on caller-owned CUDA tensors, twice in a
row on two different states, and compares each result with the totals that
the existing entry point (the statistics of ripple_fv_step) reports for the
same state.  This file is collected last on purpose.
"""
import math

import numpy as np
import pytest

import inputs
import paper_2104_08571_gb300 as R

pytestmark = pytest.mark.gpu


def _field_totals(ctx, U, layout, dtype):
    ndim = U.ndim - 1
    dims = tuple(reversed(U.shape[1:]))
    f = R.ripple_field_create(ctx, dims, ndim + 2, layout, 1, dtype)
    try:
        host = U if layout == R.RIPPLE_SOA else np.ascontiguousarray(np.moveaxis(U, 0, -1))
        R.ripple_field_upload(f, host, layout)
        st = R.ripple_fv_step(f, R.make_fv_params([1.0 / d for d in dims]), 0)
    finally:
        R.ripple_field_destroy(f)
    return np.array(st["totals"][: ndim + 2])


def test_noalloc_totals_match_existing_entry_point_two_calls():
    import torch

    assert torch.cuda.is_available()
    torch.cuda.set_device(0)
    ctx = R.ripple_ctx_create(0)
    try:
        cases = [
            (inputs.euler2d_sine(128), R.RIPPLE_SOA, R.RIPPLE_F64, np.float64),
            (inputs.euler3d_blast(48, seed=3, dims=(48, 40, 36)).astype(np.float32), R.RIPPLE_AOS, R.RIPPLE_F32,
             np.float32),
        ]
        for U, layout, dtype, npdt in cases:  # two calls in a row
            U = U.astype(npdt)
            ndim = U.ndim - 1
            dims = tuple(reversed(U.shape[1:]))
            ref = _field_totals(ctx, U, layout, dtype)
            host = U if layout == R.RIPPLE_SOA else np.ascontiguousarray(np.moveaxis(U, 0, -1))
            state = torch.from_numpy(np.ascontiguousarray(host)).cuda()
            out = torch.full((ndim + 2,), float("nan"), dtype=torch.float64, device="cuda")
            R.ripple_totals_noalloc(state, dims, ndim + 2, layout, dtype, out)
            torch.cuda.synchronize()
            got = out.cpu().numpy()
            for m in range(ndim + 2):
                scale = float(np.abs(U[m].astype(np.float64)).sum())
                exact = math.fsum(U[m].astype(np.float64).ravel())
                assert abs(got[m] - ref[m]) <= 1e-12 * scale, (m, got[m], ref[m])
                assert abs(got[m] - exact) <= 1e-12 * scale
    finally:
        R.ripple_ctx_destroy(ctx)


def test_noalloc_rejects_arrays_beyond_its_scratch():
    import torch

    state = torch.zeros(4, dtype=torch.float32, device="cuda")
    out = torch.zeros(5, dtype=torch.float64, device="cuda")
    with pytest.raises(R.RippleError) as ei:
        R.ripple_totals_noalloc(state, (4096, 4096, 3), 5, R.RIPPLE_SOA, R.RIPPLE_F32, out)
    assert ei.value.status == R.RIPPLE_ERR_INVALID
    assert "33554432" in R.ripple_last_error()
