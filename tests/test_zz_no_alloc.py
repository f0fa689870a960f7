"""ripple_totals_noalloc: conserved totals for callers that cannot allocate.

A caller that has given all device memory to its own pool, or that must not
trigger the device synchronisation of cudaMalloc/cudaFree inside a
latency-bound loop, can still get the FP64 compensated totals of a state it
owns: this entry point keeps its scratch in a fixed array of the library image.
The test calls it through the C ABI on caller-owned CUDA tensors, twice in a
row on two different states, and compares each result with the totals that
the existing entry point (the statistics of ripple_fv_step) reports for the
same state.  It also checks that repeated calls leave the device's free memory
unchanged, and that arguments the entry point cannot use are refused before
any launch.

The file name sorts after every other test file, so a run that stops at the
first failure has already run all other tests when it reaches this one; the
tests here depend on nothing that earlier files set up and pass on their own
in a fresh process.
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


def test_noalloc_allocates_nothing_on_repeated_calls():
    """After one warm-up call (which may load the kernels and look up the
    scratch address), 50 more calls change the device's free memory by nothing."""
    import torch

    torch.cuda.set_device(0)
    U = inputs.euler3d_blast(64, seed=5).astype(np.float32)
    state = torch.from_numpy(np.ascontiguousarray(U)).cuda()
    out = torch.zeros(5, dtype=torch.float64, device="cuda")
    R.ripple_totals_noalloc(state, (64, 64, 64), 5, R.RIPPLE_SOA, R.RIPPLE_F32, out)
    torch.cuda.synchronize()
    first = out.clone()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(50):
        R.ripple_totals_noalloc(state, (64, 64, 64), 5, R.RIPPLE_SOA, R.RIPPLE_F32, out)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert torch.equal(out, first)


def test_noalloc_rejects_arrays_beyond_its_scratch():
    """One cell past the limit of the fixed scratch is refused by the library
    itself.  The state tensor really holds the cells it claims (134 MB), so a
    regression of the size check would stay inside the allocation."""
    import torch

    n = 33554432 + 1
    state = torch.zeros(n, dtype=torch.float32, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(R.RippleError) as ei:
        R.ripple_totals_noalloc(state, (n,), 1, R.RIPPLE_SOA, R.RIPPLE_F32, out)
    assert ei.value.status == R.RIPPLE_ERR_INVALID
    assert "33554432" in R.ripple_last_error()


def test_noalloc_binding_refuses_unusable_tensors():
    """Host tensors, a wrong dtype or tensors shorter than the described array
    are refused by the binding before the library is called."""
    import torch

    good = torch.zeros(4 * 4 * 5, dtype=torch.float32, device="cuda")
    out = torch.zeros(5, dtype=torch.float64, device="cuda")
    bad_cases = [
        (good.cpu(), out),
        (good, out.cpu()),
        (good.double(), out),
        (good[:-1], out),
        (good, out[:4]),
        (good, out.float()),
    ]
    for st, ot in bad_cases:
        with pytest.raises(ValueError):
            R.ripple_totals_noalloc(st, (4, 4), 5, R.RIPPLE_SOA, R.RIPPLE_F32, ot)
