"""Failure detection with faults made on the host (RIPPLE_FAULT): an allocation,
an admission or an upload that fails as if its CUDA call had failed.  Each
failure surfaces as a status, frees what was reserved, and leaves the context
and the batch runtime working for the requests that follow.  No GPU fault,
trap or hang is ever provoked."""
import os

import numpy as np
import pytest

import inputs
import oracle
import paper_2104_08571_gb300 as R
from tests.gpu_util import LINF_EIK, LINF_F32, LINF_F64, assert_parity, rel_l1

pytestmark = pytest.mark.gpu


class fault:
    def __init__(self, steps):
        self.steps = steps

    def __enter__(self):
        os.environ["RIPPLE_FAULT"] = self.steps

    def __exit__(self, *exc):
        os.environ.pop("RIPPLE_FAULT", None)


@pytest.fixture()
def ctx():
    import torch
    assert torch.cuda.is_available()
    c = R.ripple_ctx_create(0, 1 << 30)
    yield c
    R.ripple_ctx_destroy(c)


def test_allocation_failure_in_field_create_and_step(ctx):
    base = R.ripple_ctx_mem_used(ctx)
    with fault("alloc"):
        with pytest.raises(R.RippleError) as ei:
            R.ripple_field_create(ctx, (40, 30), 4, R.RIPPLE_SOA, 1, R.RIPPLE_F64)
        assert ei.value.status == R.RIPPLE_ERR_OOM
    assert R.ripple_ctx_mem_used(ctx) == base  # nothing reserved is left behind
    U0 = inputs.euler2d_sine(40, ny=30)
    f = R.ripple_field_create(ctx, (40, 30), 4, R.RIPPLE_SOA, 1, R.RIPPLE_F64)
    try:
        R.ripple_field_upload(f, U0)
        prm = R.make_fv_params([1 / 40, 1 / 30])
        before = R.ripple_ctx_mem_used(ctx)
        with fault("alloc"):  # the step's second buffer cannot be had
            with pytest.raises(R.RippleError) as ei:
                R.ripple_fv_step(f, prm, 3)
            assert ei.value.status == R.RIPPLE_ERR_OOM
        assert R.ripple_ctx_mem_used(ctx) == before  # the failed allocation left nothing reserved
        R.ripple_fv_step(f, prm, 3)  # recovers once the allocation succeeds
        ref, _ = oracle.euler_run(U0, 3, dx=[1 / 40, 1 / 30])
        assert_parity(R.ripple_field_download(f), ref, 1e-12, LINF_F64)
    finally:
        R.ripple_field_destroy(f)


def _euler(n, steps=5):
    U = inputs.euler2d_sine(n, amp=0.1).astype(np.float32)
    return R.euler_request(U, steps, [1.0 / n, 1.0 / n])


@pytest.mark.parametrize("async_queue", [False, True])
@pytest.mark.parametrize("step,status", [("admit", R.RIPPLE_ERR_OOM), ("upload", R.RIPPLE_ERR_CUDA),
                                         ("alloc", R.RIPPLE_ERR_OOM)])
def test_batch_request_failure_then_recovery(ctx, step, status, async_queue):
    R.ripple_batch_configure(ctx, async_queue=async_queue)
    good = _euler(48)
    tickets = R.ripple_batch_submit(ctx, [good])
    assert R.ripple_wait(ctx, tickets[0], 60000)["status"] == R.RIPPLE_OK
    base = R.ripple_ctx_mem_used(ctx)
    with fault(step):
        bad = [_euler(40), _euler(56)]
        infos = [R.ripple_wait(ctx, t, 60000) for t in R.ripple_batch_submit(ctx, bad)]
    assert all(i["status"] == status for i in infos), infos
    assert R.ripple_ctx_mem_used(ctx) == base  # their memory came back
    again = _euler(48)
    tickets = R.ripple_batch_submit(ctx, [again])
    assert R.ripple_wait(ctx, tickets[0], 60000)["status"] == R.RIPPLE_OK
    assert np.array_equal(again["output"], good["output"])  # the same result as before the failures
    st = R.ripple_batch_get_stats(ctx)
    assert st["failed"] >= 2
