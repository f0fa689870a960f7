"""Degenerate and edge cases through the C ABI: grids of one or two cells per
axis (periodic images of a cell onto itself, ghosts deeper than the grid is
wide), zero steps, empty and invalid inputs, and single-cell eikonal problems."""
import ctypes

import numpy as np
import pytest

import inputs
import oracle
import paper_2104_08571_gb300 as R
from tests.gpu_util import LINF_EIK, LINF_F32, LINF_F64, assert_parity, gpu_euler, rel_l1

pytestmark = pytest.mark.gpu
MUSCL, RUS, FORCE = R.RIPPLE_MUSCL_HANCOCK_MINMOD, R.RIPPLE_RUSANOV1, R.RIPPLE_FORCE_SPLIT
PER, TRA = R.RIPPLE_BC_PERIODIC, R.RIPPLE_BC_TRANSMISSIVE


@pytest.fixture(scope="module")
def ctx():
    import torch
    assert torch.cuda.is_available()
    c = R.ripple_ctx_create(0)
    yield c
    R.ripple_ctx_destroy(c)


def _state(dims, seed):
    ndim = len(dims)
    r = inputs.uniform(seed, (ndim + 2) * int(np.prod(dims))).reshape((ndim + 2,) + tuple(reversed(dims)))
    return inputs.conserved(1.0 + 0.3 * r[0], [0.3 * (r[1 + d] - 0.5) for d in range(ndim)], 1.0 + 0.3 * r[ndim + 1])


@pytest.mark.parametrize("dims,scheme,bc", [((1, 1), RUS, PER), ((1, 1), RUS, TRA), ((2, 3), MUSCL, PER),
                                            ((1, 5), MUSCL, TRA), ((2, 2, 2), MUSCL, PER), ((1, 1, 3), RUS, TRA),
                                            ((1, 4), FORCE, PER), ((3, 1, 2), FORCE, TRA)])
@pytest.mark.parametrize("dtype", [R.RIPPLE_F64, R.RIPPLE_F32])
def test_tiny_grids_match_oracle(ctx, dims, scheme, bc, dtype):
    U0 = _state(dims, seed=sum(dims))
    if dtype == R.RIPPLE_F32:
        U0 = U0.astype(np.float32).astype(np.float64)
    oscheme = {RUS: oracle.RUSANOV1, MUSCL: oracle.MUSCL_HANCOCK, FORCE: oracle.FORCE_SPLIT}[scheme]
    got, _ = gpu_euler(ctx, U0, 7, dtype=dtype, scheme=scheme, bc=bc)
    ref, _ = oracle.euler_run(U0, 7, scheme=oscheme, bc=bc)
    assert_parity(got, ref, *((1e-12, LINF_F64) if dtype == R.RIPPLE_F64 else (2e-5, LINF_F32)))


def test_zero_steps_change_nothing(ctx):
    U0 = _state((13, 9), seed=3)
    got, st = gpu_euler(ctx, U0, 0)
    assert np.array_equal(got, U0)
    assert st["steps_done"] == 0 and st["t"] == 0.0


def test_empty_and_invalid_fields_are_refused(ctx):
    lib = R.load()
    out = ctypes.c_void_p()
    for dims in ((0, 4), (4, 0), (3, 3, 0)):
        d = (ctypes.c_int64 * len(dims))(*dims)
        assert lib.ripple_field_create(ctx, len(dims), d, len(dims) + 2, R.RIPPLE_SOA, 1, R.RIPPLE_F32,
                                       ctypes.byref(out)) == R.RIPPLE_ERR_INVALID
    d = (ctypes.c_int64 * 2)(8, 8)
    assert lib.ripple_field_create(ctx, 4, d, 6, R.RIPPLE_SOA, 1, R.RIPPLE_F32, ctypes.byref(out)) == \
        R.RIPPLE_ERR_INVALID  # ndim 4
    assert lib.ripple_field_create(ctx, 2, d, 4, 7, 1, R.RIPPLE_F32, ctypes.byref(out)) == R.RIPPLE_ERR_INVALID
    # maximum sizes: more than 2^32 padded cells per buffer is refused before any
    # allocation (a 2^20-cube would overflow a 64-bit byte count)
    for dims in ((1 << 20, 1 << 20), (1 << 20, 1 << 20, 1 << 20), (70000, 70000)):
        d = (ctypes.c_int64 * len(dims))(*dims)
        assert lib.ripple_field_create(ctx, len(dims), d, len(dims) + 2, R.RIPPLE_SOA, 2, R.RIPPLE_F32,
                                       ctypes.byref(out)) == R.RIPPLE_ERR_INVALID
    d = (ctypes.c_int64 * 2)(8, 8)
    # a periodic axis narrower than the halo cannot be padded
    f = R.ripple_field_create(ctx, (1, 6), 4, R.RIPPLE_SOA, 2, R.RIPPLE_F64)
    try:
        R.ripple_field_upload(f, _state((1, 6), 1))
        with pytest.raises(R.RippleError) as ei:
            R.ripple_fv_step(f, R.make_fv_params([1.0, 1.0 / 6], scheme=MUSCL, bc=PER), 1)
        assert ei.value.status == R.RIPPLE_ERR_INVALID
    finally:
        R.ripple_field_destroy(f)


def test_single_cell_and_all_source_eikonal(ctx):
    # a 1 x 1 grid whose only cell is the source; a strip of sources
    for dims, src in (((1, 1), [(0, 0)]), ((5, 1), [(i, 0) for i in range(5)])):
        s = np.ones(tuple(reversed(dims)), dtype=np.float32)
        fs = R.ripple_field_create(ctx, dims, 1, R.RIPPLE_SOA, 0, R.RIPPLE_F32)
        ft = R.ripple_field_create(ctx, dims, 1, R.RIPPLE_SOA, 1, R.RIPPLE_F32)
        try:
            R.ripple_field_upload(fs, s)
            R.ripple_eikonal_solve(fs, ft, src, 1.0, 1e-6)
            T = R.ripple_field_download(ft).reshape(s.shape)
            assert np.all(T == 0.0)
        finally:
            R.ripple_field_destroy(fs)
            R.ripple_field_destroy(ft)
    # a source on the far corner of a long strip: T = k h exactly
    dims = (1, 300)
    s = np.ones((300, 1), dtype=np.float32)
    fs = R.ripple_field_create(ctx, dims, 1, R.RIPPLE_SOA, 0, R.RIPPLE_F32)
    ft = R.ripple_field_create(ctx, dims, 1, R.RIPPLE_SOA, 1, R.RIPPLE_F32)
    try:
        R.ripple_field_upload(fs, s)
        R.ripple_eikonal_solve(fs, ft, [(0, 299)], 0.5, 1e-7)
        T = R.ripple_field_download(ft).reshape(300)
        assert np.array_equal(T, 0.5 * np.arange(299, -1, -1, dtype=np.float32))
    finally:
        R.ripple_field_destroy(fs)
        R.ripple_field_destroy(ft)


def test_empty_batch_submit(ctx):
    assert R.ripple_batch_submit(ctx, []) == []
