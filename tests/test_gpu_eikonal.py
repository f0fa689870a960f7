"""GPU parity of the FIM eikonal solver against the FP64 Fast Marching oracle.

The GPU iteration converges to the Godunov fixed point that Fast Marching
computes directly; the bar is 1e-4 relative L1 in FP32 (over all cells, T
finite everywhere) and 1e-9 in FP64 with a tight stopping tolerance.
"""
import numpy as np
import pytest

import inputs
import oracle
import paper_2104_08571_gb300 as R
from tests.gpu_util import LINF_EIK, LINF_EIK_F64

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import torch
    assert torch.cuda.is_available()
    c = R.ripple_ctx_create(0)
    R.use_torch_allocator(c, 0)
    yield c
    R.ripple_ctx_destroy(c)


def gpu_eikonal(ctx, s, sources, h, dtype=R.RIPPLE_F32, tol=1e-6, halo=1, max_iters=0):
    dims = tuple(reversed(s.shape))
    npdt = np.float32 if dtype == R.RIPPLE_F32 else np.float64
    fs = R.ripple_field_create(ctx, dims, 1, R.RIPPLE_SOA, 0, dtype)
    ft = R.ripple_field_create(ctx, dims, 1, R.RIPPLE_SOA, halo, dtype)
    try:
        R.ripple_field_upload(fs, np.ascontiguousarray(s, dtype=npdt))
        st = R.ripple_eikonal_solve(fs, ft, sources, h, tol, max_iters)
        T = R.ripple_field_download(ft)[0]
    finally:
        R.ripple_field_destroy(fs)
        R.ripple_field_destroy(ft)
    return T, st


def rel_l1(a, b):
    return float(np.abs(a.astype(np.float64) - b).sum() / np.abs(b).sum())


def max_rel(a, b):
    return float(np.abs(a.astype(np.float64) - b).max() / np.abs(b).max())


def check(T, ref, l1, linf):
    """Relative L1 over all cells and the element-wise bound beside it."""
    e1, ei = rel_l1(T, ref), max_rel(T, ref)
    print(f"parity: rel L1 {e1:.3e} (bar {l1:.0e}), max {ei:.3e} (bar {linf:.0e})")
    assert e1 <= l1 and ei <= linf, f"rel L1 {e1:.3e} (bar {l1:.0e}), max {ei:.3e} (bar {linf:.0e})"


@pytest.mark.parametrize("dims,seed", [((256, 256), 1), ((100, 70), 2), ((33, 200), 3)])
def test_fp32_2d_vs_fmm(ctx, dims, seed):
    s = inputs.eikonal_slowness(dims, seed=seed).astype(np.float32)
    src = inputs.eikonal_sources(dims, seed=seed)
    h = 1.0 / max(dims)
    T, st = gpu_eikonal(ctx, s, src, h)
    ref = oracle.eikonal_fmm(s.astype(np.float64), h, src)
    assert np.all(np.isfinite(T))
    check(T, ref, 1e-4, LINF_EIK)
    for c in src:
        assert T[tuple(reversed(c))] == 0.0
    assert st["iterations"] > 0 and st["tile_visits"] >= 1


@pytest.mark.parametrize("dims,seed", [((48, 40, 36), 4), ((19, 23, 9), 5)])
def test_fp32_3d_vs_fmm(ctx, dims, seed):
    s = inputs.eikonal_slowness(dims, seed=seed).astype(np.float32)
    src = inputs.eikonal_sources(dims, seed=seed)
    h = 1.0 / max(dims)
    T, _ = gpu_eikonal(ctx, s, src, h)
    ref = oracle.eikonal_fmm(s.astype(np.float64), h, src)
    check(T, ref, 1e-4, LINF_EIK)


@pytest.mark.parametrize("dims", [(80, 64), (24, 20, 18)])
def test_fp64_tight_tolerance(ctx, dims):
    s = inputs.eikonal_slowness(dims, seed=6)
    src = inputs.eikonal_sources(dims, seed=6)
    h = 1.0 / max(dims)
    T, _ = gpu_eikonal(ctx, s, src, h, dtype=R.RIPPLE_F64, tol=1e-13)
    ref = oracle.eikonal_fmm(s, h, src)
    check(T, ref, 1e-9, LINF_EIK_F64)


def test_unit_speed_axis_exact_fp64(ctx):
    n = 65
    h = 1.0 / 64.0
    s = np.ones((n, n))
    c = n // 2
    T, _ = gpu_eikonal(ctx, s, [(c, c)], h, dtype=R.RIPPLE_F64, tol=1e-14)
    k = np.abs(np.arange(n) - c) * h
    assert np.array_equal(T[c, :], k)
    assert np.array_equal(T[:, c], k)


def test_deterministic(ctx):
    dims = (150, 120)
    s = inputs.eikonal_slowness(dims, seed=7).astype(np.float32)
    src = inputs.eikonal_sources(dims, seed=7, count=3)
    a, sa = gpu_eikonal(ctx, s, src, 1.0 / 150)
    b, sb = gpu_eikonal(ctx, s, src, 1.0 / 150)
    assert np.array_equal(a, b) and sa == sb


def test_iteration_cap_reports_timeout(ctx):
    dims = (128, 128)
    s = np.ones(dims, dtype=np.float32)
    with pytest.raises(R.RippleError) as ei:
        gpu_eikonal(ctx, s, [(0, 0)], 1.0 / 128, max_iters=2)
    assert ei.value.status == R.RIPPLE_ERR_TIMEOUT


def test_grid_barrier_timeout_reports_its_own_cause(ctx, monkeypatch):
    """A grid-barrier wait that runs out (here: the host lowers its poll bound
    to zero, so every CTA but the last to arrive gives up at once) ends the
    solve with TIMEOUT and a message naming the barrier, not the iteration
    cap; the context keeps working for the next solve."""
    dims = (256, 256)
    s = np.ones(dims, dtype=np.float32)
    monkeypatch.setenv("RIPPLE_GRID_SPIN_LIMIT", "0")
    with pytest.raises(R.RippleError) as ei:
        gpu_eikonal(ctx, s, [(3, 5)], 1.0 / 256)
    assert ei.value.status == R.RIPPLE_ERR_TIMEOUT
    assert "barrier" in str(ei.value) and "max_iters" not in str(ei.value)
    monkeypatch.delenv("RIPPLE_GRID_SPIN_LIMIT")
    T, _ = gpu_eikonal(ctx, s, [(3, 5)], 1.0 / 256)
    ref = oracle.eikonal_fmm(s.astype(np.float64), 1.0 / 256, [(3, 5)])
    check(T, ref, 1e-4, LINF_EIK)


def test_config2_full_size_2d(ctx):
    """2048^2 FP32, seeded slowness and 1-4 sources, tol 1e-6."""
    dims = (2048, 2048)
    s = inputs.eikonal_slowness(dims, seed=1).astype(np.float32)
    src = inputs.eikonal_sources(dims, seed=1)
    h = 1.0 / 2048
    T, st = gpu_eikonal(ctx, s, src, h)
    ref = oracle.eikonal_fmm(s.astype(np.float64), h, src)
    check(T, ref, 1e-4, LINF_EIK)


def test_config2_full_size_3d(ctx):
    dims = (192, 192, 192)
    s = inputs.eikonal_slowness(dims, seed=1).astype(np.float32)
    src = inputs.eikonal_sources(dims, seed=1)
    h = 1.0 / 192
    T, st = gpu_eikonal(ctx, s, src, h)
    ref = oracle.eikonal_fmm(s.astype(np.float64), h, src)
    check(T, ref, 1e-4, LINF_EIK)
