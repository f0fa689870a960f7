"""Helpers for the GPU parity tests (call the library through its C ABI)."""
import numpy as np

import paper_2104_08571_gb300 as R


def rel_l1(got, ref):
    """Max over components of sum|got - ref| / sum|ref| (interior cells)."""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    g = got.reshape(got.shape[0], -1)
    r = ref.reshape(ref.shape[0], -1)
    out = 0.0
    for m in range(g.shape[0]):
        den = np.abs(r[m]).sum()
        num = np.abs(g[m] - r[m]).sum()
        if den == 0.0:
            den = max(np.abs(r).sum() / r.size * r.shape[1], 1e-300)
        out = max(out, num / den)
    return out


def max_rel(got, ref):
    """Max over components of max|got - ref| / max|ref|: an element-wise bound
    beside the relative L1, so that one wrong cell, a bad tile edge or a
    missed ghost layer fails even when the mean error stays small."""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    g = got.reshape(got.shape[0], -1)
    r = ref.reshape(ref.shape[0], -1)
    out = 0.0
    for m in range(g.shape[0]):
        den = np.abs(r[m]).max()
        if den == 0.0:
            den = max(np.abs(r).max(), 1e-300)
        out = max(out, float(np.abs(g[m] - r[m]).max() / den))
    return out


# Element-wise bounds (max|gpu - oracle| / max|oracle| per component), from the
# error budget of each precision: u = unit roundoff, a cell update rounds a few
# hundred operations (a few u after cancellation: measured below 1e-6 per FP32
# step), the scheme is stable (errors accumulate at most linearly), so 100
# steps stay under 100 x 8 u.
#   FP64: 100 x 8 x 1.1e-16 = 9e-14  -> bar 1e-12
#   FP32: 100 x 8 x 6.0e-8  = 4.8e-5 -> bar 5e-5
LINF_F64 = 1e-12
LINF_F32 = 5e-5
# Eikonal travel times (max|T - T_fmm| / max T_fmm): a Godunov update rounds
# to about u, and errors accumulate along a characteristic path of up to 2048
# cells (2048 u = 1.2e-4 in FP32), plus the FIM stopping tolerance (1e-6
# absolute per sweep); in FP64 with a tight tolerance 2048 u = 2.3e-13.
LINF_EIK = 2e-4
LINF_EIK_F64 = 1e-11


def assert_parity(got, ref, l1, linf):
    """Relative L1 (the workload's metric) and the element-wise bound together."""
    e1 = rel_l1(got, ref)
    ei = max_rel(got, ref)
    print(f"parity: rel L1 {e1:.3e} (bar {l1:.0e}), max {ei:.3e} (bar {linf:.0e})")
    assert e1 <= l1 and ei <= linf, f"rel L1 {e1:.3e} (bar {l1:.0e}), max {ei:.3e} (bar {linf:.0e})"
    return e1, ei


def gpu_euler(ctx, U0, nsteps, *, dtype=R.RIPPLE_F64, layout=R.RIPPLE_SOA, scheme=R.RIPPLE_RUSANOV1,
              bc=R.RIPPLE_BC_PERIODIC, dx=None, halo=None, gamma=1.4, cfl=0.4, variant=None, chunks=None):
    """Run nsteps on the GPU from the component-major state U0; returns (U, stats)."""
    ndim = U0.ndim - 1
    dims = tuple(reversed(U0.shape[1:]))
    if dx is None:
        dx = [1.0 / d for d in dims]
    if halo is None:
        halo = 2 if scheme == R.RIPPLE_MUSCL_HANCOCK_MINMOD else 1
    npdt = np.float32 if dtype == R.RIPPLE_F32 else np.float64
    f = R.ripple_field_create(ctx, dims, ndim + 2, layout, halo, dtype)
    try:
        if variant is not None or chunks is not None:
            R.ripple_field_set_sweep(f, -1 if variant is None else variant, 0 if chunks is None else chunks)
        host = np.ascontiguousarray(U0, dtype=npdt)
        if layout == R.RIPPLE_AOS:
            R.ripple_field_upload(f, np.ascontiguousarray(np.moveaxis(host, 0, -1)), R.RIPPLE_AOS)
        else:
            R.ripple_field_upload(f, host, R.RIPPLE_SOA)
        stats = R.ripple_fv_step(f, R.make_fv_params(dx, gamma=gamma, cfl=cfl, scheme=scheme, bc=bc), nsteps)
        out = R.ripple_field_download(f, R.RIPPLE_SOA)
    finally:
        R.ripple_field_destroy(f)
    return out, stats
