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
