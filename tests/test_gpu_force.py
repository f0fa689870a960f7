"""GPU parity of the paper's own Euler solver -- the dimensionally split step
with the FORCE face flux (Listing euler_graph, Section 7.3) -- against the FP64
oracle through the C ABI: FP64 <= 1e-12 and FP32 <= 2e-5 relative L1, on
grids that span several tiles with ragged tails, both layouts and both
boundary conditions; bitwise uniform state, AoS == SoA and axis symmetry."""
import math

import numpy as np
import pytest

import inputs
import oracle
import paper_2104_08571_gb300 as R
from tests.gpu_util import LINF_EIK, LINF_F32, LINF_F64, assert_parity, gpu_euler, rel_l1

pytestmark = pytest.mark.gpu
FORCE = R.RIPPLE_FORCE_SPLIT


@pytest.fixture(scope="module")
def ctx():
    import torch
    assert torch.cuda.is_available()
    c = R.ripple_ctx_create(0)
    R.use_torch_allocator(c, 0)
    yield c
    R.ripple_ctx_destroy(c)


def _random_state(dims, seed, amp=0.4):
    ndim = len(dims)
    shape = tuple(reversed(dims))
    r = inputs.uniform(seed, (ndim + 2) * int(np.prod(dims))).reshape((ndim + 2,) + shape)
    return inputs.conserved(1.0 + amp * r[0], [amp * (r[1 + d] - 0.5) for d in range(ndim)], 1.0 + amp * r[ndim + 1])


def test_force_split_config0_fp64(ctx):
    """The 2D FP64 workload (128^2 periodic sine density, CFL 0.4, 100 steps) with the paper's solver."""
    U0 = inputs.euler2d_sine(128)
    got, st = gpu_euler(ctx, U0, 100, scheme=FORCE)
    ref, info = oracle.euler_run(U0, 100, scheme=oracle.FORCE_SPLIT)
    assert_parity(got, ref, 1e-12, LINF_F64)
    assert st["t"] == pytest.approx(info["t"], rel=1e-13)
    for m in range(4):
        exact = math.fsum(ref[m].ravel())
        assert abs(st["totals"][m] - exact) <= 1e-12 * max(abs(exact), np.abs(ref[m]).sum())


@pytest.mark.parametrize("dims", [(37, 23), (64, 9), (19, 13, 11), (36, 10, 40)])
@pytest.mark.parametrize("dtype", [R.RIPPLE_F64, R.RIPPLE_F32])
@pytest.mark.parametrize("bc", [R.RIPPLE_BC_PERIODIC, R.RIPPLE_BC_TRANSMISSIVE])
@pytest.mark.parametrize("layout", [R.RIPPLE_SOA, R.RIPPLE_AOS])
def test_force_split_parity(ctx, dims, dtype, bc, layout):
    U0 = _random_state(dims, seed=len(dims) * 100 + dims[0])
    if dtype == R.RIPPLE_F32:
        U0 = U0.astype(np.float32).astype(np.float64)
    steps = 20
    got, _ = gpu_euler(ctx, U0, steps, dtype=dtype, layout=layout, scheme=FORCE, bc=bc)
    ref, _ = oracle.euler_run(U0, steps, scheme=oracle.FORCE_SPLIT, bc=bc)
    tol = 1e-12 if dtype == R.RIPPLE_F64 else 2e-5
    assert_parity(got, ref, tol, LINF_F64 if tol < 1e-9 else LINF_F32)


_LONG_WALK_REF = {}


@pytest.mark.parametrize("layout", [R.RIPPLE_SOA, R.RIPPLE_AOS])
@pytest.mark.parametrize("bc", [R.RIPPLE_BC_PERIODIC, R.RIPPLE_BC_TRANSMISSIVE])
def test_force_split_fp32_2d_long_walks(ctx, layout, bc):
    """2D FP32 split sweeps run on strip walks: on a 2000 x 1500 grid a walk
    spans several 64-cell chunks (faces carried from chunk to chunk), rows and
    strips are cut into several walks, and the last chunk and segment are
    ragged."""
    dims = (2000, 1500)
    U0 = _random_state(dims, seed=11, amp=0.3).astype(np.float32).astype(np.float64)
    if bc not in _LONG_WALK_REF:
        _LONG_WALK_REF[bc] = oracle.euler_run(U0, 3, scheme=oracle.FORCE_SPLIT, bc=bc)
    ref, info = _LONG_WALK_REF[bc]
    got, st = gpu_euler(ctx, U0, 3, dtype=R.RIPPLE_F32, layout=layout, scheme=FORCE, bc=bc)
    assert_parity(got, ref, 2e-5, LINF_F32)
    assert st["t"] == pytest.approx(info["t"], rel=1e-5)


_LONG_WALK_REF_3D = {}


@pytest.mark.parametrize("layout", [R.RIPPLE_SOA, R.RIPPLE_AOS])
@pytest.mark.parametrize("bc", [R.RIPPLE_BC_PERIODIC, R.RIPPLE_BC_TRANSMISSIVE])
def test_force_split_fp32_3d_walks(ctx, layout, bc):
    """3D FP32 split sweeps on strip walks: x walks over every (y, z) row with a
    ragged last chunk (150 = 64 + 64 + 22), y walks through the strips of every
    z plane and z walks through those of every y row, cut into several
    segments with a ragged last one; the whole field against the oracle, and
    against the tiled pair kernel's split sweeps."""
    dims = (150, 70, 61)
    U0 = _random_state(dims, seed=13, amp=0.3).astype(np.float32).astype(np.float64)
    if bc not in _LONG_WALK_REF_3D:
        _LONG_WALK_REF_3D[bc] = oracle.euler_run(U0, 4, scheme=oracle.FORCE_SPLIT, bc=bc)
    ref, info = _LONG_WALK_REF_3D[bc]
    got, st = gpu_euler(ctx, U0, 4, dtype=R.RIPPLE_F32, layout=layout, scheme=FORCE, bc=bc)
    assert_parity(got, ref, 2e-5, LINF_F32)
    assert st["t"] == pytest.approx(info["t"], rel=1e-5)
    tiled, _ = gpu_euler(ctx, U0, 4, dtype=R.RIPPLE_F32, layout=layout, scheme=FORCE, bc=bc, variant=2)
    assert_parity(got, tiled.astype(np.float64), 1e-6, 1e-5)


@pytest.mark.parametrize("ndim,dims", [(2, (40, 21)), (3, (18, 9, 12))])
@pytest.mark.parametrize("dtype", [R.RIPPLE_F64, R.RIPPLE_F32])
def test_force_split_uniform_state_bit_exact(ctx, ndim, dims, dtype):
    U0 = inputs.uniform_state(dims, 1.3, [0.7, -0.4, 0.25][:ndim], 0.9)
    if dtype == R.RIPPLE_F32:
        U0 = U0.astype(np.float32).astype(np.float64)
    for bc in (R.RIPPLE_BC_PERIODIC, R.RIPPLE_BC_TRANSMISSIVE):
        got, _ = gpu_euler(ctx, U0, 15, dtype=dtype, scheme=FORCE, bc=bc)
        assert np.array_equal(got.astype(np.float64), U0)


def test_force_split_aos_equals_soa_fp32_3d(ctx):
    U0 = _random_state((33, 17, 20), seed=5).astype(np.float32).astype(np.float64)
    a, _ = gpu_euler(ctx, U0, 12, dtype=R.RIPPLE_F32, layout=R.RIPPLE_SOA, scheme=FORCE)
    b, _ = gpu_euler(ctx, U0, 12, dtype=R.RIPPLE_F32, layout=R.RIPPLE_AOS, scheme=FORCE)
    assert np.array_equal(a, b)


def test_force_split_axis_symmetry_fp64(ctx):
    """A Sod tube along x and along y gives the same bits (the sweep across the
    uniform direction changes nothing)."""
    n, nt = 96, 3
    profiles = []
    for axis in (0, 1):
        U0 = inputs.sod(2, n, axis=axis, ntrans=nt)
        dx = [2.0 ** 100, 2.0 ** 100]
        dx[axis] = 1.0 / n
        # one tile shape for both orientations (the kernel is the same code either way)
        got, _ = gpu_euler(ctx, U0, 40, scheme=FORCE, bc=R.RIPPLE_BC_TRANSMISSIVE, dx=dx, variant=0)
        sl = [1, 1]
        sl[1 - axis] = slice(None)
        profiles.append(np.stack([got[0][tuple(sl)], got[1 + axis][tuple(sl)], got[3][tuple(sl)]]))
    diff = np.abs(profiles[0] - profiles[1]).max() / np.abs(profiles[0]).max()
    assert np.array_equal(profiles[0], profiles[1]), diff


def test_force_split_reports_negative_pressure(ctx):
    U0 = inputs.uniform_state((20, 20), 1.0, [0.0, 0.0], 1.0)
    U0[3, 10, 10] = -1.0
    with pytest.raises(R.RippleError) as ei:
        gpu_euler(ctx, U0, 2, scheme=FORCE)
    assert ei.value.status == R.RIPPLE_ERR_NUMERIC
