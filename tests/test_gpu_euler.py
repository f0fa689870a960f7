"""GPU parity of the Euler sweep against the FP64 CPU oracle, through the C ABI.

Tolerances (per-component relative L1 over interior cells):
  FP64 mode   <= 1e-12
  FP32 mode   <= 2e-5   (from FP32-rounded initial data, the oracle in FP64)
Bitwise: AoS == SoA, uniform state preserved, identical results on repeat.
"""
import math
import os

import numpy as np
import pytest

import inputs
import oracle
import paper_2104_08571_gb300 as R
from tests.gpu_util import LINF_EIK, LINF_F32, LINF_F64, assert_parity, gpu_euler, rel_l1

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import torch
    assert torch.cuda.is_available()
    c = R.ripple_ctx_create(0)
    R.use_torch_allocator(c, 0)
    yield c
    R.ripple_ctx_destroy(c)


MUSCL = R.RIPPLE_MUSCL_HANCOCK_MINMOD
RUS = R.RIPPLE_RUSANOV1
PER = R.RIPPLE_BC_PERIODIC
TRA = R.RIPPLE_BC_TRANSMISSIVE


def _random_state(dims, seed, amp=0.4):
    ndim = len(dims)
    shape = tuple(reversed(dims))
    r = inputs.uniform(seed, (ndim + 2) * int(np.prod(dims))).reshape((ndim + 2,) + shape)
    # smooth-ish positive state
    rho = 1.0 + amp * r[0]
    vel = [amp * (r[1 + d] - 0.5) for d in range(ndim)]
    p = 1.0 + amp * r[ndim + 1]
    return inputs.conserved(rho, vel, p)


def test_config0_fp64_parity(ctx):
    """2D FP64, 128^2 periodic sine density, Rusanov, CFL 0.4, 100 steps, SoA."""
    U0 = inputs.euler2d_sine(128)
    got, st = gpu_euler(ctx, U0, 100)
    ref, info = oracle.euler_run(U0, 100)
    assert_parity(got, ref, 1e-12, LINF_F64)
    assert st["t"] == pytest.approx(info["t"], rel=1e-13)
    assert st["dt_last"] == pytest.approx(info["dt_last"], rel=1e-13)
    # the device FP64 compensated totals match an exactly rounded host sum
    for m in range(4):
        exact = math.fsum(ref[m].ravel())
        assert abs(st["totals"][m] - exact) <= 1e-12 * max(abs(exact), np.abs(ref[m]).sum())


@pytest.mark.parametrize("dims", [(37, 23), (64, 9)])
@pytest.mark.parametrize("scheme", [RUS, MUSCL])
@pytest.mark.parametrize("bc", [PER, TRA])
@pytest.mark.parametrize("layout", [R.RIPPLE_SOA, R.RIPPLE_AOS])
def test_fp64_parity_2d_ragged(ctx, dims, scheme, bc, layout):
    U0 = _random_state(dims, seed=3)
    got, _ = gpu_euler(ctx, U0, 12, scheme=scheme, bc=bc, layout=layout)
    ref, _ = oracle.euler_run(U0, 12, scheme=scheme, bc=bc)
    assert_parity(got, ref, 1e-12, LINF_F64)


@pytest.mark.parametrize("dims", [(19, 13, 11), (36, 10, 40)])
@pytest.mark.parametrize("scheme", [RUS, MUSCL])
@pytest.mark.parametrize("bc", [PER, TRA])
def test_fp64_parity_3d_ragged(ctx, dims, scheme, bc):
    U0 = _random_state(dims, seed=5)
    got, _ = gpu_euler(ctx, U0, 6, scheme=scheme, bc=bc)
    ref, _ = oracle.euler_run(U0, 6, scheme=scheme, bc=bc)
    assert_parity(got, ref, 1e-12, LINF_F64)


def test_fp64_larger_halo(ctx):
    """A field with more ghost layers than the stencil needs (halo 3) gives the same result."""
    U0 = _random_state((33, 18, 12), seed=6)
    got, _ = gpu_euler(ctx, U0, 4, scheme=MUSCL, bc=TRA, halo=3)
    ref, _ = oracle.euler_run(U0, 4, scheme=MUSCL, bc=TRA)
    assert_parity(got, ref, 1e-12, LINF_F64)


def test_config0_fp32_parity(ctx):
    U0 = inputs.euler2d_sine(128).astype(np.float32)
    got, _ = gpu_euler(ctx, U0, 100, dtype=R.RIPPLE_F32)
    ref, _ = oracle.euler_run(U0.astype(np.float64), 100)
    assert_parity(got, ref, 2e-5, LINF_F32)


ROW, PAIR = 3, 2  # sweep variants of the FP32 3D MUSCL-Hancock step: row kernel (default), pair kernel


@pytest.mark.parametrize("variant", [ROW, PAIR])
@pytest.mark.parametrize("layout", [R.RIPPLE_SOA, R.RIPPLE_AOS])
def test_blast_fp32_parity(ctx, layout, variant):
    U0 = inputs.euler3d_blast(40, seed=1, dims=(40, 36, 28)).astype(np.float32)
    got, _ = gpu_euler(ctx, U0, 20, dtype=R.RIPPLE_F32, scheme=MUSCL, bc=TRA, layout=layout, variant=variant)
    ref, _ = oracle.euler_run(U0.astype(np.float64), 20, scheme=MUSCL, bc=TRA)
    assert_parity(got, ref, 2e-5, LINF_F32)


@pytest.mark.parametrize("variant", [ROW, PAIR])
@pytest.mark.parametrize("dims", [(37, 21, 70), (37, 21, 33), (130, 30, 9)])
@pytest.mark.parametrize("layout", [R.RIPPLE_SOA, R.RIPPLE_AOS])
def test_blast_fp32_parity_several_z_chunks(ctx, layout, dims, variant):
    # 70 planes: three z chunks per tile (32, 32, 6); 33: a last chunk of one
    # plane; ragged x and y tiles (130 x 30: three 64-wide row tiles, the last
    # two cells wide, and a 2-row last tile)
    nz = dims[2]
    U0 = inputs.euler3d_blast(nz, seed=2, dims=dims).astype(np.float32)
    got, _ = gpu_euler(ctx, U0, 6, dtype=R.RIPPLE_F32, scheme=MUSCL, bc=TRA, layout=layout, variant=variant)
    ref, _ = oracle.euler_run(U0.astype(np.float64), 6, scheme=MUSCL, bc=TRA)
    assert_parity(got, ref, 2e-5, LINF_F32)
    per, _ = gpu_euler(ctx, U0, 6, dtype=R.RIPPLE_F32, scheme=MUSCL, bc=PER, layout=layout, variant=variant)
    ref_p, _ = oracle.euler_run(U0.astype(np.float64), 6, scheme=MUSCL, bc=PER)
    assert_parity(per, ref_p, 2e-5, LINF_F32)


_FULL_RUNS = {}


def _oracle_blast_runs(dims, seed):
    """FP32-rounded blast state and the oracle's states after 50 and 100 steps
    (one 100-step run, split at step 50: each step takes dt from its own start
    state, so the split changes no bit).  Cached per grid."""
    key = (dims, seed)
    if key not in _FULL_RUNS:
        U0 = inputs.euler3d_blast(0, seed=seed, dims=dims).astype(np.float32)
        prev = oracle.threads_used()
        oracle.set_threads(os.cpu_count() or 1)
        try:
            U50, i50 = oracle.euler_run(U0.astype(np.float64), 50, scheme=MUSCL, bc=TRA)
            U100, i100 = oracle.euler_run(U50, 50, scheme=MUSCL, bc=TRA)
        finally:
            oracle.set_threads(prev)
        _FULL_RUNS[key] = (U0, {50: (U50, i50), 100: (U100, i100)})
    return _FULL_RUNS[key]


@pytest.mark.parametrize("dims", [(72, 40, 70), (96, 96, 96)])
@pytest.mark.parametrize("layout", [R.RIPPLE_SOA, R.RIPPLE_AOS])
def test_blast_fp32_full_run_50_and_100_steps(ctx, dims, layout):
    """The headline scheme (3D FP32 MUSCL-Hancock + Rusanov, transmissive
    blast with 1 % noise) over whole runs: the full field after 50 steps (the
    headline step count) and after 100 steps (the FP32 horizon of the 2e-5
    bar) against the FP64 oracle, every cell under the element-wise bound.
    Grids span several tiles with ragged x/y tails and several z chunks."""
    U0, ref = _oracle_blast_runs(dims, seed=11)
    f = R.ripple_field_create(ctx, dims, 5, layout, 2, R.RIPPLE_F32)
    try:
        host = U0 if layout == R.RIPPLE_SOA else np.ascontiguousarray(np.moveaxis(U0, 0, -1))
        R.ripple_field_upload(f, host, layout)
        prm = R.make_fv_params([1.0 / d for d in dims], scheme=MUSCL, bc=TRA)
        for steps in (50, 100):
            st = R.ripple_fv_step(f, prm, 50)
            got = R.ripple_field_download(f, R.RIPPLE_SOA)
            want, info = ref[steps]
            e1, ei = assert_parity(got, want, 2e-5, LINF_F32)
            print(f"{dims} layout {layout} step {steps}: rel L1 {e1:.3e}, max {ei:.3e}")
            assert st["t"] == pytest.approx(info["t"], rel=1e-5)
            assert st["dt_last"] == pytest.approx(info["dt_last"], rel=1e-5)
    finally:
        R.ripple_field_destroy(f)


@pytest.mark.parametrize("layout", [R.RIPPLE_SOA, R.RIPPLE_AOS])
@pytest.mark.parametrize("bc", [PER, TRA])
def test_row_kernel_equals_pair_kernel_bitwise(ctx, layout, bc):
    """The row kernel (one warp per 64-cell row, x faces by shuffles) and the
    pair kernel evaluate every predicted state and face once, with the same
    packed arithmetic in the same order, so they give identical bits; the
    grid has a ragged 64-wide x tile, a ragged 14-row y tile and three z chunks."""
    U0 = inputs.euler3d_blast(0, seed=9, dims=(150, 47, 70)).astype(np.float32)
    a, sa = gpu_euler(ctx, U0, 8, dtype=R.RIPPLE_F32, scheme=MUSCL, bc=bc, layout=layout, variant=ROW)
    b, sb = gpu_euler(ctx, U0, 8, dtype=R.RIPPLE_F32, scheme=MUSCL, bc=bc, layout=layout, variant=PAIR)
    assert np.array_equal(a, b)
    assert sa["t"] == sb["t"] and sa["dt_last"] == sb["dt_last"]


@pytest.mark.parametrize("layout", [R.RIPPLE_SOA, R.RIPPLE_AOS])
def test_row_kernel_equals_pair_kernel_bitwise_with_subnormal_values(ctx, layout):
    """By step 24 the blast's momentum ahead of the shock has decayed into
    subnormal numbers (a rescaling of the faces by a power of two is then no
    longer exact, so only the same arithmetic gives the same bits): the two
    kernels still agree bit for bit, on a grid of four 64-wide x tiles."""
    dims = (256, 64, 64)
    U0 = inputs.euler3d_blast(256, seed=9, dims=dims).astype(np.float32)
    kw = dict(dtype=R.RIPPLE_F32, scheme=MUSCL, bc=TRA, layout=layout, dx=[1.0 / 256] * 3)
    a, sa = gpu_euler(ctx, U0, 24, variant=ROW, **kw)
    b, sb = gpu_euler(ctx, U0, 24, variant=PAIR, **kw)
    tiny = np.finfo(np.float32).tiny
    assert np.any((a != 0) & (np.abs(a) < tiny)), "no subnormal values: the case does not cover them"
    assert np.array_equal(a, b)
    assert sa["t"] == sb["t"] and sa["dt_last"] == sb["dt_last"]


def test_many_tiles_per_cta_many_launches(ctx):
    # 1024 z-chunked tiles over the persistent CTAs (several tiles per CTA) for
    # 200 launches: every tile boundary hands the plane ring over between warps
    # that wait for different planes; no bounded wait may run out
    dims = (128, 256, 256)
    U0 = inputs.euler3d_blast(256, seed=4, dims=dims).astype(np.float32)
    f = R.ripple_field_create(ctx, dims, 5, R.RIPPLE_SOA, 2, R.RIPPLE_F32)
    try:
        R.ripple_field_upload(f, U0)
        prm = R.make_fv_params([1 / 256] * 3, scheme=MUSCL, bc=TRA)
        st = R.ripple_fv_step(f, prm, 200)
        assert st["steps_done"] == 200
        out = R.ripple_field_download(f)
        assert np.isfinite(out).all()
    finally:
        R.ripple_field_destroy(f)


@pytest.mark.parametrize("dtype", [R.RIPPLE_F32, R.RIPPLE_F64])
@pytest.mark.parametrize("dims,scheme", [((45, 30), MUSCL), ((21, 17, 15), MUSCL), ((21, 17, 15), RUS)])
def test_aos_equals_soa_bitwise(ctx, dtype, dims, scheme):
    U0 = _random_state(dims, seed=8)
    a, _ = gpu_euler(ctx, U0, 7, dtype=dtype, scheme=scheme, bc=TRA, layout=R.RIPPLE_AOS)
    b, _ = gpu_euler(ctx, U0, 7, dtype=dtype, scheme=scheme, bc=TRA, layout=R.RIPPLE_SOA)
    assert np.array_equal(a, b)


@pytest.mark.parametrize("dtype", [R.RIPPLE_F32, R.RIPPLE_F64])
@pytest.mark.parametrize("dims", [(40, 24), (18, 12, 20)])
@pytest.mark.parametrize("scheme", [RUS, MUSCL])
def test_uniform_state_bit_exact(ctx, dtype, dims, scheme):
    vel = [0.7, -0.4, 0.25][: len(dims)]
    U0 = inputs.uniform_state(dims, 1.3, vel, 0.9)
    npdt = np.float32 if dtype == R.RIPPLE_F32 else np.float64
    U0 = U0.astype(npdt)
    for bc in (PER, TRA):
        got, _ = gpu_euler(ctx, U0, 15, dtype=dtype, scheme=scheme, bc=bc)
        assert np.array_equal(got, U0)


def test_periodic_conservation_fp64(ctx):
    U0 = _random_state((48, 40, 20), seed=9)
    got, st = gpu_euler(ctx, U0, 30, scheme=MUSCL, bc=PER)
    for m in range(5):
        t0 = math.fsum(U0[m].ravel())
        t1 = math.fsum(got[m].ravel())
        scale = np.abs(U0[m]).sum()
        assert abs(t1 - t0) <= 1e-13 * scale
        assert abs(st["totals"][m] - t1) <= 1e-14 * scale


def test_repeat_is_deterministic(ctx):
    U0 = inputs.euler3d_blast(32, seed=2).astype(np.float32)
    a, sa = gpu_euler(ctx, U0, 10, dtype=R.RIPPLE_F32, scheme=MUSCL, bc=TRA)
    b, sb = gpu_euler(ctx, U0, 10, dtype=R.RIPPLE_F32, scheme=MUSCL, bc=TRA)
    assert np.array_equal(a, b)
    assert sa["t"] == sb["t"] and sa["totals"] == sb["totals"]


def test_split_calls_equal_one_call(ctx):
    """Checkpoint/resume: 10 steps == 4 + download/upload + 6 (bitwise)."""
    U0 = _random_state((30, 26, 14), seed=12)
    full, _ = gpu_euler(ctx, U0, 10, scheme=MUSCL, bc=PER)
    part, _ = gpu_euler(ctx, U0, 4, scheme=MUSCL, bc=PER)
    rest, _ = gpu_euler(ctx, part, 6, scheme=MUSCL, bc=PER)
    assert np.array_equal(full, rest)


def test_negative_pressure_reports_numeric(ctx):
    U0 = inputs.uniform_state((16, 16), 1.0, [0.0, 0.0], 1.0)
    U0[3, 5, 5] = -1.0
    with pytest.raises(R.RippleError) as ei:
        gpu_euler(ctx, U0, 2)
    assert ei.value.status == R.RIPPLE_ERR_NUMERIC


def test_invalid_halo_rejected(ctx):
    f = R.ripple_field_create(ctx, (16, 16), 4, R.RIPPLE_SOA, 1, R.RIPPLE_F32)
    try:
        with pytest.raises(R.RippleError) as ei:
            R.ripple_fv_step(f, R.make_fv_params([1 / 16] * 2, scheme=MUSCL), 1)
        assert ei.value.status == R.RIPPLE_ERR_INVALID
    finally:
        R.ripple_field_destroy(f)


def test_budget_enforced():
    c = R.ripple_ctx_create(0, 1 << 20)
    try:
        with pytest.raises(R.RippleError) as ei:
            R.ripple_field_create(c, (256, 256), 4, R.RIPPLE_SOA, 1, R.RIPPLE_F32)
        assert ei.value.status == R.RIPPLE_ERR_BUDGET
    finally:
        R.ripple_ctx_destroy(c)


@pytest.mark.parametrize("layout", [R.RIPPLE_SOA, R.RIPPLE_AOS])
def test_config1_full_size_sampled(ctx, layout):
    """256^3 FP32 MUSCL-Hancock blast, transmissive, in the launch configuration
    the benchmark times.  After 49 steps, step 50 is checked against the
    oracle's single-step evaluation at 4096 sampled cells (from the same
    GPU state), and the whole run against conservation (waves stay inside)."""
    n = 256
    U0 = inputs.euler3d_blast(n, seed=1).astype(np.float32)
    dims = (n, n, n)
    f = R.ripple_field_create(ctx, dims, 5, layout, 2, R.RIPPLE_F32)
    try:
        host = U0 if layout == R.RIPPLE_SOA else np.ascontiguousarray(np.moveaxis(U0, 0, -1))
        R.ripple_field_upload(f, host, layout)
        prm = R.make_fv_params([1 / n] * 3, scheme=MUSCL, bc=TRA)
        R.ripple_fv_step(f, prm, 49, stats=False)
        U49 = R.ripple_field_download(f, R.RIPPLE_SOA)
        st = R.ripple_fv_step(f, prm, 1)
        U50 = R.ripple_field_download(f, R.RIPPLE_SOA)
    finally:
        R.ripple_field_destroy(f)
    rng = inputs.uniform(77, 4096)
    cells = (rng * n ** 3).astype(np.int64)
    # include boundary and corner cells
    cells = np.concatenate([cells, [0, n - 1, n * n - 1, n ** 3 - 1, n * n * (n // 2) + n * (n // 2) + n // 2]])
    vals, dt = oracle.euler_step_cells(U49.astype(np.float64), cells, scheme=MUSCL, bc=TRA)
    gpu = U50.reshape(5, -1)[:, cells].T
    assert dt == pytest.approx(st["dt_last"], rel=1e-6)
    err = np.abs(gpu - vals).sum(axis=0) / np.abs(vals).sum(axis=0).clip(1e-30)
    assert err.max() <= 2e-6, err
    # conservation over the run (FP64 device totals vs the initial state)
    for m in (0, 4):
        t0 = math.fsum(U0[m].astype(np.float64).ravel())
        assert abs(st["totals"][m] - t0) <= 2e-6 * abs(t0)
