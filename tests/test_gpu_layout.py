"""GPU parity of the layout microbenchmarks (Section 7.1 SAXPY, Section 7.2
particle update) against the FP64 oracle, through the C ABI: sizes that span
several vectors, chunks and CTAs with ragged tails, misaligned arrays, both
layouts, direct and staged kernels."""
import ctypes

import numpy as np
import pytest

import oracle
import paper_2104_08571_gb300 as R

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import torch
    torch.cuda.init()
    c = R.ripple_ctx_create(0)
    yield c
    R.ripple_ctx_destroy(c)


def ulps32(got, ref64):
    """Distance in FP32 units in the last place between got (float32) and ref rounded to FP32."""
    a = np.asarray(got, dtype=np.float32).view(np.int32).astype(np.int64)
    b = np.asarray(ref64, dtype=np.float64).astype(np.float32).view(np.int32).astype(np.int64)
    return np.abs(a - b)


@pytest.mark.parametrize("n", [1, 3, 4, 17, 1000, 4 * 1024 * 1024 + 5])
@pytest.mark.parametrize("offsets", [(0, 0), (1, 1), (1, 2)])
def test_saxpy_matches_oracle(ctx, n, offsets):
    import torch
    rng = np.random.default_rng(n + 7 * offsets[1])
    x = rng.standard_normal(n + 4).astype(np.float32)
    y = rng.standard_normal(n + 4).astype(np.float32)
    a = np.float32(1.7)
    xd = torch.from_numpy(x).cuda()[offsets[0]:offsets[0] + n]
    yd = torch.from_numpy(y).cuda()[offsets[1]:offsets[1] + n]
    torch.cuda.synchronize()  # torch's copies are done before the library's stream reads the tensors
    R.ripple_saxpy(ctx, float(a), xd, yd)
    R.ripple_ctx_sync(ctx)
    ref = oracle.saxpy(a, x[offsets[0]:offsets[0] + n], y[offsets[1]:offsets[1] + n])
    d = ulps32(yd.cpu().numpy(), ref)
    assert d.max() <= 1
    assert (d > 0).mean() < 1e-3  # a fused multiply-add equals the once-rounded exact result


def _particles(n, layout, seed):
    rng = np.random.default_rng(seed)
    pos = rng.uniform(-1, 1, size=(n, 3)).astype(np.float32)
    vel = rng.uniform(-2, 2, size=(n, 3)).astype(np.float32)
    if layout == R.RIPPLE_AOS:
        return np.ascontiguousarray(np.concatenate([pos, vel], axis=1).reshape(-1))
    return np.ascontiguousarray(np.concatenate([pos.T, vel.T], axis=0).reshape(-1))


@pytest.mark.parametrize("n", [1, 2, 5, 2048, 3 * 2048 + 4, 1 << 20, (1 << 20) + 3])
@pytest.mark.parametrize("layout", [R.RIPPLE_AOS, R.RIPPLE_SOA])
@pytest.mark.parametrize("staged", [False, True])
def test_particle_update_matches_oracle(ctx, n, layout, staged):
    import torch
    p = _particles(n, layout, n)
    dt = np.float32(0.01)
    pd = torch.from_numpy(p).cuda()
    torch.cuda.synchronize()
    R.ripple_particle_update(ctx, pd, float(dt), layout=layout, staged=staged)
    R.ripple_ctx_sync(ctx)
    got = pd.cpu().numpy()
    ref = oracle.particle_update(p, dt, "aos" if layout == R.RIPPLE_AOS else "soa")
    d = ulps32(got, ref)
    assert d.max() <= 1
    assert (d > 0).mean() < 1e-3


@pytest.mark.parametrize("layout", [R.RIPPLE_AOS, R.RIPPLE_SOA])
def test_particle_staged_equals_direct_and_layouts_agree(ctx, layout):
    import torch
    n = 5 * 2048 + 8
    p = _particles(n, layout, 11)
    a = torch.from_numpy(p).cuda()
    b = a.clone()
    torch.cuda.synchronize()
    for _ in range(3):
        R.ripple_particle_update(ctx, a, 0.02, layout=layout, staged=False)
        R.ripple_particle_update(ctx, b, 0.02, layout=layout, staged=True)
    R.ripple_ctx_sync(ctx)
    assert torch.equal(a, b)
    # the other layout of the same particles gives the same positions, bit for bit
    other = R.RIPPLE_SOA if layout == R.RIPPLE_AOS else R.RIPPLE_AOS
    if layout == R.RIPPLE_AOS:
        q = np.ascontiguousarray(p.reshape(n, 6).T.reshape(-1))
    else:
        q = np.ascontiguousarray(p.reshape(6, n).T.reshape(-1))
    c = torch.from_numpy(q).cuda()
    torch.cuda.synchronize()
    for _ in range(3):
        R.ripple_particle_update(ctx, c, 0.02, layout=other, staged=True)
    R.ripple_ctx_sync(ctx)
    got = c.cpu().numpy()
    got = got.reshape(6, n).T.reshape(-1) if other == R.RIPPLE_SOA else got.reshape(n, 6).T.reshape(-1)
    assert np.array_equal(got, a.cpu().numpy())


def test_layout_entry_points_reject_bad_arguments(ctx):
    lib = R.load()
    assert lib.ripple_saxpy(ctx, -1, ctypes.c_float(1.0), None, None) == R.RIPPLE_ERR_INVALID
    assert lib.ripple_saxpy(None, 4, ctypes.c_float(1.0), None, None) == R.RIPPLE_ERR_INVALID
    assert lib.ripple_particle_update(ctx, 4, ctypes.c_float(0.1), None, R.RIPPLE_SOA, 0) == R.RIPPLE_ERR_INVALID
    import torch
    t = torch.zeros(12, device="cuda")
    assert lib.ripple_particle_update(ctx, 2, ctypes.c_float(0.1), ctypes.c_void_p(t.data_ptr()), 7, 0) == \
        R.RIPPLE_ERR_INVALID
    assert lib.ripple_saxpy(ctx, 0, ctypes.c_float(1.0), None, None) == R.RIPPLE_OK
