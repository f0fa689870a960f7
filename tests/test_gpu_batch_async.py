"""Dependency-driven batch rounds (async_queue = 1): one persistent launch runs
up to steps_per_sync steps of every resident Euler problem, each problem
starting its next step as soon as its own previous step is complete.  Every
problem's arithmetic is the per-step kernel's, so results equal the
one-launch-per-global-step mode bit for bit; parity with the FP64 oracle and
the eikonal Fast Marching solution is checked as well."""
import ctypes

import numpy as np
import pytest

import inputs
import oracle
import paper_2104_08571_gb300 as R
from tests.gpu_util import LINF_EIK, LINF_F32, LINF_F64, assert_parity, rel_l1

pytestmark = pytest.mark.gpu


@pytest.fixture()
def ctx():
    import torch
    assert torch.cuda.is_available()
    c = R.ripple_ctx_create(0)
    # the tests of this file compare batched rounds with one another bit for bit:
    # a lone problem stays on the batched kernels (solo rounds have their own test)
    R.ripple_batch_configure(c, solo_rounds=False)
    yield c
    R.ripple_ctx_destroy(c)


def _euler(nx, ny, amp, nsteps, bc=R.RIPPLE_BC_PERIODIC, U=None):
    if U is None:
        U = inputs.euler2d_sine(nx, amp=amp, ny=ny).astype(np.float32)
    return R.euler_request(U, nsteps, [1.0 / nx, 1.0 / ny], bc=bc)


def _again(req):
    return R.euler_request(req["input"], req["nsteps"], req["dx"], bc=req.get("bc", R.RIPPLE_BC_PERIODIC))


def _run(ctx, reqs, timeout_ms=120000):
    tickets = R.ripple_batch_submit(ctx, reqs)
    return [R.ripple_wait(ctx, t, timeout_ms) for t in tickets]


def _mix():
    # sides from one tile to many, ragged edges, both boundary kinds, uneven step counts
    return [_euler(32, 32, 0.2, 40), _euler(45, 77, 0.1, 25), _euler(100, 64, 0.3, 60),
            _euler(33, 129, 0.05, 10, bc=R.RIPPLE_BC_TRANSMISSIVE), _euler(128, 128, 0.2, 100),
            _euler(257, 31, 0.15, 1), _euler(200, 180, 0.25, 64)]


def test_async_rounds_equal_per_step_launches_bitwise(ctx):
    ref = _mix()
    infos = _run(ctx, ref)
    assert all(i["status"] == R.RIPPLE_OK for i in infos)
    for sps in (64, 7, 1):
        R.ripple_batch_configure(ctx, steps_per_sync=sps, async_queue=True, solo_rounds=False)
        reqs = [_again(r) for r in ref]
        infos = _run(ctx, reqs)
        for r, q, i in zip(ref, reqs, infos):
            assert i["status"] == R.RIPPLE_OK and i["work"] == r["nsteps"]
            assert np.array_equal(q["output"], r["output"]), (sps, r["input"].shape)


def test_async_walk_rounds_equal_per_step_launches_bitwise(ctx):
    # walk staging: dependency-driven rounds take walk units (30 columns x 16
    # rows) from the round's counter; every unit is the per-step walk's
    # arithmetic, which is the tiled step's bit for bit
    ref = _mix()
    infos = _run(ctx, ref)
    assert all(i["status"] == R.RIPPLE_OK for i in infos)
    for sps, async_q in ((64, False), (64, True), (7, True), (1, True)):
        R.ripple_batch_configure(ctx, steps_per_sync=sps, staging=2, async_queue=async_q, solo_rounds=False)
        reqs = [_again(r) for r in ref]
        infos = _run(ctx, reqs)
        for r, q, i in zip(ref, reqs, infos):
            assert i["status"] == R.RIPPLE_OK and i["work"] == r["nsteps"]
            assert np.array_equal(q["output"], r["output"]), (sps, async_q, r["input"].shape)


def test_async_rounds_match_oracle(ctx):
    R.ripple_batch_configure(ctx, steps_per_sync=128, async_queue=True, solo_rounds=False)
    reqs = _mix()
    infos = _run(ctx, reqs)
    for req, info in zip(reqs, infos):
        assert info["status"] == R.RIPPLE_OK
        ref, _ = oracle.euler_run(req["input"].astype(np.float64), req["nsteps"], dx=req["dx"],
                                  bc=req.get("bc", 0))
        assert_parity(req["output"], ref, 2e-5, LINF_F32)


@pytest.mark.parametrize("staging", [0, 2])
def test_one_launch_per_round(ctx, staging):
    # uneven step counts: per-step launches shrink a round to the shortest
    # remaining problem; a dependency-driven round runs each to its own end
    # (staging 0: tiles staged by TMA; 2: walk units)
    reqs = [_euler(64 + 8 * i, 48, 0.1 + 0.01 * i, 5 + 7 * i) for i in range(8)]
    R.ripple_batch_configure(ctx, steps_per_sync=64, async_queue=True, use_graphs=False, staging=staging,
                             solo_rounds=False)
    s0 = R.ripple_batch_get_stats(ctx)
    infos = _run(ctx, reqs)
    s1 = R.ripple_batch_get_stats(ctx)
    assert all(i["status"] == R.RIPPLE_OK for i in infos)
    assert s1["launches"] - s0["launches"] == 1
    assert s1["global_steps"] - s0["global_steps"] == max(r["nsteps"] for r in reqs)
    R.ripple_batch_configure(ctx, steps_per_sync=64, async_queue=False, use_graphs=False, staging=staging,
                             solo_rounds=False)
    again = [_again(r) for r in reqs]
    s2 = R.ripple_batch_get_stats(ctx)
    _run(ctx, again)
    s3 = R.ripple_batch_get_stats(ctx)
    assert s3["launches"] - s2["launches"] == max(r["nsteps"] for r in reqs)
    for a, b in zip(reqs, again):
        assert np.array_equal(a["output"], b["output"])


def test_async_layouts_and_tile_shapes(ctx):
    base = _euler(77, 61, 0.2, 21)
    _run(ctx, [base])
    for layout in (R.RIPPLE_SOA, R.RIPPLE_AOS):
        for v in range(3):
            R.ripple_batch_configure(ctx, layout=layout, tile_variant=v, async_queue=True, solo_rounds=False)
            r = _again(base)
            other = _euler(150, 40, 0.3, 33)
            infos = _run(ctx, [r, other])
            assert all(i["status"] == R.RIPPLE_OK for i in infos)
            assert np.array_equal(r["output"], base["output"]), (layout, v)
    R.ripple_batch_configure(ctx, solo_rounds=False)


@pytest.mark.parametrize("staging", [0, 2])
def test_async_with_eikonal_requests(ctx, staging):
    R.ripple_batch_configure(ctx, steps_per_sync=16, async_queue=True, staging=staging, solo_rounds=False)
    s = inputs.eikonal_slowness((120, 90), seed=4).astype(np.float32)
    src = inputs.eikonal_sources((120, 90), seed=4)
    e = R.eikonal_request(s, src, 1.0 / 120)
    a = _euler(90, 70, 0.25, 37)
    infos = _run(ctx, [a, e, _euler(40, 40, 0.1, 5)])
    assert all(i["status"] == R.RIPPLE_OK for i in infos)
    ref = oracle.eikonal_fmm(s.astype(np.float64), 1.0 / 120, src)
    assert_parity(e["output"][None], ref[None], 1e-4, LINF_EIK)
    R.ripple_batch_configure(ctx, solo_rounds=False)
    alone = _again(a)
    _run(ctx, [alone])
    assert np.array_equal(alone["output"], a["output"])


@pytest.mark.parametrize("staging", [0, 2])
def test_async_with_cell_budget_and_late_requests(ctx, staging):
    # a per-round cell budget: problems join the stepped set as others finish
    R.ripple_batch_configure(ctx, steps_per_sync=8, async_queue=True, active_cells=64 * 64 * 2, staging=staging,
                             solo_rounds=False)
    reqs = [_euler(64, 64, 0.1 + 0.03 * i, 12 + 5 * i) for i in range(5)]
    t1 = R.ripple_batch_submit(ctx, reqs[:3])
    t2 = R.ripple_batch_submit(ctx, reqs[3:])
    infos = [R.ripple_wait(ctx, t, 120000) for t in t1 + t2]
    assert all(i["status"] == R.RIPPLE_OK and i["work"] == r["nsteps"] for i, r in zip(infos, reqs))
    R.ripple_batch_configure(ctx, solo_rounds=False)
    for r in reqs:
        b = _again(r)
        _run(ctx, [b])
        assert np.array_equal(b["output"], r["output"])


@pytest.mark.parametrize("staging", [0, 2])
def test_async_numeric_error_reported_per_request(ctx, staging):
    R.ripple_batch_configure(ctx, steps_per_sync=16, async_queue=True, staging=staging, solo_rounds=False)
    bad = _euler(40, 40, 0.2, 5)
    bad["input"][3, 10, 10] = -1.0  # negative energy -> negative pressure
    good = _euler(40, 40, 0.2, 9)
    infos = _run(ctx, [bad, good])
    assert infos[0]["status"] == R.RIPPLE_ERR_NUMERIC
    assert infos[1]["status"] == R.RIPPLE_OK


def test_configure_rejects_bad_async_flag(ctx):
    cfg = R.ripple_batch_config(R.RIPPLE_SOA, 0, 16, 1, R.RIPPLE_F32, 4, 0, 0, 2)
    assert R.load().ripple_batch_configure(ctx, ctypes.byref(cfg)) == R.RIPPLE_ERR_INVALID
