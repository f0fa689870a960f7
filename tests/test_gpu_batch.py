"""Batched and served execution (one launch per global step over many
independent problems) against the FP64 oracle, plus the serving invariants:
a problem gives the same bits alone and in a mix, requests wait for memory
under a budget, and requests that arrive while others run are admitted."""
import time

import numpy as np
import pytest

import inputs
import oracle
import paper_2104_08571_gb300 as R
from tests.gpu_util import LINF_EIK, LINF_F32, LINF_F64, assert_parity, max_rel, rel_l1

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


def _euler(nx, ny, amp, nsteps, bc=R.RIPPLE_BC_PERIODIC):
    U = inputs.euler2d_sine(nx, amp=amp, ny=ny).astype(np.float32)
    return R.euler_request(U, nsteps, [1.0 / nx, 1.0 / ny], bc=bc)


def _eik(nx, ny, seed):
    s = inputs.eikonal_slowness((nx, ny), seed=seed).astype(np.float32)
    src = inputs.eikonal_sources((nx, ny), seed=seed)
    return R.eikonal_request(s, src, 1.0 / max(nx, ny))


def _again(req):
    """A fresh request with the same input as req (Euler or eikonal)."""
    if req["kind"] == R.RIPPLE_REQ_EULER:
        return R.euler_request(req["input"], req["nsteps"], req["dx"], bc=req.get("bc", R.RIPPLE_BC_PERIODIC))
    return R.eikonal_request(req["input"], req["sources"], req["h"])


def _run(ctx, reqs, timeout_ms=120000):
    tickets = R.ripple_batch_submit(ctx, reqs)
    return [R.ripple_wait(ctx, t, timeout_ms) for t in tickets]


def _oracle_euler(req):
    U0 = req["input"].astype(np.float64)
    ref, _ = oracle.euler_run(U0, req["nsteps"], dx=req["dx"], bc=req.get("bc", 0))
    return ref


def test_batch_euler_matches_oracle(ctx):
    reqs = [_euler(32, 32, 0.2, 40), _euler(45, 77, 0.1, 25), _euler(100, 64, 0.3, 60),
            _euler(33, 129, 0.05, 10, bc=R.RIPPLE_BC_TRANSMISSIVE), _euler(128, 128, 0.2, 100)]
    infos = _run(ctx, reqs)
    for req, info in zip(reqs, infos):
        assert info["status"] == R.RIPPLE_OK
        assert info["work"] == req["nsteps"]
        assert_parity(req["output"], _oracle_euler(req), 2e-5, LINF_F32)


def test_batch_eikonal_matches_fmm(ctx):
    reqs = [_eik(100, 100, 1), _eik(64, 150, 2), _eik(257, 97, 3)]
    infos = _run(ctx, reqs)
    for req, info in zip(reqs, infos):
        assert info["status"] == R.RIPPLE_OK and info["work"] > 0
        ref = oracle.eikonal_fmm(req["input"].astype(np.float64), req["h"], req["sources"])
        assert_parity(req["output"][None], ref[None], 1e-4, LINF_EIK)


def test_alone_equals_in_mix_bitwise(ctx):
    # every problem on the batched kernels (a lone problem too): same bits alone and in the mix
    R.ripple_batch_configure(ctx, solo_rounds=False)
    a = _euler(90, 70, 0.25, 37)
    e = _eik(120, 80, 5)
    _run(ctx, [a])
    _run(ctx, [e])
    alone_a, alone_e = a["output"].copy(), e["output"].copy()
    a2 = R.euler_request(a["input"], 37, a["dx"])
    e2 = R.eikonal_request(e["input"], e["sources"], e["h"])
    mix = [_euler(64, 64, 0.1, 80), a2, _eik(200, 150, 6), _euler(300, 40, 0.2, 15), e2, _euler(33, 33, 0.3, 50)]
    infos = _run(ctx, mix)
    assert all(i["status"] == R.RIPPLE_OK for i in infos)
    assert np.array_equal(a2["output"], alone_a)
    assert np.array_equal(e2["output"], alone_e)
    # with a small per-step cell budget problems are paused and resumed: same bits
    R.ripple_batch_configure(ctx, active_cells=5000, steps_per_sync=5, solo_rounds=False)
    a3 = R.euler_request(a["input"], 37, a["dx"])
    mix = [_euler(64, 64, 0.1, 80), a3, _euler(300, 40, 0.2, 15), _euler(33, 33, 0.3, 50)]
    infos = _run(ctx, mix)
    assert all(i["status"] == R.RIPPLE_OK and i["work"] == r["nsteps"] for i, r in zip(infos, mix))
    assert np.array_equal(a3["output"], alone_a)


def test_solo_rounds_alone_and_in_mix(ctx):
    """A request served alone runs on the single-problem kernels (solo rounds):
    an Euler problem on the multi-step solver, bit for bit the batched step,
    also when it is joined by other requests part-way (it then continues on
    the batched kernel from its own step); an eikonal problem with the same
    bits; both against the oracle."""
    R.ripple_batch_configure(ctx)  # solo rounds on (the default)
    a = _euler(150, 130, 0.25, 150)
    e = _eik(200, 170, 8)
    _run(ctx, [a])
    _run(ctx, [e])
    mix = [_again(a), _euler(64, 64, 0.1, 40), _again(e), _euler(40, 40, 0.2, 20)]
    infos = _run(ctx, mix)
    assert all(i["status"] == R.RIPPLE_OK for i in infos)
    assert np.array_equal(mix[0]["output"], a["output"])
    assert np.array_equal(mix[2]["output"], e["output"])
    assert_parity(a["output"], _oracle_euler(a), 2e-5, LINF_F32)
    # joined part-way: a long problem alone, a second one submitted while it runs
    long = _euler(300, 260, 0.2, 400)
    t1 = R.ripple_batch_submit(ctx, [long])
    time.sleep(0.002)
    late = _euler(50, 50, 0.15, 30)
    t2 = R.ripple_batch_submit(ctx, [late])
    assert R.ripple_wait(ctx, t1[0], 120000)["status"] == R.RIPPLE_OK
    assert R.ripple_wait(ctx, t2[0], 120000)["status"] == R.RIPPLE_OK
    assert_parity(long["output"], _oracle_euler(long), 2e-5, LINF_F32)
    assert_parity(late["output"], _oracle_euler(late), 2e-5, LINF_F32)
    R.ripple_batch_configure(ctx, solo_rounds=False)
    batched = [_again(long), _again(late)]
    _run(ctx, batched)
    assert np.array_equal(batched[0]["output"], long["output"])
    assert np.array_equal(batched[1]["output"], late["output"])


def test_solo_rounds_over_a_batched_start_bitwise(ctx):
    """More resident problems than the solo bound start in batched rounds; as
    they finish, the rest continue in solo rounds (an eikonal problem already
    iterating in batched rounds is solved again whole): every result is the
    same bits as the problem alone in batched rounds."""
    reqs = [_euler(40 + 7 * i, 36 + 5 * i, 0.1 + 0.02 * i, 15 + 9 * i) for i in range(5)]
    reqs += [_eik(150, 120, 11), _eik(90, 200, 12)]
    R.ripple_batch_configure(ctx, solo_rounds=False)
    alone = []
    for r in reqs:
        a = _again(r)
        assert _run(ctx, [a])[0]["status"] == R.RIPPLE_OK
        alone.append(a["output"])
    for bound in (2, 4):
        R.ripple_batch_configure(ctx, solo_rounds=bound)
        mix = [_again(r) for r in reqs]
        infos = _run(ctx, mix)
        assert all(i["status"] == R.RIPPLE_OK for i in infos)
        for m, a in zip(mix, alone):
            assert np.array_equal(m["output"], a)
    R.ripple_batch_configure(ctx, solo_rounds=False)


@pytest.mark.parametrize("layout", [R.RIPPLE_SOA, R.RIPPLE_AOS])
@pytest.mark.parametrize("dtype", [R.RIPPLE_F32, R.RIPPLE_F64])
def test_solo_solver_equals_batched_step_bitwise(ctx, layout, dtype):
    """The multi-step solo solver against the batched step, bit for bit, on
    grids that leave ragged strips (widths not multiples of 30) and segments,
    one-cell-wide and one-row grids, both boundary conditions."""
    npdt = np.float32 if dtype == R.RIPPLE_F32 else np.float64
    shapes = [(64, 64, 0.2, 120, R.RIPPLE_BC_PERIODIC), (31, 47, 0.3, 77, R.RIPPLE_BC_TRANSMISSIVE),
              (1, 40, 0.1, 20, R.RIPPLE_BC_PERIODIC), (45, 1, 0.1, 20, R.RIPPLE_BC_TRANSMISSIVE),
              (2, 2, 0.2, 9, R.RIPPLE_BC_PERIODIC), (611, 333, 0.15, 60, R.RIPPLE_BC_PERIODIC),
              (1000, 700, 0.2, 330, R.RIPPLE_BC_TRANSMISSIVE)]  # the last takes several solo launches
    out = {}
    for solo in (True, False):
        R.ripple_batch_configure(ctx, layout=layout, dtype=dtype, solo_rounds=solo)
        res = []
        for nx, ny, amp, nsteps, bc in shapes:
            U = inputs.euler2d_sine(nx, amp=amp, ny=ny).astype(npdt)
            req = R.euler_request(U, nsteps, [1.0 / nx, 1.0 / ny], bc=bc)
            info = _run(ctx, [req])[0]
            assert info["status"] == R.RIPPLE_OK and info["work"] == nsteps
            res.append((req["output"], info["t"]))
        out[solo] = res
    R.ripple_batch_configure(ctx, solo_rounds=False)
    for (a, ta), (b, tb), shp in zip(out[True], out[False], shapes):
        assert np.array_equal(a, b), shp
        assert ta == tb, shp


def test_solo_barrier_timeout_reports(ctx, monkeypatch):
    """A grid-barrier wait of the solo solver that runs out (the wait bound
    forced to zero polls) fails the request with RIPPLE_ERR_TIMEOUT; the
    runtime keeps serving."""
    monkeypatch.setenv("RIPPLE_GRID_SPIN_LIMIT", "0")
    R.ripple_batch_configure(ctx)
    info = _run(ctx, [_euler(300, 300, 0.2, 50)])[0]
    monkeypatch.delenv("RIPPLE_GRID_SPIN_LIMIT")
    assert info["status"] == R.RIPPLE_ERR_TIMEOUT
    req = _euler(60, 60, 0.2, 30)
    assert _run(ctx, [req])[0]["status"] == R.RIPPLE_OK
    assert_parity(req["output"], _oracle_euler(req), 2e-5, LINF_F32)
    R.ripple_batch_configure(ctx, solo_rounds=False)


def test_pageable_and_page_locked_requests(ctx):
    """Pageable request arrays go through the runtime's page-locked arena (the
    result is copied out when the ticket is retrieved, by wait or by poll);
    page-locked arrays are copied directly: the same bits either way."""
    import torch
    R.ripple_batch_configure(ctx, solo_rounds=False)
    base = _euler(120, 90, 0.2, 25)
    pin_in = torch.from_numpy(base["input"]).pin_memory().numpy()
    pin_out = torch.empty(base["input"].shape, dtype=torch.float32, pin_memory=True).numpy()
    pinned = R.euler_request(pin_in, 25, base["dx"], out=pin_out)
    polled = _again(base)
    infos = _run(ctx, [base, pinned])
    assert all(i["status"] == R.RIPPLE_OK for i in infos)
    assert np.array_equal(base["output"], pinned["output"])
    t = R.ripple_batch_submit(ctx, [polled])[0]
    deadline = time.time() + 60
    info = None
    while info is None and time.time() < deadline:
        info = R.ripple_poll(ctx, t)
        time.sleep(0.001)
    assert info is not None and info["status"] == R.RIPPLE_OK
    assert np.array_equal(polled["output"], base["output"])


def test_batch_matches_single_field_sweep(ctx):
    req = _euler(96, 80, 0.2, 30)
    _run(ctx, [req])
    f = R.ripple_field_create(ctx, (96, 80), 4, R.RIPPLE_SOA, 1, R.RIPPLE_F32)
    try:
        R.ripple_field_upload(f, req["input"])
        R.ripple_fv_step(f, R.make_fv_params(req["dx"]), 30)
        single = R.ripple_field_download(f)
    finally:
        R.ripple_field_destroy(f)
    assert rel_l1(req["output"], single) <= 1e-6
    assert max_rel(req["output"], single) <= 1e-5  # another kernel: FP32 rounding of its own order


def test_graphs_and_sync_interval_do_not_change_results(ctx):
    R.ripple_batch_configure(ctx, solo_rounds=False)
    reqs1 = [_euler(70, 50, 0.2, 33), _eik(90, 90, 7)]
    _run(ctx, reqs1)
    R.ripple_batch_configure(ctx, steps_per_sync=3, use_graphs=False, fim_iters_per_step=1, solo_rounds=False)
    reqs2 = [R.euler_request(reqs1[0]["input"], 33, reqs1[0]["dx"]),
             R.eikonal_request(reqs1[1]["input"], reqs1[1]["sources"], reqs1[1]["h"])]
    _run(ctx, reqs2)
    assert np.array_equal(reqs1[0]["output"], reqs2[0]["output"])
    assert np.array_equal(reqs1[1]["output"], reqs2[1]["output"])


def test_aos_layout_tile_variants_and_staging(ctx):
    base = _euler(77, 61, 0.2, 21)
    _run(ctx, [base])
    for staging in (0, 1, 2):
        for layout in (R.RIPPLE_SOA, R.RIPPLE_AOS):
            for v in range(3):
                R.ripple_batch_configure(ctx, layout=layout, tile_variant=v, staging=staging, solo_rounds=False)
                r = R.euler_request(base["input"], 21, base["dx"])
                _run(ctx, [r])
                # tile shape, layout and halo staging change no arithmetic
                assert np.array_equal(r["output"], base["output"]), (staging, layout, v)
    R.ripple_batch_configure(ctx, solo_rounds=False)


def test_budget_admission_waits_for_memory():
    c = R.ripple_ctx_create(0, 24 << 20)  # 24 MiB: about two 512^2 FP32 instances at once
    try:
        reqs = [_euler(512, 512, 0.1 + 0.02 * i, 20) for i in range(6)]
        infos = _run(c, reqs)
        assert all(i["status"] == R.RIPPLE_OK for i in infos)
        # some request had to wait for an earlier one to finish before admission
        finishes = sorted(i["finish_s"] for i in infos)
        assert max(i["admit_s"] for i in infos) >= finishes[0]
        for req in reqs[:2]:
            assert_parity(req["output"], _oracle_euler(req), 2e-5, LINF_F32)
        # a request that can never fit fails with RIPPLE_ERR_BUDGET
        big = _euler(2048, 2048, 0.1, 1)
        info = _run(c, [big])[0]
        assert info["status"] == R.RIPPLE_ERR_BUDGET
    finally:
        R.ripple_ctx_destroy(c)


def test_requests_arriving_while_others_run(ctx):
    R.ripple_batch_configure(ctx, steps_per_sync=2, solo_rounds=False)
    first = [_euler(256, 256, 0.2, 3000), _eik(300, 300, 8)]
    t_first = R.ripple_batch_submit(ctx, first)
    time.sleep(0.005)
    late = [_euler(64, 48, 0.15, 20), _eik(80, 60, 9)]
    t_late = R.ripple_batch_submit(ctx, late)
    info_late = [R.ripple_wait(ctx, t, 120000) for t in t_late]
    info_first = [R.ripple_wait(ctx, t, 120000) for t in t_first]
    assert all(i["status"] == R.RIPPLE_OK for i in info_first + info_late)
    # the small late Euler request ran and finished while the long first one was resident
    assert info_late[0]["start_s"] < info_first[0]["finish_s"]
    assert info_late[0]["finish_s"] < info_first[0]["finish_s"]
    assert_parity(late[0]["output"], _oracle_euler(late[0]), 2e-5, LINF_F32)
    ref = oracle.eikonal_fmm(late[1]["input"].astype(np.float64), late[1]["h"], late[1]["sources"])
    assert_parity(late[1]["output"][None], ref[None], 1e-4, LINF_EIK)
    # the long one equals the same problem on the single-field path
    f = R.ripple_field_create(ctx, (256, 256), 4, R.RIPPLE_SOA, 1, R.RIPPLE_F32)
    try:
        R.ripple_field_upload(f, first[0]["input"])
        R.ripple_fv_step(f, R.make_fv_params(first[0]["dx"]), 3000)
        single = R.ripple_field_download(f)
    finally:
        R.ripple_field_destroy(f)
    assert rel_l1(first[0]["output"], single) <= 1e-5
    assert max_rel(first[0]["output"], single) <= 1e-4  # 3000 steps of another kernel's rounding
    stats = R.ripple_batch_get_stats(ctx)
    assert stats["completed"] == 4 and stats["failed"] == 0


def test_poll_and_unknown_ticket(ctx):
    t = R.ripple_batch_submit(ctx, [_euler(40, 40, 0.2, 200)])[0]
    seen_not_ready = R.ripple_poll(ctx, t) is None
    info = R.ripple_wait(ctx, t, 60000)
    assert info["status"] == R.RIPPLE_OK
    assert seen_not_ready or info["finish_s"] > 0
    with pytest.raises(R.RippleError) as ei:
        R.ripple_poll(ctx, t)  # retired
    assert ei.value.status == R.RIPPLE_ERR_INVALID


def test_numeric_error_reported_per_request(ctx):
    bad = _euler(40, 40, 0.2, 5)
    bad["input"][3, 10, 10] = -1.0  # negative energy -> negative pressure
    good = _euler(40, 40, 0.2, 5)
    infos = _run(ctx, [bad, good])
    assert infos[0]["status"] == R.RIPPLE_ERR_NUMERIC
    assert infos[1]["status"] == R.RIPPLE_OK


def test_autotune_picks_a_candidate(ctx):
    sides = [s for s, _ in inputs.batch_problems(32, seed=2)]
    cfg, timings = R.ripple_batch_autotune(ctx, sides)
    assert cfg["layout"] in (R.RIPPLE_SOA, R.RIPPLE_AOS) and 0 <= cfg["tile_variant"] < 3
    assert cfg["staging"] in (0, 1, 2)
    assert len(timings) == 18 and all(v > 0 for v in timings.values())
    assert timings[(cfg["layout"], cfg["tile_variant"], cfg["staging"])] == min(timings.values())
