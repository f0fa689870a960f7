"""Benchmark of the stencil-sweep hot path on GB300.

Headline workload: 3D compressible Euler, FP32 stencil (FP64 dt and totals),
256^3 cells, 5 conserved variables, MUSCL-Hancock with minmod slopes and
Rusanov faces, halo 2, transmissive boundaries, spherical blast with 1 %
seeded noise on rho (synthetic, seeded).  One benchmark step = one explicit
time step of the whole field (one sweep launch: padding fill, staging,
reconstruction, predictor, face fluxes, conservative update, CFL reduction).
Metric: cell-updates/s (higher is better).  Inputs (335 MB per buffer) are
larger than the 129 MB L2, so no flush is needed between steps.

Also reported (secondary objects on the same JSON line): the AoS layout, the
2D FP64 128^2 workload, the FIM eikonal solves (2048^2 and 192^3), the
end-to-end solve through host buffers, the FP64 CPU oracle baseline, the
roofline of the sweep kernel and the SM clocks during the timed region.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
For N > 1 launch with torch.distributed.run: every rank runs an independent
replica of the workload on its own GPU (the path is one GPU per problem),
value = all ranks' cell-updates / max-over-ranks time.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import inputs  # noqa: E402

N3 = 256
NSTEPS_SOLVE = 50
BYTES_PER_CELL_UPDATE = 40  # FP32, 5 components: 20 B read + 20 B written per cell per step
# DRAM bytes per cell update of the sweep kernel (the row kernel, SoA) as measured by ncu
# (dram__bytes_read.sum + dram__bytes_write.sum of one 256x256x128 launch, divided by its cells);
# traffic scales with the cells of a launch.  Re-measure whenever the kernel changes.
DRAM_BYTES_PER_CELL_UPDATE = (216594688 + 137211392) / (256 * 256 * 128)
METRIC = "cell-updates/s"
ACTIVE_CELLS = 4 << 20  # serving: per-step cell budget of stepped Euler problems


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            pk = json.load(f)
        return float(pk["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi sampling of SM clocks / throttle reasons during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int, period_ms: int = 200):
        self.device = device
        self.period_ms = period_ms
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", str(self.period_ms)],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        self.out = ""
        if self.proc is not None:
            time.sleep(0.2)
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        rows = []
        for line in (self.out or "").strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append(dict(sm=float(parts[1]), smax=float(parts[2]), power=float(parts[3]),
                                 hw=parts[5], hwt=parts[6], swt=parts[7], pcap=parts[8]))
            except ValueError:
                continue
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        reasons = set()
        for r in rows:
            if r["hw"] == "Active":
                reasons.add("hw_slowdown")
            if r["hwt"] == "Active":
                reasons.add("hw_thermal_slowdown")
            if r["swt"] == "Active":
                reasons.add("sw_thermal_slowdown")
            if r["pcap"] == "Active":
                reasons.add("sw_power_cap")
        return {"sm_mhz": float(np.median([r["sm"] for r in rows])), "sm_max_mhz": max(r["smax"] for r in rows),
                "reasons": sorted(reasons), "samples": len(rows),
                "power_w_max": max(r["power"] for r in rows)}


# Thread instructions per Godunov update of the FIM solve kernels, from one ncu
# capture of each solve (smsp__inst_executed.sum x 32 / the solve's Godunov
# updates); the eikonal roofline is issue-bound, so these set its achieved
# rate.  Re-measure whenever the kernels change.
FIM_INSTR_PER_UPDATE = {"2d_2048": 38.44, "3d_192": 85.87}


def eikonal_roofline(name, updates_per_s, clocks, sms):
    """Issue roofline of the FIM solve: thread instructions per second against
    the SMs' issue rate (4 schedulers x 32 lanes per SM per clock, at the
    median SM clock sampled during the solves)."""
    mhz = clocks.get("sm_mhz") or 2070.0
    peak = sms * 128 * mhz * 1e6
    ipu = FIM_INSTR_PER_UPDATE.get(name)
    out = {"bound": "issue", "peak": peak / 1e12, "unit": "T thread-instructions/s",
           "peak_source": f"{sms} SMs x 128 lanes x {mhz:.0f} MHz (sampled)",
           "instructions_per_update": ipu}
    if ipu is None:
        out.update(achieved=None, frac=None)
    else:
        out.update(achieved=ipu * updates_per_s / 1e12, frac=ipu * updates_per_s / peak)
    return out


def host_description():
    """Host cores and CPU model of the machine the oracle runs on."""
    model = None
    try:
        txt = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in txt.splitlines():
            if line.lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if model is None:
        import platform
        model = platform.processor() or platform.machine()
    return {"nproc": os.cpu_count(), "cpu_model": model}


def dist_setup(n_gpus):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        dist.init_process_group(backend=backend)
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def allreduce_max(value, world):
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def bench_gpu(args, rank, world, local):
    import torch

    import paper_2104_08571_gb300 as R

    torch.cuda.set_device(local)
    ctx = R.ripple_ctx_create(local)
    R.use_torch_allocator(ctx, local)
    stream = torch.cuda.Stream(device=local)
    R.ripple_set_stream(ctx, stream)
    MUSCL, TRA = R.RIPPLE_MUSCL_HANCOCK_MINMOD, R.RIPPLE_BC_TRANSMISSIVE
    dims = tuple(args.sweep_dims)
    ncell = int(np.prod(dims))
    prm = R.make_fv_params([1.0 / N3] * 3, scheme=MUSCL, bc=TRA)
    U0 = inputs.euler3d_blast(N3, seed=1, dims=dims).astype(np.float32)
    U0_dev = torch.from_numpy(U0).to(f"cuda:{local}")
    U0_dev_aos = torch.from_numpy(np.ascontiguousarray(np.moveaxis(U0, 0, -1))).to(f"cuda:{local}")
    result = {}

    def timed_steps(field, k, w, per_step=None):
        """W warm-up steps, then K steps, each bracketed by CUDA events on the
        library's stream: returns the total of the K steps (ms); the K per-step
        times go to per_step."""
        for _ in range(w):
            R.ripple_fv_step(field, prm, 1, stats=False)
        torch.cuda.synchronize()
        barrier(world)
        torch.cuda.synchronize()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(k + 1)]
        ev[0].record(stream)
        for i in range(k):
            R.ripple_fv_step(field, prm, 1, stats=False)
            ev[i + 1].record(stream)
        torch.cuda.synchronize()
        ms = ev[0].elapsed_time(ev[k])
        if per_step is not None:
            per_step.extend(ev[i].elapsed_time(ev[i + 1]) for i in range(k))
        barrier(world)
        return ms

    # ---- headline: SoA, inputs resident in HBM ----
    f = R.ripple_field_create(ctx, dims, 5, R.RIPPLE_SOA, 2, R.RIPPLE_F32)
    if args.sweep_only and args.sweep_variant >= 0:
        R.ripple_field_set_sweep(f, args.sweep_variant, 0)
    R.ripple_field_upload(f, U0_dev, R.RIPPLE_SOA)
    R.ripple_fv_step(f, prm, 1, stats=False)  # first call: second buffer, prep, tensor maps
    torch.cuda.synchronize()
    per_step = []
    with ClockSampler(local) as clk:
        ms = timed_steps(f, args.steps, args.warmup, per_step)
    clocks = clk.summary()
    result["per_step_ms"] = per_step
    ms_max = allreduce_max(ms, world)
    st = R.ripple_fv_step(f, prm, 0)  # synchronous error check + totals of the final state
    result["soa_ms_per_step"] = ms / args.steps
    result["soa_totals_mass"] = st["totals"][0]
    # parity data (checked against the oracle in the CPU leg): the state after the
    # timed steps and one more GPU step of it at seeded sampled cells
    par = {}
    if rank == 0 and not args.skip_cpu_baseline and not args.sweep_only:
        Un = R.ripple_field_download(f)
        st1 = R.ripple_fv_step(f, prm, 1)
        cells = np.random.default_rng(7).choice(ncell, 4096, replace=False)
        par["headline"] = dict(Un=Un, cells=cells, gpu=R.ripple_field_download(f).reshape(5, -1)[:, cells].T,
                               dt=st1["dt_last"], dx=[1.0 / N3] * 3)
    R.ripple_field_destroy(f)
    if "headline" in par:
        # the whole field after a full 50-step run of the headline scheme at 128^3
        # (SoA, the headline kernel), for the oracle's 50-step run of the same state
        n1 = 128
        U1 = inputs.euler3d_blast(n1, seed=1).astype(np.float32)
        f1 = R.ripple_field_create(ctx, (n1, n1, n1), 5, R.RIPPLE_SOA, 2, R.RIPPLE_F32)
        R.ripple_field_upload(f1, U1)
        prm1 = R.make_fv_params([1.0 / n1] * 3, scheme=MUSCL, bc=TRA)
        st50 = R.ripple_fv_step(f1, prm1, NSTEPS_SOLVE)
        par["full_run_128"] = dict(U0=U1, gpu=R.ripple_field_download(f1), t=st50["t"], n=n1)
        R.ripple_field_destroy(f1)
    hbm_peak, peak_kind = load_peaks()
    achieved = BYTES_PER_CELL_UPDATE * ncell / (ms / args.steps / 1e3) / 1e9
    if args.sweep_only:
        R.ripple_ctx_destroy(ctx)
        return dict(value=world * args.steps * ncell / (ms_max / 1e3), ms_per_step=ms_max / args.steps,
                    clocks=clocks, achieved=achieved, hbm_peak=hbm_peak, peak_kind=peak_kind)

    # ---- AoS layout, same workload ----
    fa = R.ripple_field_create(ctx, dims, 5, R.RIPPLE_AOS, 2, R.RIPPLE_F32)
    R.ripple_field_upload(fa, U0_dev_aos, R.RIPPLE_AOS)
    R.ripple_fv_step(fa, prm, 1, stats=False)
    torch.cuda.synchronize()
    per_step_aos = []
    with ClockSampler(local) as clk_aos:
        ms_aos = timed_steps(fa, args.steps, args.warmup, per_step_aos)
    result["aos_per_step_ms"] = per_step_aos
    result["aos_clocks"] = clk_aos.summary()
    R.ripple_fv_step(fa, prm, 0)
    R.ripple_field_destroy(fa)

    # ---- end to end: full 50-step solves from pinned host memory to host memory ----
    pin_in = torch.from_numpy(U0).pin_memory()
    pin_out = torch.empty_like(pin_in).pin_memory()
    fe = R.ripple_field_create(ctx, dims, 5, R.RIPPLE_SOA, 2, R.RIPPLE_F32)
    e2e_solves = max(1, args.e2e_solves)

    def one_solve():
        R.ripple_field_upload(fe, pin_in.numpy(), R.RIPPLE_SOA)
        R.ripple_fv_step(fe, prm, NSTEPS_SOLVE, stats=False)
        R.ripple_field_download(fe, R.RIPPLE_SOA, out=pin_out)

    one_solve()  # warm-up
    torch.cuda.synchronize()
    barrier(world)
    with ClockSampler(local) as clk_e2e:
        t0 = time.perf_counter()
        for _ in range(e2e_solves):
            one_solve()
        torch.cuda.synchronize()
        e2e_s = allreduce_max(time.perf_counter() - t0, world)
    result["e2e_clocks"] = clk_e2e.summary()
    R.ripple_field_destroy(fe)
    e2e_value = world * e2e_solves * NSTEPS_SOLVE * ncell / e2e_s

    # ---- secondary: 2D FP64 128^2 periodic Rusanov, 100 steps (latency bound) ----
    U2 = inputs.euler2d_sine(128)
    f2 = R.ripple_field_create(ctx, (128, 128), 4, R.RIPPLE_SOA, 1, R.RIPPLE_F64)
    prm2 = R.make_fv_params([1.0 / 128] * 2)
    R.ripple_field_upload(f2, U2)
    R.ripple_fv_step(f2, prm2, 100)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk2:
        e0.record(stream)
        R.ripple_fv_step(f2, prm2, 100, stats=False)
        e1.record(stream)
        torch.cuda.synchronize()
    ms2 = e0.elapsed_time(e1)
    result["euler2d_clocks"] = clk2.summary()
    R.ripple_fv_step(f2, prm2, 0)
    if "headline" in par:  # 100 steps from the initial state, for the oracle comparison
        R.ripple_field_upload(f2, U2)
        R.ripple_fv_step(f2, prm2, 100)
        par["euler2d_fp64_128"] = dict(U0=U2, gpu=R.ripple_field_download(f2))
    R.ripple_field_destroy(f2)

    # ---- secondary: eikonal FIM solves ----
    eik = {}
    if not args.skip_eikonal:
        eik = bench_eikonal(R, torch, local, keep=par if "headline" in par else None, ctx=ctx, stream=stream)

    R.ripple_ctx_destroy(ctx)
    batched = None if args.skip_batched else bench_batched(R, torch, local, keep=par if "headline" in par else None)
    serve = None if args.skip_serve else bench_serving(R, torch, local, count=args.serve_requests)
    solo = bench_solo(R, torch, local)
    layout = None if args.skip_layout else bench_layout(R, torch, local)
    force = bench_force_split(R, torch, local, par=par if "headline" in par else None)
    value = world * args.steps * ncell / (ms_max / 1e3)
    return dict(value=value, ms_per_step=ms_max / args.steps, clocks=clocks, ms_aos=ms_aos / args.steps,
                e2e_value=e2e_value, e2e_s=e2e_s, e2e_solves=e2e_solves, ms2=ms2, eik=eik,
                achieved=achieved, hbm_peak=hbm_peak, peak_kind=peak_kind, extra=result, batched=batched, solo=solo,
                serve=serve, layout=layout, force=force, parity_data=par)


def bench_eikonal(R, torch, local, keep=None, ctx=None, stream=None, steps=5):
    """FIM eikonal solves, FP32: 2048^2 and 192^3, seeded smoothed-Gaussian
    slowness, 1-4 seeded sources, tol 1e-6.  Each solve is timed between CUDA
    events on the library's stream; the median of `steps` solves is reported."""
    own = ctx is None
    if own:
        ctx = R.ripple_ctx_create(local)
        R.use_torch_allocator(ctx, local)
        stream = torch.cuda.Stream(device=local)
        R.ripple_set_stream(ctx, stream)
    eik = {}
    try:
        for name, edims in (("2d_2048", (2048, 2048)), ("3d_192", (192, 192, 192))):
            s = inputs.eikonal_slowness(edims, seed=1).astype(np.float32)
            src = inputs.eikonal_sources(edims, seed=1)
            fs = R.ripple_field_create(ctx, edims, 1, R.RIPPLE_SOA, 0, R.RIPPLE_F32)
            ft = R.ripple_field_create(ctx, edims, 1, R.RIPPLE_SOA, 1, R.RIPPLE_F32)
            R.ripple_field_upload(fs, s)
            R.ripple_eikonal_solve(fs, ft, src, 1.0 / edims[0], 1e-6)  # warm-up
            torch.cuda.synchronize()
            times = []
            with ClockSampler(local) as clk_e:
                for _ in range(max(1, steps)):
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    est = R.ripple_eikonal_solve(fs, ft, src, 1.0 / edims[0], 1e-6)
                    e1.record(stream)
                    torch.cuda.synchronize()
                    times.append(e0.elapsed_time(e1) / 1e3)
            dt = float(np.median(times))
            ncells = int(np.prod(edims))
            eik[name] = {"solve_ms": dt * 1e3, "solve_ms_min_max": [min(times) * 1e3, max(times) * 1e3],
                         "solves": len(times), "solved_cells_per_s": ncells / dt,
                         "godunov_updates_per_s": est["cell_updates"] / dt, "iterations": est["iterations"],
                         "tile_visits": est["tile_visits"], "sources": len(src),
                         "roofline": eikonal_roofline(name, est["cell_updates"] / dt, clk_e.summary(),
                                                      torch.cuda.get_device_properties(local).multi_processor_count),
                         "clocks": clk_e.summary()}
            if keep is not None:
                keep["eikonal_" + name] = dict(s=s, src=src, h=1.0 / edims[0], gpu=R.ripple_field_download(ft))
            R.ripple_field_destroy(fs)
            R.ripple_field_destroy(ft)
    finally:
        if own:
            R.ripple_ctx_destroy(ctx)
    return eik


def bench_solo(R, torch, local, sides=(64, 256, 1024), nsteps=400):
    """One 2D Euler request (sine density, FP32, periodic Rusanov, 400 steps)
    served alone, per side: on the multi-step solo solver (solo rounds), on the
    batched step launched once per step (solo rounds off; the results must be
    the same bits), and through the single-field API's per-step launch loop
    on a device-resident field."""
    out = {}
    ctx = R.ripple_ctx_create(local)
    clk = ClockSampler(local).__enter__()
    try:
        for side in sides:
            U = inputs.euler2d_sine(side).astype(np.float32)
            row, res = {}, {}
            for mode, solo in (("solo_rounds", True), ("batched_per_step", False)):
                R.ripple_batch_configure(ctx, steps_per_sync=16, use_graphs=True, solo_rounds=solo)
                for _ in range(3):  # warm-up twice, then timed
                    req = R.euler_request(U, nsteps, [1.0 / side] * 2)
                    s0 = R.ripple_batch_get_stats(ctx)
                    info = R.ripple_wait(ctx, R.ripple_batch_submit(ctx, [req])[0], 600000)
                    s1 = R.ripple_batch_get_stats(ctx)
                assert info["status"] == R.RIPPLE_OK, "solo leg failed"
                row[mode] = {"us_per_step_device": (s1["device_s"] - s0["device_s"]) * 1e6 / nsteps,
                             "latency_ms": (info["finish_s"] - info["submit_s"]) * 1e3,
                             "launches": s1["launches"] - s0["launches"]}
                res[mode] = req["output"]
            row["bitwise_equal"] = bool(np.array_equal(res["solo_rounds"], res["batched_per_step"]))
            f = R.ripple_field_create(ctx, (side, side), 4, R.RIPPLE_SOA, 1, R.RIPPLE_F32)
            try:
                R.ripple_field_upload(f, U)
                prm = R.make_fv_params([1.0 / side] * 2)
                R.ripple_fv_step(f, prm, 10, stats=False)
                R.ripple_ctx_sync(ctx)
                t0 = time.perf_counter()
                R.ripple_fv_step(f, prm, nsteps, stats=False)
                R.ripple_ctx_sync(ctx)
                row["field_api_per_step_launches"] = {"us_per_step": (time.perf_counter() - t0) * 1e6 / nsteps}
            finally:
                R.ripple_field_destroy(f)
            out[str(side)] = row
    finally:
        clk.__exit__(None, None, None)
        R.ripple_ctx_destroy(ctx)
    out["steps"] = nsteps
    out["clocks"] = clk.summary()
    return out


def bench_batched(R, torch, local, nsteps=100, count=512, keep=None):
    """512 independent 2D Euler problems (sides log-uniform in [32, 512], FP32,
    sine density with per-instance amplitude, periodic Rusanov, 100 steps):
    one batched launch per global step (autotuned layout and tile shape, CUDA
    graphs) against the per-instance launch loop on the same GPU."""
    probs = inputs.batch_problems(count, seed=1)
    pageable = [inputs.euler2d_sine(side, amp=amp).astype(np.float32) for side, amp in probs]

    def pinned(a):
        t = torch.empty(a.shape, dtype=torch.float32, pin_memory=True)
        t.numpy()[...] = a
        return t.numpy()

    # requests read and write page-locked host arrays (the end-to-end form);
    # the pageable form is timed once beside it
    states = [pinned(a) for a in pageable]
    outs = [pinned(a) for a in pageable]
    sides = [side for side, _ in probs]
    cells = float(sum(side * side for side in sides))
    ctx = R.ripple_ctx_create(local)
    try:
        cfg, timings = R.ripple_batch_autotune(ctx, sides)
        R.ripple_batch_configure(ctx, layout=cfg["layout"], tile_variant=cfg["tile_variant"],
                                 steps_per_sync=nsteps, use_graphs=True, staging=cfg["staging"])

        def run_batch(src=None, dst=None):
            src = states if src is None else src
            dst = outs if dst is None else dst
            reqs = [R.euler_request(U, nsteps, [1.0 / U.shape[2], 1.0 / U.shape[1]], out=o) for U, o in zip(src, dst)]
            t0 = time.perf_counter()
            tickets = R.ripple_batch_submit(ctx, reqs)
            infos = [R.ripple_wait(ctx, t, 600000) for t in tickets]
            dt = time.perf_counter() - t0
            assert all(i["status"] == R.RIPPLE_OK for i in infos), "batched run failed"
            return reqs, infos, dt

        run_batch()  # warm-up: table capacities, graph capture
        st0 = R.ripple_batch_get_stats(ctx)
        with ClockSampler(local) as clk_b:
            reqs, infos, t_batch = run_batch()
        st1 = R.ripple_batch_get_stats(ctx)
        host_ms = {k: 1e3 * (st1[k] - st0[k]) for k in ("host_admit_s", "host_round_s", "host_finish_s")}
        kept = [np.array(r["output"]) for r in reqs]
        outs_p = [np.empty_like(a) for a in pageable]
        run_batch(pageable, outs_p)
        _, _, t_pageable = run_batch(pageable, outs_p)
        if keep is not None:  # four instances (the smallest, two middle, the largest) for the oracle
            order = np.argsort(sides)
            pick = [int(order[0]), int(order[count // 3]), int(order[2 * count // 3]), int(order[-1])]
            keep["batched"] = [dict(U0=pageable[i], gpu=kept[i], side=sides[i]) for i in pick]
        span = max(i["finish_s"] for i in infos) - min(i["start_s"] for i in infos)
        dev_s = st1["device_s"] - st0["device_s"]
        # dependency-driven rounds: the same batch in ONE persistent launch
        R.ripple_batch_configure(ctx, layout=cfg["layout"], tile_variant=cfg["tile_variant"],
                                 steps_per_sync=nsteps, use_graphs=True, staging=cfg["staging"], async_queue=True)
        run_batch()
        sa0 = R.ripple_batch_get_stats(ctx)
        with ClockSampler(local) as clk_a:
            reqs_a, infos_a, t_async = run_batch()
        sa1 = R.ripple_batch_get_stats(ctx)
        span_a = max(i["finish_s"] for i in infos_a) - min(i["start_s"] for i in infos_a)
        same = all(np.array_equal(x, y["output"]) for x, y in zip(kept, reqs_a))
        # uneven step counts (uniform in [nsteps/2, 3 nsteps/2], seeded): per-step
        # launches shrink each round to the shortest remaining problem
        steps_u = [int(nsteps // 2 + u * nsteps) for u in inputs.uniform(3, count, stream=6)]
        cells_u = float(sum(side * side * k for side, k in zip(sides, steps_u)))
        uneven = {}
        for mode in ("per_step_launches", "dependency_driven"):
            R.ripple_batch_configure(ctx, layout=cfg["layout"], tile_variant=cfg["tile_variant"],
                                     steps_per_sync=max(steps_u), use_graphs=True, staging=cfg["staging"],
                                     async_queue=mode == "dependency_driven")
            for rep_ in range(2):  # warm-up, then timed
                rq = [R.euler_request(U, k, [1.0 / U.shape[2], 1.0 / U.shape[1]], out=o)
                      for U, k, o in zip(states, steps_u, outs)]
                s0 = R.ripple_batch_get_stats(ctx)
                t0 = time.perf_counter()
                inf = [R.ripple_wait(ctx, t, 600000) for t in R.ripple_batch_submit(ctx, rq)]
                dt_u = time.perf_counter() - t0
                s1 = R.ripple_batch_get_stats(ctx)
            assert all(i["status"] == R.RIPPLE_OK for i in inf), "uneven batched run failed"
            sp = max(i["finish_s"] for i in inf) - min(i["start_s"] for i in inf)
            uneven[mode] = {"value": cells_u / dt_u, "value_compute_span": cells_u / sp,
                            "value_device": cells_u / (s1["device_s"] - s0["device_s"]),
                            "launches": s1["launches"] - s0["launches"],
                            "outputs": [np.array(r["output"]) for r in rq]}
        uneven_same = all(np.array_equal(x, y) for x, y in zip(uneven["per_step_launches"].pop("outputs"),
                                                               uneven["dependency_driven"].pop("outputs")))
        # per-instance launch loop over device-resident fields (no transfers timed)
        fields = []
        for U in states:
            f = R.ripple_field_create(ctx, (U.shape[2], U.shape[1]), 4, R.RIPPLE_SOA, 1, R.RIPPLE_F32)
            R.ripple_field_upload(f, U)
            fields.append(f)
        prms = [R.make_fv_params([1.0 / U.shape[2], 1.0 / U.shape[1]]) for U in states]
        for f, prm in zip(fields, prms):  # warm-up: second buffers, prep, tensor maps
            R.ripple_fv_step(f, prm, 0)
        for f, U in zip(fields, states):
            R.ripple_field_upload(f, U)
        torch.cuda.synchronize()
        with ClockSampler(local) as clk_l:
            t0 = time.perf_counter()
            for f, prm in zip(fields, prms):
                R.ripple_fv_step(f, prm, nsteps, stats=False)
            R.ripple_ctx_sync(ctx)
            t_loop = time.perf_counter() - t0
        worst = 0.0
        for f, out_b in zip(fields, kept):
            loop_out = R.ripple_field_download(f)
            a = np.abs(out_b.astype(np.float64) - loop_out).reshape(4, -1).sum(1)
            b = np.abs(loop_out.astype(np.float64)).reshape(4, -1).sum(1)
            worst = max(worst, float((a / b).max()))
            R.ripple_field_destroy(f)
    finally:
        R.ripple_ctx_destroy(ctx)
    return {
        "workload": f"{count} x 2D Euler FP32 Rusanov, sides log-uniform [32,512], {nsteps} steps",
        "instances": count, "total_cells": int(cells), "steps": nsteps,
        "value": cells * nsteps / t_batch, "unit": METRIC,
        "batched_seconds_end_to_end": t_batch,
        "host_arrays": "page-locked (pinned) inputs and outputs",
        "value_pageable_host_arrays": cells * nsteps / t_pageable,
        "scheduler_host_ms": host_ms,
        "clocks": clk_b.summary(), "clocks_dependency_driven": clk_a.summary(), "clocks_loop": clk_l.summary(),
        "batched_compute_span_s": span,
        "batched_value_compute_span": cells * nsteps / span,
        "launches": st1["launches"] - st0["launches"], "graph_replays": st1["graph_replays"] - st0["graph_replays"],
        "roofline": {"bound": "hbm", "achieved": 32.0 * cells * nsteps / dev_s / 1e9, "peak": load_peaks()[0],
                     "unit": "GB/s", "frac": 32.0 * cells * nsteps / dev_s / 1e9 / load_peaks()[0],
                     "algorithmic_bytes_per_cell_update": 32,
                     "timing": "GPU time of the compute rounds (CUDA events on the runtime's compute stream)"},
        "batched_value_device": cells * nsteps / dev_s,
        "dependency_driven_round": {
            "value": cells * nsteps / t_async, "value_compute_span": cells * nsteps / span_a,
            "value_device": cells * nsteps / (sa1["device_s"] - sa0["device_s"]),
            "launches": sa1["launches"] - sa0["launches"], "speedup_vs_per_step_launches": t_batch / t_async,
            "bitwise_equal_to_per_step_launches": same,
            "uneven_steps": dict(uneven, workload=f"same instances, steps uniform in [{nsteps // 2}, {3 * nsteps // 2}]",
                                 bitwise_equal=uneven_same,
                                 speedup=uneven["dependency_driven"]["value"] / uneven["per_step_launches"]["value"])},
        "per_instance_loop_value": cells * nsteps / t_loop, "per_instance_loop_seconds": t_loop,
        "per_instance_loop_launches": count * nsteps,
        "speedup_vs_loop": t_loop / t_batch,
        "max_rel_l1_vs_loop": worst,
        "autotune": {"layout": "SoA" if cfg["layout"] == R.RIPPLE_SOA else "AoS",
                     "tile": ["32x8", "8x32", "16x16"][cfg["tile_variant"]],
                     "staging": ["tma", "direct", "walk"][cfg["staging"]],
                     "ms_per_global_step": {
                         f"{['tma', 'direct', 'walk'][k[2]]}/{'SoA' if k[0] == R.RIPPLE_SOA else 'AoS'}/"
                         f"{['32x8', '8x32', '16x16'][k[1]]}": v for k, v in timings.items()}},
    }


def bench_force_split(R, torch, local, par=None, legs=None):
    """The paper's own Euler solver (dimensionally split sweeps, x then y [then
    z], FORCE face flux), one sweep launch per axis: 2D FP32 8192^2 periodic sine
    density (a Table flux size), 3D FP32 256^3 blast (the headline state,
    transmissive), and the 2D FP64 128^2 workload."""
    ctx = R.ripple_ctx_create(local)
    R.use_torch_allocator(ctx, local)
    stream = torch.cuda.Stream(device=local)
    R.ripple_set_stream(ctx, stream)
    out = {}
    try:
        if legs is None:
            legs = (("fp32_8192", 2, 8192, R.RIPPLE_F32, 20), ("fp32_3d_256", 3, 256, R.RIPPLE_F32, 10),
                    ("fp64_128", 2, 128, R.RIPPLE_F64, 100))
        for name, ndim, n, dtype, steps in legs:
            npdt = np.float32 if dtype == R.RIPPLE_F32 else np.float64
            if ndim == 2:
                U0 = inputs.euler2d_sine(n).astype(npdt)
                bc = R.RIPPLE_BC_PERIODIC
            else:
                U0 = inputs.euler3d_blast(n, seed=1).astype(npdt)
                bc = R.RIPPLE_BC_TRANSMISSIVE
            nc = ndim + 2
            f = R.ripple_field_create(ctx, (n,) * ndim, nc, R.RIPPLE_SOA, 1, dtype)
            prm = R.make_fv_params([1.0 / n] * ndim, scheme=R.RIPPLE_FORCE_SPLIT, bc=bc)
            R.ripple_field_upload(f, U0)
            R.ripple_fv_step(f, prm, 3)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            with ClockSampler(local) as clk_f:
                e0.record(stream)
                R.ripple_fv_step(f, prm, steps, stats=False)
                e1.record(stream)
                torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / steps
            R.ripple_fv_step(f, prm, 0)
            es = nc * (4 if dtype == R.RIPPLE_F32 else 8)
            cells = n ** ndim
            gbs = ndim * 2 * es * cells / (ms / 1e3) / 1e9  # each sweep reads and writes the state
            out[name] = {"cells": cells, "ms_per_step": ms, "cell_updates_per_s": cells / (ms / 1e3),
                         "launches_per_step": ndim, "algorithmic_bytes_per_cell_update": ndim * 2 * es,
                         "GB_s_algorithmic": gbs, "hbm_frac": gbs / load_peaks()[0], "clocks": clk_f.summary()}
            if name == "fp32_8192":
                out[name]["paper_v100_flux_difference_ms_8k"] = {"ripple_s": 3.5533, "ripple_c": 5.5284,
                                                                   "kokkos": 12.919}
            if name == "fp64_128" and par is not None:
                R.ripple_field_upload(f, U0)
                R.ripple_fv_step(f, prm, 100)
                par["force_split_fp64_128"] = dict(U0=U0, gpu=R.ripple_field_download(f))
            R.ripple_field_destroy(f)
        if par is not None:
            # the 3D FP32 split step on the walk sweeps: the whole 128^3 blast after
            # 10 steps, for the oracle's run of the same state
            n1 = 128
            U1 = inputs.euler3d_blast(n1, seed=1).astype(np.float32)
            f = R.ripple_field_create(ctx, (n1,) * 3, 5, R.RIPPLE_SOA, 1, R.RIPPLE_F32)
            R.ripple_field_upload(f, U1)
            R.ripple_fv_step(f, R.make_fv_params([1.0 / n1] * 3, scheme=R.RIPPLE_FORCE_SPLIT,
                                                 bc=R.RIPPLE_BC_TRANSMISSIVE), 10)
            par["force_split_fp32_3d_128"] = dict(U0=U1, gpu=R.ripple_field_download(f), n=n1)
            R.ripple_field_destroy(f)
    finally:
        R.ripple_ctx_destroy(ctx)
    return out


def bench_layout(R, torch, local, n_saxpy=1 << 30, n_particles=80_000_000, reps=10):
    """Section 7.1 SAXPY (1 G elements) and Section 7.2 particle update (80 M
    particles) in both layouts, read directly or staged through shared memory
    by bulk copies; CUDA-event times on the library's stream, inputs far larger
    than L2.  The paper's V100 times of the same sizes are quoted as context."""
    ctx = R.ripple_ctx_create(local)
    stream = torch.cuda.Stream(device=local)
    R.ripple_set_stream(ctx, stream)
    peak = load_peaks()[0]
    out = {}

    def timed(fn):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        st = R.ripple_ctx_sync(ctx)
        return e0.elapsed_time(e1) / reps

    clk_lay = ClockSampler(local).__enter__()
    try:
        x = torch.rand(n_saxpy, device=f"cuda:{local}")
        y = torch.rand(n_saxpy, device=f"cuda:{local}")
        torch.cuda.synchronize()
        ms = timed(lambda: R.ripple_saxpy(ctx, 1.0001, x, y))
        gbs = 12.0 * n_saxpy / (ms / 1e3) / 1e9
        out["saxpy"] = {"elements": n_saxpy, "ms": ms, "GB_s": gbs, "hbm_frac": gbs / peak,
                        "bytes_per_element": 12, "paper_v100_ms_1e9": {"ripple": 15.048, "cublas": 14.556}}
        del x, y
        p = torch.rand(6 * n_particles, device=f"cuda:{local}")
        torch.cuda.synchronize()
        out["particle_update"] = {"particles": n_particles, "bytes_per_particle": 36,
                                  "note": "AoS stores whole 24-byte records back (48 B moved per particle)",
                                  "paper_v100_ms_80M": {"s": 6.7914, "c": 11.452, "ss": 9.3259, "cs": 16.3081}}
        for name, layout, staged in (("soa", R.RIPPLE_SOA, False), ("aos", R.RIPPLE_AOS, False),
                                     ("soa_staged", R.RIPPLE_SOA, True), ("aos_staged", R.RIPPLE_AOS, True)):
            ms = timed(lambda: R.ripple_particle_update(ctx, p, 1e-3, layout=layout, staged=staged))
            gbs = 36.0 * n_particles / (ms / 1e3) / 1e9
            out["particle_update"][name] = {"ms": ms, "GB_s": gbs, "hbm_frac": gbs / peak}
        del p
    finally:
        clk_lay.__exit__(None, None, None)
        R.ripple_ctx_destroy(ctx)
    out["clocks"] = clk_lay.summary()
    return out


def _serve_requests(R, reqs_spec):
    out = []
    for r in reqs_spec:
        side = r["side"]
        if r["kind"] == "euler":
            U = inputs.euler2d_sine(side, amp=r["amp"]).astype(np.float32)
            out.append((r, U, None))
        else:
            s = inputs.eikonal_slowness((side, side), seed=r["seed"]).astype(np.float32)
            src = inputs.eikonal_sources((side, side), seed=r["seed"], count=r["nsrc"])
            out.append((r, s, src))
    return out


def _make_req(R, r, data, src):
    side = r["side"]
    if r["kind"] == "euler":
        return R.euler_request(data, r["steps"], [1.0 / side, 1.0 / side])
    return R.eikonal_request(data, src, 1.0 / side, tol=1e-6)


SERVE_RATES = (50, 100, 200, 500, 1000, 2000)
# The served runs are timed in real time; an nvidia-smi query of the clocks
# and throttle reasons stalls the runtime's CUDA calls while it runs, so the
# serving legs sample every 2 s (the kernel legs every 200 ms)
SERVE_CLOCK_PERIOD_MS = 2000


def bench_serving(R, torch, local, rates=SERVE_RATES, count=400):
    """Poisson arrivals of mixed requests (70 % 2D Euler side log-U[64,1024],
    50-500 steps; 30 % 2D eikonal side log-U[128,1024], 1-4 sources) under a
    40 GB budget.  Latency = submit -> result in host memory.  Baseline: the
    same arrival stream served one request at a time through the single-field
    API (service times measured here, queue replayed)."""
    spec_all = inputs.serve_stream(1.0, count, seed=1)
    prepared = _serve_requests(R, spec_all)
    work_euler = sum(r["side"] ** 2 * r["steps"] for r in spec_all if r["kind"] == "euler")
    cells_eik = sum(r["side"] ** 2 for r in spec_all if r["kind"] == "eikonal")
    result = {"requests_per_rate": count, "mix": "70% Euler / 30% eikonal", "budget_gb": 40,
              "policy": f"least remaining work first, {ACTIVE_CELLS} active cells per step, 4 FIM iterations per step",
              "euler_cell_updates": int(work_euler), "eikonal_cells": int(cells_eik), "rates": {}}
    # sequential baseline: service time of every request alone, through fields
    # (under the clock sampler, as the served runs)
    clk_seq = ClockSampler(local, SERVE_CLOCK_PERIOD_MS).__enter__()
    ctx = R.ripple_ctx_create(local)
    R.use_torch_allocator(ctx, local)  # cached allocations: no cudaMalloc per request
    service = []
    try:
        for (r, data, src) in prepared:
            side = r["side"]
            t0 = time.perf_counter()
            if r["kind"] == "euler":
                f = R.ripple_field_create(ctx, (side, side), 4, R.RIPPLE_SOA, 1, R.RIPPLE_F32)
                R.ripple_field_upload(f, data)
                R.ripple_fv_step(f, R.make_fv_params([1.0 / side] * 2), r["steps"], stats=False)
                R.ripple_field_download(f)
                R.ripple_field_destroy(f)
            else:
                fs = R.ripple_field_create(ctx, (side, side), 1, R.RIPPLE_SOA, 0, R.RIPPLE_F32)
                ft = R.ripple_field_create(ctx, (side, side), 1, R.RIPPLE_SOA, 1, R.RIPPLE_F32)
                R.ripple_field_upload(fs, data)
                R.ripple_eikonal_solve(fs, ft, src, 1.0 / side, 1e-6)
                R.ripple_field_download(ft)
                R.ripple_field_destroy(fs)
                R.ripple_field_destroy(ft)
            service.append(time.perf_counter() - t0)
    finally:
        R.ripple_ctx_destroy(ctx)
        clk_seq.__exit__(None, None, None)
    result["baseline_clocks"] = clk_seq.summary()
    ctx = R.ripple_ctx_create(local, 40 << 30)
    try:
        for mode in ("per_step_launches", "dependency_driven"):
            R.ripple_batch_configure(ctx, steps_per_sync=8, use_graphs=True, active_cells=ACTIVE_CELLS,
                                     async_queue=mode == "dependency_driven")
            warm = [_make_req(R, r, d, s) for (r, d, s) in prepared[:8]]
            for t in R.ripple_batch_submit(ctx, warm):
                R.ripple_wait(ctx, t, 600000)
            dest = result["rates"] if mode == "per_step_launches" else result.setdefault("rates_dependency_driven", {})
            for rate in rates:
                with ClockSampler(local, SERVE_CLOCK_PERIOD_MS) as clk_s:
                    arrivals = [r["t"] for r in inputs.serve_stream(rate, count, seed=1)]
                    reqs = [_make_req(R, r, d, s) for (r, d, s) in prepared]
                    tickets, done = [], {}
                    t0 = time.perf_counter()
                    head = 0  # oldest ticket not yet collected
                    for a, req in zip(arrivals, reqs):
                        # a client collects finished results while it waits for
                        # its next request (oldest first, as they mostly finish)
                        while True:
                            while head < len(tickets) and tickets[head] in done:
                                head += 1
                            if head == len(tickets) or t0 + a - time.perf_counter() < 2e-4:
                                break
                            info = R.ripple_poll(ctx, tickets[head])
                            if info is None:
                                break
                            done[tickets[head]] = info
                        delay = t0 + a - time.perf_counter()
                        if delay > 0:
                            time.sleep(delay)
                        tickets.append(R.ripple_batch_submit(ctx, [req])[0])
                    infos = [done[t] if t in done else R.ripple_wait(ctx, t, 600000) for t in tickets]
                    makespan = time.perf_counter() - t0
                ok = sum(1 for i in infos if i["status"] == R.RIPPLE_OK)
                lat = np.array([i["finish_s"] - i["submit_s"] for i in infos]) * 1e3
                # baseline queue: one request at a time in arrival order
                clock, blat = 0.0, []
                for a, svc in zip(arrivals, service):
                    clock = max(clock, a) + svc
                    blat.append((clock - a) * 1e3)
                blat = np.array(blat)
                base_makespan = clock
                dest[str(rate)] = {
                    "completed": ok, "makespan_s": makespan,
                    "cell_updates_per_s": work_euler / makespan, "eikonal_cells_per_s": cells_eik / makespan,
                    "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                    "baseline_sequential": {"makespan_s": base_makespan,
                                            "cell_updates_per_s": work_euler / base_makespan,
                                            "p50_ms": float(np.percentile(blat, 50)),
                                            "p99_ms": float(np.percentile(blat, 99))},
                    "clocks": clk_s.summary(),
                }
    finally:
        R.ripple_ctx_destroy(ctx)
    return result


def cpu_baseline_sample():
    """The FP64 oracle, as it stands, on the host cores: one full 256^3 step of
    the headline workload on all cores, and the whole 2D FP64 128^2 workload
    (100 steps) on one thread and on all cores (the oracle's results do not
    depend on its thread count)."""
    import oracle
    oracle.build()
    host = host_description()
    ncores = oracle.set_threads(os.cpu_count() or 1)
    try:
        U0 = inputs.euler3d_blast(N3, seed=1).astype(np.float32).astype(np.float64)
        t0 = time.perf_counter()
        oracle.euler_run(U0, 1, scheme=oracle.MUSCL_HANCOCK, bc=oracle.TRANSMISSIVE)
        dt = time.perf_counter() - t0
        U2 = inputs.euler2d_sine(128)
        c0 = {}
        for nt in (1, ncores):
            oracle.set_threads(nt)
            t0 = time.perf_counter()
            oracle.euler_run(U2, 100)
            t2 = time.perf_counter() - t0
            c0[f"threads_{nt}"] = {"cell_updates_per_s": 128 * 128 * 100 / t2, "seconds": t2}
    finally:
        oracle.set_threads(1)
    return {"value": N3 ** 3 / dt, "unit": METRIC, "cores": ncores, "kind": "oracle",
            "sample": f"one MUSCL-Hancock step of the 256^3 blast in FP64 on {ncores} threads ({dt:.1f} s)",
            "host": host, "euler2d_fp64_128_100_steps": c0}


def rel_l1(a, b):
    """Per-component relative L1 of a against b (component axis first), max over components."""
    a = np.asarray(a, dtype=np.float64).reshape(np.shape(b)[0] if np.ndim(b) > 1 else 1, -1)
    b = np.asarray(b, dtype=np.float64).reshape(a.shape)
    return float((np.abs(a - b).sum(1) / np.abs(b).sum(1).clip(1e-300)).max())


def oracle_legs(par):
    """The FP64 oracle beside each GPU result of this run: its time on the host
    cores (a reported baseline) and the GPU result's error against it."""
    import oracle
    oracle.build()
    out = {}
    if "headline" in par:
        p = par["headline"]
        t0 = time.perf_counter()
        vals, dt = oracle.euler_step_cells(p["Un"].astype(np.float64), p["cells"], scheme=oracle.MUSCL_HANCOCK,
                                           bc=oracle.TRANSMISSIVE, dx=p["dx"])
        t = time.perf_counter() - t0
        err = float((np.abs(p["gpu"] - vals).sum(0) / np.abs(vals).sum(0)).max())
        out["euler3d_256"] = {"rel_l1_vs_oracle": err, "tolerance": 2e-5,
                              "check": "one step from the GPU state after the timed steps, 4096 seeded cells",
                              "dt_rel_diff": abs(dt - p["dt"]) / dt, "oracle_seconds": t}
    if "full_run_128" in par:
        p = par["full_run_128"]
        n1 = p["n"]
        nt = oracle.set_threads(os.cpu_count() or 1)
        try:
            t0 = time.perf_counter()
            ref, info = oracle.euler_run(p["U0"].astype(np.float64), NSTEPS_SOLVE, scheme=oracle.MUSCL_HANCOCK,
                                         bc=oracle.TRANSMISSIVE)
            t = time.perf_counter() - t0
        finally:
            oracle.set_threads(1)
        g = np.asarray(p["gpu"], dtype=np.float64).reshape(5, -1)
        r_ = ref.reshape(5, -1)
        linf = float((np.abs(g - r_).max(1) / np.abs(r_).max(1)).max())
        out["euler3d_128_full_50_steps"] = {
            "rel_l1_vs_oracle": rel_l1(p["gpu"], ref), "tolerance": 2e-5, "max_elementwise_rel": linf,
            "elementwise_tolerance": 5e-5, "t_rel_diff": abs(p["t"] - info["t"]) / info["t"],
            "check": f"whole {n1}^3 field after {NSTEPS_SOLVE} steps from the initial blast (SoA, the headline kernel)",
            "oracle_cell_updates_per_s": n1 ** 3 * NSTEPS_SOLVE / t, "oracle_threads": nt, "oracle_seconds": t}
    if "force_split_fp32_3d_128" in par:
        p = par["force_split_fp32_3d_128"]
        nt = oracle.set_threads(os.cpu_count() or 1)
        try:
            t0 = time.perf_counter()
            ref, _ = oracle.euler_run(p["U0"].astype(np.float64), 10, scheme=oracle.FORCE_SPLIT,
                                      bc=oracle.TRANSMISSIVE)
            t = time.perf_counter() - t0
        finally:
            oracle.set_threads(1)
        g = np.asarray(p["gpu"], dtype=np.float64).reshape(5, -1)
        r_ = ref.reshape(5, -1)
        out["force_split_fp32_3d_128"] = {
            "rel_l1_vs_oracle": rel_l1(p["gpu"], ref), "tolerance": 2e-5,
            "max_elementwise_rel": float((np.abs(g - r_).max(1) / np.abs(r_).max(1)).max()),
            "elementwise_tolerance": 5e-5,
            "check": "whole 128^3 blast after 10 split FORCE steps (x, y, z walk sweeps)",
            "oracle_cell_updates_per_s": p["n"] ** 3 * 10 / t, "oracle_threads": nt, "oracle_seconds": t}
    if "force_split_fp64_128" in par:
        p = par["force_split_fp64_128"]
        t0 = time.perf_counter()
        ref, _ = oracle.euler_run(p["U0"], 100, scheme=oracle.FORCE_SPLIT)
        t = time.perf_counter() - t0
        out["force_split_fp64_128"] = {"rel_l1_vs_oracle": rel_l1(p["gpu"], ref), "tolerance": 1e-12,
                                       "check": "100 split FORCE steps from the initial state",
                                       "oracle_cell_updates_per_s": 128 * 128 * 100 / t, "oracle_seconds": t}
    if "euler2d_fp64_128" in par:
        p = par["euler2d_fp64_128"]
        t0 = time.perf_counter()
        ref, _ = oracle.euler_run(p["U0"], 100)
        t = time.perf_counter() - t0
        out["euler2d_fp64_128"] = {"rel_l1_vs_oracle": rel_l1(p["gpu"], ref), "tolerance": 1e-12,
                                   "check": "100 steps from the initial state",
                                   "oracle_cell_updates_per_s": 128 * 128 * 100 / t, "oracle_seconds": t}
    for name in ("2d_2048", "3d_192"):
        key = "eikonal_" + name
        if key in par:
            p = par[key]
            t0 = time.perf_counter()
            T = oracle.eikonal_fmm(p["s"].astype(np.float64), p["h"], p["src"])
            t = time.perf_counter() - t0
            out[key] = {"rel_l1_vs_oracle": rel_l1(np.asarray(p["gpu"]).reshape(T.shape)[None], T[None]),
                        "tolerance": 1e-4, "check": "whole grid against Fast Marching",
                        "oracle_solved_cells_per_s": T.size / t, "oracle_seconds": t}
    if "batched" in par:
        errs, cells, t = [], 0, 0.0
        for p in par["batched"]:
            side = p["side"]
            t0 = time.perf_counter()
            ref, _ = oracle.euler_run(p["U0"].astype(np.float64), 100, dx=[1.0 / side] * 2)
            t += time.perf_counter() - t0
            errs.append(rel_l1(p["gpu"], ref))
            cells += side * side
        out["batched"] = {"rel_l1_vs_oracle": max(errs), "tolerance": 2e-5,
                          "check": f"4 of the 512 problems (sides {[p['side'] for p in par['batched']]}), 100 steps",
                          "oracle_cell_updates_per_s": cells * 100 / t, "oracle_seconds": t}
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--e2e-solves", type=int, default=2)
    ap.add_argument("--skip-eikonal", action="store_true")
    ap.add_argument("--skip-cpu-baseline", action="store_true")
    ap.add_argument("--skip-batched", action="store_true")
    ap.add_argument("--skip-serve", action="store_true")
    ap.add_argument("--skip-layout", action="store_true")
    ap.add_argument("--sweep-only", action="store_true",
                    help="time only the SoA sweep (a small case for profiling; not the headline line)")
    ap.add_argument("--sweep-dims", type=int, nargs=3, default=[N3, N3, N3], metavar=("NX", "NY", "NZ"))
    ap.add_argument("--sweep-variant", type=int, default=-1,
                    help="sweep kernel of the sweep-only run (ripple_field_set_sweep; -1: the default)")
    ap.add_argument("--force-only", action="store_true",
                    help="time only the split FORCE step, FP32 SoA (profiling; not the headline line)")
    ap.add_argument("--force-n", type=int, default=8192)
    ap.add_argument("--force-dim", type=int, default=2, choices=[2, 3])
    ap.add_argument("--solo-only", action="store_true",
                    help="run only the single-request solo solver leg (profiling; not the headline line)")
    ap.add_argument("--batched-only", action="store_true",
                    help="run only the 512-instance batched workload (profiling; not the headline line)")
    ap.add_argument("--eikonal-only", action="store_true",
                    help="run only the FIM eikonal solves (profiling; not the headline line)")
    ap.add_argument("--serve-only", action="store_true",
                    help="run only the serving workload (not the headline line)")
    ap.add_argument("--serve-requests", type=int, default=400,
                    help="requests per arrival rate of the serving workload")
    ap.add_argument("--serve-full", action="store_true",
                    help="the serving workload as stated: 2,000 requests at each of the six rates")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.serve_full:
        args.serve_requests = 2000
    rank, world, local = dist_setup(args.gpus)
    ncell = int(np.prod(args.sweep_dims))
    nx, ny, nz = args.sweep_dims
    workload = "euler3d_muscl_hancock_256^3_blast" if (nx, ny, nz) == (N3, N3, N3) else \
        f"euler3d_muscl_hancock_{nx}x{ny}x{nz}_blast"
    config = {"workload": workload, "cells": ncell, "ncomp": 5, "halo": 2,
              "scheme": "MUSCL-Hancock minmod + Rusanov", "bc": "transmissive", "layout": "SoA",
              "l2": f"inputs larger than L2 ({ncell * 20 / 1e6:.0f} MB per buffer), no flush"}

    if args.impl == "reference":
        if rank != 0:
            return
        import oracle
        oracle.build()
        ncores = oracle.set_threads(os.cpu_count() or 1)
        side = 128  # bounded sample: the central 128^3 crop of the blast, one step each
        U0 = inputs.euler3d_blast(N3, seed=1).astype(np.float32).astype(np.float64)
        lo = (N3 - side) // 2
        crop = np.ascontiguousarray(U0[:, lo:lo + side, lo:lo + side, lo:lo + side])
        dxs = [1.0 / N3] * 3
        for _ in range(args.warmup):
            oracle.euler_run(crop, 1, scheme=oracle.MUSCL_HANCOCK, bc=oracle.TRANSMISSIVE, dx=dxs)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            oracle.euler_run(crop, 1, scheme=oracle.MUSCL_HANCOCK, bc=oracle.TRANSMISSIVE, dx=dxs)
        dt = time.perf_counter() - t0
        value = args.steps * side ** 3 / dt
        line = {"impl": "reference", "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": args.gpus,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic", "config": config,
                "cpu_baseline": {"value": value, "unit": METRIC, "cores": ncores, "kind": "oracle",
                                 "sample": f"one FP64 step of the central {side}^3 crop of the 256^3 blast per step",
                                 "host": host_description()},
                "e2e": {"value": value, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return

    if args.force_only:
        import torch
        import paper_2104_08571_gb300 as R
        torch.cuda.set_device(local)
        fs = bench_force_split(R, torch, local, legs=(("fp32", args.force_dim, args.force_n, R.RIPPLE_F32,
                                                       args.steps),))
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": fs["fp32"]["cell_updates_per_s"], "unit": METRIC,
                              "n_gpus": world,
                              "config": {"workload": f"force_split_{args.force_dim}d_fp32_{args.force_n}^{args.force_dim}"},
                              "force_split": fs}))
        return
    if args.serve_only:
        import torch
        import paper_2104_08571_gb300 as R
        torch.cuda.set_device(local)
        sv = bench_serving(R, torch, local, count=args.serve_requests)
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": sv["rates"]["2000"]["cell_updates_per_s"], "unit": METRIC,
                              "n_gpus": world, "config": {"workload": "served mix, Poisson arrivals"},
                              "serve": sv}))
        return
    if args.eikonal_only:
        import torch
        import paper_2104_08571_gb300 as R
        torch.cuda.set_device(local)
        ek = bench_eikonal(R, torch, local, steps=args.steps)
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": ek["2d_2048"]["godunov_updates_per_s"], "unit": METRIC,
                              "n_gpus": world, "config": {"workload": "FIM eikonal 2048^2 and 192^3"},
                              "eikonal": ek}))
        return
    if args.solo_only:
        import torch
        import paper_2104_08571_gb300 as R
        torch.cuda.set_device(local)
        so = bench_solo(R, torch, local)
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": 1024 * 1024 / (so["1024"]["solo_rounds"]["us_per_step_device"] * 1e-6),
                              "unit": METRIC, "n_gpus": world,
                              "config": {"workload": "one 2D Euler request served alone, sides 64/256/1024"},
                              "solo": so}))
        return
    if args.batched_only:
        import torch
        import paper_2104_08571_gb300 as R
        torch.cuda.set_device(local)
        b = bench_batched(R, torch, local)
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": b["value"], "unit": METRIC, "n_gpus": world,
                              "config": {"workload": b["workload"]}, "batched": b}))
        return
    r = bench_gpu(args, rank, world, local)
    if rank != 0:
        return
    if args.sweep_only:
        print(json.dumps({
            "metric": METRIC, "value": r["value"], "unit": METRIC, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": r["ms_per_step"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": config, "gpu_launches": args.steps,
            "roofline": {"bound": "hbm", "achieved": r["achieved"], "peak": r["hbm_peak"], "unit": "GB/s",
                         "frac": r["achieved"] / r["hbm_peak"], "traffic": None, "peak_source": r["peak_kind"]},
            "clocks": r["clocks"]}))
        return
    cpu = None
    parity = None
    if not args.skip_cpu_baseline and world == 1:
        cpu = cpu_baseline_sample()
        legs = oracle_legs(r["parity_data"])
        cpu["workloads"] = {k: {kk: v for kk, v in d.items() if kk.startswith("oracle")} for k, d in legs.items()}
        parity = {k: {kk: v for kk, v in d.items() if not kk.startswith("oracle")} for k, d in legs.items()}
    state_bytes = ncell * 5 * 4
    line = {
        "metric": METRIC, "value": r["value"], "unit": METRIC, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": r["ms_per_step"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": config,
        "gpu_launches": args.steps,
        "roofline": {"bound": "hbm", "achieved": r["achieved"], "peak": r["hbm_peak"], "unit": "GB/s",
                     "frac": r["achieved"] / r["hbm_peak"], "traffic": DRAM_BYTES_PER_CELL_UPDATE * ncell,
                     "traffic_source": "ncu dram bytes of a 256x256x128 launch, scaled by cells",
                     "peak_source": r["peak_kind"],
                     "algorithmic_bytes_per_cell_update": BYTES_PER_CELL_UPDATE},
        "clocks": r["clocks"],
        "ms_per_step_median": float(np.median(r["extra"]["per_step_ms"])),
        "ms_per_step_spread": {"min": float(np.min(r["extra"]["per_step_ms"])),
                               "p10": float(np.percentile(r["extra"]["per_step_ms"], 10)),
                               "p90": float(np.percentile(r["extra"]["per_step_ms"], 90)),
                               "max": float(np.max(r["extra"]["per_step_ms"])),
                               "repeats": len(r["extra"]["per_step_ms"]),
                               "timing": "each step between its own CUDA events on the library stream"},
        "e2e": {"value": r["e2e_value"], "unit": METRIC,
                "h2d_bytes_per_step": state_bytes // NSTEPS_SOLVE, "d2h_bytes_per_step": state_bytes // NSTEPS_SOLVE,
                "h2d_bytes_per_solve": state_bytes, "d2h_bytes_per_solve": state_bytes,
                "step": f"one {NSTEPS_SOLVE}-step solve: pinned host -> device, {NSTEPS_SOLVE} sweeps, "
                        "device -> pinned host; bytes per step = bytes per solve / steps per solve",
                "solves": r["e2e_solves"], "seconds": r["e2e_s"], "clocks": r["extra"]["e2e_clocks"]},
        "cpu_baseline": cpu,
        "parity": parity,
        "aos": {"value": ncell / (r["ms_aos"] / 1e3), "ms_per_step": r["ms_aos"],
                "ms_per_step_median": float(np.median(r["extra"]["aos_per_step_ms"])),
                "kernel": "pair kernel (the row kernel's per-lane loads of AoS planes conflict in shared memory)",
                "clocks": r["extra"]["aos_clocks"]},
        "euler2d_fp64_128": {"ms_per_100_steps": r["ms2"], "us_per_step": r["ms2"] * 10.0,
                             "cell_updates_per_s": 100 * 128 * 128 / (r["ms2"] / 1e3),
                             "clocks": r["extra"]["euler2d_clocks"]},
        "eikonal": r["eik"],
        "batched": r["batched"],
        "serve": r["serve"],
        "solo": r["solo"],
        "layout_microbench": r["layout"],
        "force_split": r["force"],
    }
    print(json.dumps(line))


if __name__ == "__main__":
    main()
