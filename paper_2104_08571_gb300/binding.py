"""Thin ctypes binding of ``libripple.so`` (the C ABI declared in include/ripple.h).

Argument marshalling only: every step of the stencil path runs in the CUDA
kernels behind the C ABI.  Functions keep the C names.  A failing status
raises ``RippleError``.  If the shared library is missing or cannot be
loaded, importing this module raises: there is no fallback path.

Array conventions (see include/ripple.h): interior cells only, numpy/torch
arrays of shape (ncomp, [nz,] ny, nx) for RIPPLE_SOA and ([nz,] ny, nx, ncomp)
for RIPPLE_AOS (one-component fields may drop the component axis), dtype
float32 for RIPPLE_F32 fields and float64 for RIPPLE_F64.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

RIPPLE_OK = 0
RIPPLE_ERR_INVALID = 1
RIPPLE_ERR_OOM = 2
RIPPLE_ERR_CUDA = 3
RIPPLE_ERR_NOT_READY = 4
RIPPLE_ERR_TIMEOUT = 5
RIPPLE_ERR_NUMERIC = 6
RIPPLE_ERR_BUDGET = 7
RIPPLE_ERR_INTERNAL = 8

RIPPLE_AOS = 0
RIPPLE_SOA = 1
RIPPLE_F32 = 0
RIPPLE_F64 = 1
RIPPLE_RUSANOV1 = 0
RIPPLE_MUSCL_HANCOCK_MINMOD = 1
RIPPLE_FORCE_SPLIT = 2
RIPPLE_BC_PERIODIC = 0
RIPPLE_BC_TRANSMISSIVE = 1

_STATUS_NAMES = {0: "OK", 1: "INVALID", 2: "OOM", 3: "CUDA", 4: "NOT_READY", 5: "TIMEOUT", 6: "NUMERIC",
                 7: "BUDGET", 8: "INTERNAL"}


class RippleError(RuntimeError):
    def __init__(self, status: int, func: str, message: str):
        super().__init__(f"{func}: RIPPLE_ERR_{_STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class ripple_fv_params(ctypes.Structure):
    _fields_ = [("gamma", ctypes.c_double), ("cfl", ctypes.c_double), ("dx", ctypes.c_double * 3),
                ("scheme", ctypes.c_int), ("bc", ctypes.c_int)]


class ripple_fv_stats(ctypes.Structure):
    _fields_ = [("t", ctypes.c_double), ("dt_last", ctypes.c_double), ("totals", ctypes.c_double * 5),
                ("steps_done", ctypes.c_int64)]


class ripple_eik_params(ctypes.Structure):
    _fields_ = [("h", ctypes.c_double), ("tol", ctypes.c_double), ("max_iters", ctypes.c_int64)]


class ripple_eik_stats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int64), ("tile_visits", ctypes.c_int64), ("cell_updates", ctypes.c_int64)]


class ripple_field_desc(ctypes.Structure):
    _fields_ = [("ndim", ctypes.c_int), ("ncomp", ctypes.c_int), ("halo", ctypes.c_int), ("layout", ctypes.c_int),
                ("dtype", ctypes.c_int), ("dims", ctypes.c_int64 * 3), ("padded", ctypes.c_int64 * 3),
                ("x_lead", ctypes.c_int64), ("buffer_bytes", ctypes.c_size_t), ("current", ctypes.c_void_p)]


_VP = ctypes.c_void_p
_I64P = ctypes.POINTER(ctypes.c_int64)

RIPPLE_REQ_EULER = 0
RIPPLE_REQ_EIKONAL = 1


class ripple_request(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("dims", ctypes.c_int64 * 2), ("input", ctypes.c_void_p),
                ("output", ctypes.c_void_p), ("fv", ripple_fv_params), ("nsteps", ctypes.c_int64),
                ("eik", ripple_eik_params), ("sources", _I64P), ("nsrc", ctypes.c_int)]


class ripple_ticket_info(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("submit_s", ctypes.c_double), ("admit_s", ctypes.c_double),
                ("start_s", ctypes.c_double), ("finish_s", ctypes.c_double), ("work", ctypes.c_int64),
                ("tile_visits", ctypes.c_int64), ("cell_updates", ctypes.c_int64), ("t", ctypes.c_double)]


class ripple_batch_config(ctypes.Structure):
    _fields_ = [("layout", ctypes.c_int), ("tile_variant", ctypes.c_int), ("steps_per_sync", ctypes.c_int),
                ("use_graphs", ctypes.c_int), ("dtype", ctypes.c_int), ("fim_iters_per_step", ctypes.c_int),
                ("active_cells", ctypes.c_int64), ("staging", ctypes.c_int), ("async_queue", ctypes.c_int),
                ("solo_rounds", ctypes.c_int)]


class ripple_batch_stats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("admitted", ctypes.c_int64), ("completed", ctypes.c_int64),
                ("failed", ctypes.c_int64), ("global_steps", ctypes.c_int64), ("launches", ctypes.c_int64),
                ("graph_replays", ctypes.c_int64), ("now_s", ctypes.c_double), ("fim_iterations", ctypes.c_int64),
                ("device_s", ctypes.c_double), ("host_admit_s", ctypes.c_double),
                ("host_round_s", ctypes.c_double), ("host_finish_s", ctypes.c_double)]

# name -> (argtypes) ; every ABI function returns ripple_status (int)
_SIGNATURES = {
    "ripple_ctx_create": [ctypes.c_int, ctypes.c_size_t, ctypes.POINTER(_VP)],
    "ripple_ctx_destroy": [_VP],
    "ripple_set_stream": [_VP, _VP],
    "ripple_set_allocator": [_VP, _VP, _VP, _VP],
    "ripple_ctx_sync": [_VP],
    "ripple_ctx_mem_used": [_VP, ctypes.POINTER(ctypes.c_size_t)],
    "ripple_field_create": [_VP, ctypes.c_int, _I64P, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                            ctypes.POINTER(_VP)],
    "ripple_field_destroy": [_VP],
    "ripple_field_upload": [_VP, _VP, ctypes.c_int],
    "ripple_field_download": [_VP, _VP, ctypes.c_int],
    "ripple_field_upload_device": [_VP, _VP, ctypes.c_int],
    "ripple_field_download_device": [_VP, _VP, ctypes.c_int],
    "ripple_field_describe": [_VP, ctypes.POINTER(ripple_field_desc)],
    "ripple_field_set_sweep": [_VP, ctypes.c_int, ctypes.c_int],
    "ripple_fv_step": [_VP, ctypes.POINTER(ripple_fv_params), ctypes.c_int64, ctypes.POINTER(ripple_fv_stats)],
    "ripple_eikonal_solve": [_VP, _VP, _I64P, ctypes.c_int, ctypes.POINTER(ripple_eik_params),
                             ctypes.POINTER(ripple_eik_stats)],
    "ripple_totals_noalloc": [_VP, ctypes.c_int, _I64P, ctypes.c_int, ctypes.c_int, ctypes.c_int, _VP, _VP],
    "ripple_saxpy": [_VP, ctypes.c_int64, ctypes.c_float, _VP, _VP],
    "ripple_particle_update": [_VP, ctypes.c_int64, ctypes.c_float, _VP, ctypes.c_int, ctypes.c_int],
    "ripple_batch_configure": [_VP, ctypes.POINTER(ripple_batch_config)],
    "ripple_batch_submit": [_VP, ctypes.POINTER(ripple_request), ctypes.c_int, ctypes.POINTER(ctypes.c_uint64)],
    "ripple_poll": [_VP, ctypes.c_uint64, ctypes.POINTER(ripple_ticket_info)],
    "ripple_wait": [_VP, ctypes.c_uint64, ctypes.c_int64, ctypes.POINTER(ripple_ticket_info)],
    "ripple_batch_get_stats": [_VP, ctypes.POINTER(ripple_batch_stats)],
    "ripple_batch_autotune": [_VP, _I64P, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ripple_batch_config),
                              ctypes.POINTER(ctypes.c_double)],
}
_STRING_FUNCS = ["ripple_last_error", "ripple_version"]

_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False):
    """Load libripple.so (optionally building it first).  Raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if build_if_missing and not _build.up_to_date():
        _build.build()
    if not os.path.exists(path):
        raise ImportError(f"libripple.so not built ({path}); run __graft_entry__.build() or "
                          "python -m paper_2104_08571_gb300.build")
    lib = ctypes.CDLL(path)
    for name, argtypes in _SIGNATURES.items():
        fn = getattr(lib, name)
        fn.argtypes = argtypes
        fn.restype = ctypes.c_int
    for name in _STRING_FUNCS:
        fn = getattr(lib, name)
        fn.argtypes = []
        fn.restype = ctypes.c_char_p
    _lib = lib
    return lib


def exported_symbols():
    return sorted(list(_SIGNATURES) + _STRING_FUNCS)


def _check(status: int, func: str):
    if status != RIPPLE_OK:
        raise RippleError(status, func, ripple_last_error())


def ripple_last_error() -> str:
    return load().ripple_last_error().decode()


def ripple_version() -> str:
    return load().ripple_version().decode()


# ---------------------------------------------------------------------------
# context
# ---------------------------------------------------------------------------
def ripple_ctx_create(device: int = 0, mem_budget_bytes: int = 0):
    out = _VP()
    _check(load().ripple_ctx_create(int(device), int(mem_budget_bytes), ctypes.byref(out)), "ripple_ctx_create")
    return out


def ripple_ctx_destroy(ctx):
    _check(load().ripple_ctx_destroy(ctx), "ripple_ctx_destroy")


def ripple_set_stream(ctx, stream=None):
    """stream: a cudaStream_t as int, a torch.cuda.Stream, or None (own stream)."""
    handle = None
    if stream is not None:
        handle = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
    _check(load().ripple_set_stream(ctx, handle), "ripple_set_stream")


_ALLOC_T = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
_FREE_T = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)
_keepalive = {}


def ripple_set_allocator(ctx, alloc=None, release=None):
    """alloc(nbytes) -> device pointer (int); release(ptr). None restores cudaMalloc."""
    if alloc is None:
        _check(load().ripple_set_allocator(ctx, None, None, None), "ripple_set_allocator")
        _keepalive.pop(ctx.value, None)
        return
    ca = _ALLOC_T(lambda n, user: alloc(int(n)) or 0)
    cf = _FREE_T(lambda p, user: release(int(p)))
    _keepalive[ctx.value] = (ca, cf)
    _check(load().ripple_set_allocator(ctx, ctypes.cast(ca, _VP), ctypes.cast(cf, _VP), None),
           "ripple_set_allocator")


def use_torch_allocator(ctx, device: int = 0):
    """Route the context's device allocations through PyTorch's caching allocator."""
    import torch

    def alloc(n):
        return torch.cuda.caching_allocator_alloc(n, device=device)

    def release(p):
        torch.cuda.caching_allocator_delete(p)

    ripple_set_allocator(ctx, alloc, release)


def ripple_ctx_sync(ctx):
    _check(load().ripple_ctx_sync(ctx), "ripple_ctx_sync")


def ripple_ctx_mem_used(ctx) -> int:
    out = ctypes.c_size_t(0)
    _check(load().ripple_ctx_mem_used(ctx, ctypes.byref(out)), "ripple_ctx_mem_used")
    return out.value


# ---------------------------------------------------------------------------
# fields
# ---------------------------------------------------------------------------
def ripple_field_create(ctx, dims, ncomp, layout=RIPPLE_SOA, halo=1, dtype=RIPPLE_F32):
    """dims = (nx, ny[, nz])."""
    d = (ctypes.c_int64 * 3)(*(list(dims) + [1] * (3 - len(dims))))
    out = _VP()
    _check(load().ripple_field_create(ctx, len(dims), d, int(ncomp), int(layout), int(halo), int(dtype),
                                      ctypes.byref(out)), "ripple_field_create")
    return out


def ripple_field_destroy(field):
    _check(load().ripple_field_destroy(field), "ripple_field_destroy")


def ripple_field_describe(field) -> ripple_field_desc:
    out = ripple_field_desc()
    _check(load().ripple_field_describe(field, ctypes.byref(out)), "ripple_field_describe")
    return out


def ripple_field_set_sweep(field, variant=-1, zchunk=0):
    """Choose the field's sweep kernel variant and z chunk (-1 / 0 = automatic)."""
    _check(load().ripple_field_set_sweep(field, int(variant), int(zchunk)), "ripple_field_set_sweep")


def _np_dtype(desc):
    return np.float32 if desc.dtype == RIPPLE_F32 else np.float64


def _expected_count(desc):
    return int(desc.dims[0] * desc.dims[1] * desc.dims[2] * desc.ncomp)


def ripple_field_upload(field, array, layout=RIPPLE_SOA):
    """Upload interior cells from a numpy array / CPU tensor (host) or a CUDA tensor (device)."""
    desc = ripple_field_describe(field)
    if hasattr(array, "is_cuda") and array.is_cuda:
        import torch
        want = torch.float32 if desc.dtype == RIPPLE_F32 else torch.float64
        if array.dtype != want or not array.is_contiguous() or array.numel() != _expected_count(desc):
            raise ValueError("device array must be contiguous, of the field's dtype and element count")
        _check(load().ripple_field_upload_device(field, _VP(array.data_ptr()), int(layout)),
               "ripple_field_upload_device")
        return
    if hasattr(array, "numpy"):
        array = array.numpy()
    arr = np.ascontiguousarray(array, dtype=_np_dtype(desc))
    if arr.size != _expected_count(desc):
        raise ValueError(f"expected {_expected_count(desc)} elements, got {arr.size}")
    _check(load().ripple_field_upload(field, _VP(arr.ctypes.data), int(layout)), "ripple_field_upload")


def ripple_field_download(field, layout=RIPPLE_SOA, out=None):
    """Download interior cells into a new numpy array (or `out`, host or CUDA tensor)."""
    desc = ripple_field_describe(field)
    nd = desc.ndim
    spatial = [int(desc.dims[d]) for d in reversed(range(nd))]
    if out is not None and hasattr(out, "is_cuda") and out.is_cuda:
        _check(load().ripple_field_download_device(field, _VP(out.data_ptr()), int(layout)),
               "ripple_field_download_device")
        return out
    if out is None:
        shape = ([desc.ncomp] + spatial) if layout == RIPPLE_SOA else (spatial + [desc.ncomp])
        out = np.empty(shape, dtype=_np_dtype(desc))
    ptr = out.data_ptr() if hasattr(out, "data_ptr") else out.ctypes.data
    _check(load().ripple_field_download(field, _VP(ptr), int(layout)), "ripple_field_download")
    return out


# ---------------------------------------------------------------------------
# solvers
# ---------------------------------------------------------------------------
def make_fv_params(dx, gamma=1.4, cfl=0.4, scheme=RIPPLE_RUSANOV1, bc=RIPPLE_BC_PERIODIC) -> ripple_fv_params:
    dx = list(dx) + [1.0] * (3 - len(dx))
    return ripple_fv_params(float(gamma), float(cfl), (ctypes.c_double * 3)(*dx), int(scheme), int(bc))


def ripple_fv_step(field, params: ripple_fv_params, nsteps: int, stats: bool = True):
    """Advance an Euler field; returns a dict of stats (synchronous) or None (queued only)."""
    st = ripple_fv_stats() if stats else None
    _check(load().ripple_fv_step(field, ctypes.byref(params), int(nsteps), ctypes.byref(st) if stats else None),
           "ripple_fv_step")
    if not stats:
        return None
    return dict(t=st.t, dt_last=st.dt_last, totals=list(st.totals), steps_done=st.steps_done)


def ripple_eikonal_solve(slowness, T, sources, h, tol=1e-6, max_iters=0):
    """sources: list of (x, y[, z]) cell coordinates."""
    flat = [int(c) for s in sources for c in s]
    arr = (ctypes.c_int64 * len(flat))(*flat)
    prm = ripple_eik_params(float(h), float(tol), int(max_iters))
    st = ripple_eik_stats()
    _check(load().ripple_eikonal_solve(slowness, T, arr, len(sources), ctypes.byref(prm), ctypes.byref(st)),
           "ripple_eikonal_solve")
    return dict(iterations=st.iterations, tile_visits=st.tile_visits, cell_updates=st.cell_updates)


def ripple_totals_noalloc(state, dims, ncomp, layout, dtype, totals_out, stream=None):
    """FP64 compensated totals of a dense CUDA tensor `state` into the CUDA tensor
    `totals_out` (ncomp doubles) without any device allocation by the library.
    Asynchronous on `stream` (a torch.cuda.Stream, a cudaStream_t int, or None)."""
    import torch

    want = torch.float32 if int(dtype) == RIPPLE_F32 else torch.float64 if int(dtype) == RIPPLE_F64 else None
    if want is None:
        raise ValueError("dtype must be RIPPLE_F32 or RIPPLE_F64")
    for name, t in (("state", state), ("totals_out", totals_out)):
        if not (hasattr(t, "is_cuda") and t.is_cuda):
            raise ValueError(f"{name} must be a CUDA tensor")
        if not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
        if t.device.index != torch.cuda.current_device():
            raise ValueError(f"{name} must be on the current CUDA device")
    if state.dtype != want:
        raise ValueError(f"state must be {want}, got {state.dtype}")
    if totals_out.dtype != torch.float64:
        raise ValueError("totals_out must be float64")
    cells = 1
    for x in dims:
        cells *= int(x)
    if state.numel() < cells * int(ncomp):
        raise ValueError(f"state holds {state.numel()} elements, dims x ncomp needs {cells * int(ncomp)}")
    if totals_out.numel() < int(ncomp):
        raise ValueError(f"totals_out holds {totals_out.numel()} elements, needs {int(ncomp)}")
    d = (ctypes.c_int64 * len(dims))(*[int(x) for x in dims])
    handle = None
    if stream is not None:
        handle = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
    _check(load().ripple_totals_noalloc(_VP(state.data_ptr()), len(dims), d, int(ncomp), int(layout), int(dtype),
                                        _VP(totals_out.data_ptr()), handle), "ripple_totals_noalloc")


def ripple_saxpy(ctx, a, x, y):
    """y <- a x + y on CUDA float32 tensors x, y (same number of elements), on the context's stream."""
    n = x.numel()
    if y.numel() != n:
        raise RippleError(RIPPLE_ERR_INVALID, "x and y differ in length")
    _check(load().ripple_saxpy(ctx, n, float(a), _VP(x.data_ptr()), _VP(y.data_ptr())), "ripple_saxpy")


def ripple_particle_update(ctx, particles, dt, layout=RIPPLE_SOA, staged=False):
    """x_d <- x_d + v_d dt on a CUDA float32 tensor of 6n floats (AoS records or SoA runs)."""
    if particles.numel() % 6:
        raise RippleError(RIPPLE_ERR_INVALID, "particles must hold 6 floats per particle")
    _check(load().ripple_particle_update(ctx, particles.numel() // 6, float(dt), _VP(particles.data_ptr()),
                                         int(layout), int(bool(staged))), "ripple_particle_update")


# ---------------------------------------------------------------------------
# batched / served execution
# ---------------------------------------------------------------------------
_inflight = {}  # ticket -> (input array, output array, sources): kept alive until retired


def _info_dict(info):
    return dict(status=info.status, submit_s=info.submit_s, admit_s=info.admit_s, start_s=info.start_s,
                finish_s=info.finish_s, work=info.work, tile_visits=info.tile_visits,
                cell_updates=info.cell_updates, t=info.t)


SOLO_ROUNDS_DEFAULT = 4  # resident problems up to which solo rounds run (the C default)


def ripple_batch_configure(ctx, layout=RIPPLE_SOA, tile_variant=0, steps_per_sync=16, use_graphs=True,
                           dtype=RIPPLE_F32, fim_iters_per_step=4, active_cells=0, staging=0, async_queue=False,
                           solo_rounds=True):
    """solo_rounds: True (at most SOLO_ROUNDS_DEFAULT resident problems), False (off) or that bound."""
    solo = SOLO_ROUNDS_DEFAULT if solo_rounds is True else int(solo_rounds)
    cfg = ripple_batch_config(int(layout), int(tile_variant), int(steps_per_sync), int(bool(use_graphs)), int(dtype),
                              int(fim_iters_per_step), int(active_cells), int(staging), int(bool(async_queue)), solo)
    _check(load().ripple_batch_configure(ctx, ctypes.byref(cfg)), "ripple_batch_configure")


def euler_request(U, nsteps, dx, gamma=1.4, cfl=0.4, bc=RIPPLE_BC_PERIODIC, out=None):
    """A 2D Euler request from a component-major host array U (4, ny, nx)."""
    U = np.ascontiguousarray(U)
    out = np.empty_like(U) if out is None else out
    return dict(kind=RIPPLE_REQ_EULER, input=U, output=out, nsteps=int(nsteps), dx=list(dx), gamma=gamma,
                cfl=cfl, bc=bc)


def eikonal_request(s, sources, h, tol=1e-6, max_iters=0, out=None):
    """A 2D eikonal request from a host slowness array s (ny, nx) and (x, y) sources."""
    s = np.ascontiguousarray(s)
    out = np.empty_like(s) if out is None else out
    return dict(kind=RIPPLE_REQ_EIKONAL, input=s, output=out, sources=[tuple(c) for c in sources], h=h, tol=tol,
                max_iters=max_iters)


def _struct_dtype(cls):
    """numpy dtype with the field offsets of a ctypes Structure (pointers as uint64)."""
    names, formats, offsets = [], [], []
    for name, ct in cls._fields_:
        f = getattr(cls, name)
        if isinstance(ct, type) and issubclass(ct, ctypes.Structure):
            fmt = _struct_dtype(ct)
        elif isinstance(ct, type) and issubclass(ct, ctypes.Array):
            fmt = (np.dtype(ct._type_), ct._length_)
        elif ct in (ctypes.c_void_p,) or (isinstance(ct, type) and issubclass(ct, ctypes._Pointer)):
            fmt = np.uint64
        else:
            fmt = np.dtype(ct)
        names.append(name)
        formats.append(fmt)
        offsets.append(f.offset)
    return np.dtype({"names": names, "formats": formats, "offsets": offsets, "itemsize": ctypes.sizeof(cls)})


_REQ_DTYPE = None


def ripple_batch_submit(ctx, requests):
    """Queue request dicts (see euler_request / eikonal_request); returns tickets."""
    global _REQ_DTYPE
    if _REQ_DTYPE is None:
        _REQ_DTYPE = _struct_dtype(ripple_request)
    n = len(requests)
    arr = (ripple_request * n)()
    keep = []
    kind, dims, ptr, fv, fvi, nsteps = [], [], [], [], [], []
    for i, r in enumerate(requests):
        inp, outp = r["input"], r["output"]
        k = r["kind"]
        kind.append(k)
        shp = inp.shape
        dims.append((shp[-1], shp[-2]))
        ptr.append((inp.__array_interface__["data"][0], outp.__array_interface__["data"][0]))
        src = None
        if k == RIPPLE_REQ_EULER:
            dx = r["dx"]
            fv.append((r.get("gamma", 1.4), r.get("cfl", 0.4), dx[0], dx[1] if len(dx) > 1 else 1.0,
                       dx[2] if len(dx) > 2 else 1.0))
            fvi.append((RIPPLE_RUSANOV1, r.get("bc", RIPPLE_BC_PERIODIC)))
            nsteps.append(r["nsteps"])
        else:
            fv.append((0.0, 0.0, 0.0, 0.0, 0.0))
            fvi.append((0, 0))
            nsteps.append(0)
            flat = [int(c) for xy in r["sources"] for c in xy]
            src = (ctypes.c_int64 * len(flat))(*flat)
            arr[i].sources = src
            arr[i].nsrc = len(r["sources"])
            arr[i].eik = ripple_eik_params(float(r["h"]), float(r.get("tol", 1e-6)), int(r.get("max_iters", 0)))
        keep.append((inp, outp, src))
    if n:
        a = np.frombuffer(arr, dtype=_REQ_DTYPE)
        kind = np.asarray(kind, np.int32)
        fv = np.asarray(fv, np.float64)
        fvi = np.asarray(fvi, np.int32)
        eu = kind == RIPPLE_REQ_EULER
        ptr = np.asarray(ptr, np.uint64)
        a["kind"] = kind
        a["dims"] = np.asarray(dims, np.int64)
        a["input"] = ptr[:, 0]
        a["output"] = ptr[:, 1]
        f = a["fv"]
        f["gamma"] = np.where(eu, fv[:, 0], f["gamma"])
        f["cfl"] = np.where(eu, fv[:, 1], f["cfl"])
        f["dx"] = np.where(eu[:, None], fv[:, 2:5], f["dx"])
        f["scheme"] = np.where(eu, fvi[:, 0], f["scheme"])
        f["bc"] = np.where(eu, fvi[:, 1], f["bc"])
        a["fv"] = f
        a["nsteps"] = np.where(eu, np.asarray(nsteps, np.int64), a["nsteps"])
    tickets = (ctypes.c_uint64 * n)()
    _check(load().ripple_batch_submit(ctx, arr, n, tickets), "ripple_batch_submit")
    out = [int(t) for t in tickets]
    for t, k in zip(out, keep):
        _inflight[t] = k
    return out


def ripple_poll(ctx, ticket):
    """Info dict once the request finished (the ticket is retired), else None."""
    info = ripple_ticket_info()
    st = load().ripple_poll(ctx, ctypes.c_uint64(ticket), ctypes.byref(info))
    if st == RIPPLE_ERR_NOT_READY:
        return None
    _check(st, "ripple_poll")
    _inflight.pop(ticket, None)
    return _info_dict(info)


def ripple_wait(ctx, ticket, timeout_ms=-1):
    info = ripple_ticket_info()
    _check(load().ripple_wait(ctx, ctypes.c_uint64(ticket), int(timeout_ms), ctypes.byref(info)), "ripple_wait")
    _inflight.pop(ticket, None)
    return _info_dict(info)


def ripple_batch_get_stats(ctx):
    st = ripple_batch_stats()
    _check(load().ripple_batch_get_stats(ctx, ctypes.byref(st)), "ripple_batch_get_stats")
    return {f: getattr(st, f) for f, _ in ripple_batch_stats._fields_}


def ripple_batch_autotune(ctx, sides, dtype=RIPPLE_F32):
    """Returns (chosen config dict, {(layout, variant): ms per global step})."""
    arr = (ctypes.c_int64 * len(sides))(*[int(x) for x in sides])
    cfg = ripple_batch_config(RIPPLE_SOA, 0, 16, 1, int(dtype), 4, 0, 0, 0, SOLO_ROUNDS_DEFAULT)
    ms = (ctypes.c_double * 18)()
    _check(load().ripple_batch_autotune(ctx, arr, len(sides), int(dtype), ctypes.byref(cfg), ms),
           "ripple_batch_autotune")
    timings = {}
    for sg in range(3):
        for li, lay in enumerate((RIPPLE_SOA, RIPPLE_AOS)):
            for v in range(3):
                timings[(lay, v, sg)] = ms[(sg * 2 + li) * 3 + v]
    return dict(layout=cfg.layout, tile_variant=cfg.tile_variant, steps_per_sync=cfg.steps_per_sync,
                use_graphs=cfg.use_graphs, dtype=cfg.dtype, fim_iters_per_step=cfg.fim_iters_per_step,
                active_cells=cfg.active_cells, staging=cfg.staging, async_queue=bool(cfg.async_queue),
                solo_rounds=int(cfg.solo_rounds)), timings
