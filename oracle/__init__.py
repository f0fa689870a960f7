"""FP64 CPU oracle for the Ripple (arXiv 2104.08571) stencil-sweep hot path.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py`` (its ``cpu_baseline`` leg and ``--impl reference``) may import
this package.  It shares no code with the CUDA library in
``paper_2104_08571_gb300`` and never imports it.

The arithmetic lives in ``ripple_oracle.c`` (plain C, double precision,
``-ffp-contract=off``; one thread unless ``set_threads`` splits the independent
grid lines of an Euler step, which changes no bit of a result); this module
only compiles it (``build()``) and marshals numpy arrays through ctypes.

Array convention: interior cells only, component-major, x fastest, i.e. a
numpy array of shape ``(ncomp, nz, ny, nx)`` (3D) or ``(ncomp, ny, nx)`` (2D)
for Euler, ``(nz, ny, nx)`` / ``(ny, nx)`` for eikonal fields.

Parity status of each function (what pins it, see ``tests/test_oracle_*.py``):
  euler_run / euler_step_cells / euler_dt -- pinned: uniform state preserved
      bit-exactly, periodic conservation to 1e-13, the closed-form advection
      solution of the sine-density problem, the exact Riemann solution of the
      Sod tube (L1 error shrinking under refinement), x/y/z symmetry, and
      2D == 3D reduction.  The 3D spherical blast itself has no closed form
      (its parity beyond oracle agreement is unpinned; only the invariants
      above and conservation before waves reach the boundary pin it).
  euler_run with FORCE_SPLIT (the split step with the FORCE flux) -- pinned:
      uniform state bit-exact, periodic conservation, the advected sine
      density keeping u, v, p uniform with first-order convergence, on a
      contact the mass update equal to the mean of the Lax-Friedrichs and
      Lax-Wendroff updates at the same Courant number, Sod L1 error
      shrinking under refinement, 1-D Sod along x, y, z bit-identical.
  eikonal_fmm -- pinned: exact k*h on 1-D strips and grid axes, |x - x0|
      under refinement, equality with Jacobi iteration to its fixed point,
      and the 4-neighbour graph-Dijkstra upper bound.
  godunov -- pinned through the same tests plus its 1-term/2-term/3-term
      closed forms.
  saxpy / particle_update (numpy, FP64) -- pinned: exact results on
      integer-valued inputs, the identities a = 0 and dt = 0, and the two
      layouts of one particle set giving the same positions.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import sys

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ripple_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libripple_oracle.so")

RUSANOV1 = 0
MUSCL_HANCOCK = 1
FORCE_SPLIT = 2  # dimensionally split step with the FORCE flux (Listing euler_graph, Section 7.3)
PERIODIC = 0
TRANSMISSIVE = 1

OK = 0
INVALID = 1
OOM = 2
NUMERIC = 6

_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle shared library (gcc, portable flags only)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    base = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
            "-shared", "-o", tmp, _SRC, "-lm"]
    # OpenMP only splits independent lines of a step over threads; without it
    # the oracle is the same single-threaded program
    if subprocess.run(base[:1] + ["-fopenmp"] + base[1:], capture_output=True).returncode != 0:
        subprocess.run(base, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        path = build()
        lib = ctypes.CDLL(path)
        i64p = ctypes.POINTER(ctypes.c_int64)
        dp = ctypes.POINTER(ctypes.c_double)
        lib.oracle_euler_run.argtypes = [ctypes.c_int, i64p, dp, ctypes.c_double, ctypes.c_double,
                                         dp, ctypes.c_int, ctypes.c_int, ctypes.c_int64, dp, dp,
                                         i64p]
        lib.oracle_euler_run.restype = ctypes.c_int
        lib.oracle_euler_dt.argtypes = [ctypes.c_int, i64p, dp, ctypes.c_double, ctypes.c_double,
                                        dp, dp]
        lib.oracle_euler_dt.restype = ctypes.c_int
        lib.oracle_euler_step_cells.argtypes = [ctypes.c_int, i64p, dp, ctypes.c_double,
                                                ctypes.c_double, dp, ctypes.c_int, ctypes.c_int,
                                                ctypes.c_double, ctypes.c_int64, i64p, dp, dp]
        lib.oracle_euler_step_cells.restype = ctypes.c_int
        lib.oracle_eikonal_fmm.argtypes = [ctypes.c_int, i64p, dp, ctypes.c_double, ctypes.c_int,
                                           i64p, dp]
        lib.oracle_eikonal_fmm.restype = ctypes.c_int
        lib.oracle_godunov.argtypes = [ctypes.c_int, dp, ctypes.c_double]
        lib.oracle_godunov.restype = ctypes.c_double
        lib.oracle_set_threads.argtypes = [ctypes.c_int]
        lib.oracle_set_threads.restype = ctypes.c_int
        lib.oracle_threads.argtypes = []
        lib.oracle_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


class OracleError(RuntimeError):
    def __init__(self, status: int, what: str):
        super().__init__(f"{what}: oracle status {status}")
        self.status = status


def _dims_of(shape_tail):
    """numpy (.., [nz,] ny, nx) -> ndim, int64[3] (x, y, z)."""
    ndim = len(shape_tail)
    dims = list(reversed(shape_tail)) + [1] * (3 - ndim)
    return ndim, np.asarray(dims, dtype=np.int64)


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))


def _dx3(dx, ndim, dims):
    if dx is None:
        dx = [1.0 / float(dims[d]) for d in range(ndim)]
    dx = list(dx) + [1.0] * (3 - len(dx))
    return np.asarray(dx, dtype=np.float64)


def euler_run(U, nsteps, *, gamma=1.4, cfl=0.4, dx=None, scheme=RUSANOV1, bc=PERIODIC,
              allow_numeric=False):
    """Advance the conserved state U (ncomp, [nz,] ny, nx) by nsteps steps.

    Returns (U_new, info) with info = dict(t, dt_last, steps_done, status).
    """
    U = np.array(U, dtype=np.float64, order="C", copy=True)
    ndim, dims = _dims_of(U.shape[1:])
    assert U.shape[0] == ndim + 2
    dx3 = _dx3(dx, ndim, dims)
    t = ctypes.c_double(0.0)
    dtl = ctypes.c_double(0.0)
    done = ctypes.c_int64(0)
    st = _load().oracle_euler_run(ndim, _ip(dims), _dp(U), gamma, cfl, _dp(dx3), scheme, bc,
                                  int(nsteps), ctypes.byref(t), ctypes.byref(dtl),
                                  ctypes.byref(done))
    if st != OK and not (allow_numeric and st == NUMERIC):
        raise OracleError(st, "euler_run")
    return U, dict(t=t.value, dt_last=dtl.value, steps_done=done.value, status=st)


def euler_dt(U, *, gamma=1.4, cfl=0.4, dx=None):
    U = np.ascontiguousarray(U, dtype=np.float64)
    ndim, dims = _dims_of(U.shape[1:])
    dx3 = _dx3(dx, ndim, dims)
    out = ctypes.c_double(0.0)
    st = _load().oracle_euler_dt(ndim, _ip(dims), _dp(U), gamma, cfl, _dp(dx3), ctypes.byref(out))
    if st != OK:
        raise OracleError(st, "euler_dt")
    return out.value


def euler_step_cells(U, cells, *, gamma=1.4, cfl=0.4, dx=None, scheme=RUSANOV1, bc=PERIODIC,
                     dt=0.0):
    """One step from U evaluated only at the given linear interior cell indices.

    Returns (values (ncells, ncomp), dt_used).
    """
    U = np.ascontiguousarray(U, dtype=np.float64)
    ndim, dims = _dims_of(U.shape[1:])
    dx3 = _dx3(dx, ndim, dims)
    cells = np.ascontiguousarray(cells, dtype=np.int64)
    out = np.zeros((cells.size, ndim + 2), dtype=np.float64)
    dt_used = ctypes.c_double(0.0)
    st = _load().oracle_euler_step_cells(ndim, _ip(dims), _dp(U), gamma, cfl, _dp(dx3), scheme,
                                         bc, float(dt), cells.size, _ip(cells), _dp(out),
                                         ctypes.byref(dt_used))
    if st != OK:
        raise OracleError(st, "euler_step_cells")
    return out, dt_used.value


def eikonal_fmm(s, h, sources):
    """Fast Marching travel times for slowness s ([nz,] ny, nx), sources = list of
    cell coordinates (x, y[, z])."""
    s = np.ascontiguousarray(s, dtype=np.float64)
    ndim, dims = _dims_of(s.shape)
    lin = []
    for c in sources:
        c = list(c) + [0] * (3 - len(c))
        lin.append((c[2] * dims[1] + c[1]) * dims[0] + c[0])
    lin = np.asarray(lin, dtype=np.int64)
    T = np.empty_like(s)
    st = _load().oracle_eikonal_fmm(ndim, _ip(dims), _dp(s), float(h), lin.size, _ip(lin), _dp(T))
    if st != OK:
        raise OracleError(st, "eikonal_fmm")
    return T


def godunov(a, f):
    """Godunov upwind local solver for neighbour minima a (len 2 or 3) and f = s*h."""
    a = np.ascontiguousarray(a, dtype=np.float64)
    return _load().oracle_godunov(a.size, _dp(a), float(f))


def threads_used() -> int:
    """Threads the Euler steps run on (1 unless set_threads was called)."""
    return int(_load().oracle_threads())


def set_threads(n: int) -> int:
    """Let the Euler steps split their independent grid lines over n threads
    (results are bitwise the same for any n); returns the count in effect
    (1 if the oracle was built without OpenMP)."""
    return int(_load().oracle_set_threads(int(n)))


if __name__ == "__main__":  # pragma: no cover
    print(build(force="--force" in sys.argv))


def saxpy(a, x, y):
    """Section 7.1 (SAXPY): y + a x, in FP64.  FP32 operands make the product
    exact, so rounding the result once to FP32 gives the fused multiply-add of
    the same operands except when the FP64 sum itself rounded onto an FP32
    rounding midpoint (at most one unit in the last FP32 place)."""
    return np.asarray(y, dtype=np.float64) + np.float64(a) * np.asarray(x, dtype=np.float64)


def particle_update(p, dt, layout):
    """Section 7.2 (particle update in three dimensions): x_d + v_d dt for
    d = 0, 1, 2 of n particles held as 6n numbers, in FP64.
    layout "aos" ("contiguous"): record r = (x0 x1 x2 v0 v1 v2) at [6r, 6r+6);
    layout "soa" ("strided"): component d at [d n, d n + n).
    Returns the updated 6n array (velocities unchanged)."""
    q = np.array(p, dtype=np.float64).reshape(-1)
    n = q.size // 6
    if layout == "aos":
        r = q.reshape(n, 6)
        for d in range(3):
            r[:, d] = r[:, d] + r[:, 3 + d] * np.float64(dt)
    else:
        r = q.reshape(6, n)
        for d in range(3):
            r[d] = r[d] + r[3 + d] * np.float64(dt)
    return q
