"""Seeded synthetic inputs shared, as data only, by the oracle tests and the CUDA path.

This module holds no step of the method: it only draws random numbers and
writes down initial states.  Both sides receive the arrays it returns.

Random numbers: counter-based SplitMix64 (Steele, Lea & Flood, "Fast
splittable pseudorandom number generators", OOPSLA 2014) applied to
``seed * 2**32 + counter``; uniforms take the top 53 bits / 2**53, Gaussians
use Box-Muller on two independent uniform streams.  The draw for a cell
depends only on (seed, cell index), never on thread count or order.

Workload recipes (the paper's benchmarks are synthetic PDE states, Sections
7.3-7.4 and 8; no dataset is involved):
  * ``euler2d_sine``      2D advected density wave: rho = 1 + A sin(2 pi x) sin(2 pi y),
                          u = 1, v = 0.5, p = 1, periodic, on [0,1]^2.
  * ``euler3d_blast``     spherical blast: rho = 1, p = 1 inside r < 0.2 around the
                          centre, else rho = 0.125, p = 0.1; zero velocity;
                          rho multiplied by (1 + 0.01 (2 xi - 1)), xi uniform per cell.
  * ``sod``               Sod shock tube along one axis (rho,u,p) = (1,0,1) | (0.125,0,0.1).
  * ``uniform_state``     constant state.
  * ``eikonal_slowness``  s = exp(0.5 g), g = i.i.d. N(0,1) per cell smoothed by a
                          periodic 3-wide box mean (3x3 in 2D, 3x3x3 in 3D).
  * ``eikonal_sources``   1-4 distinct random cells.
  * ``batch_problems``    per-instance sides log-uniform in [32, 512], amplitudes in
                          [0.05, 0.3].
  * ``serve_stream``      Poisson arrivals of mixed Euler / eikonal requests.
All Euler states are returned as conserved variables (rho, rho u_1.., E) with
E = p/(gamma - 1) + rho |u|^2 / 2, component-major, x fastest.
"""
from __future__ import annotations

import math

import numpy as np

_MASK64 = np.uint64(0xFFFFFFFFFFFFFFFF)


def splitmix64(x: np.ndarray) -> np.ndarray:
    """SplitMix64 output function for a uint64 counter array."""
    with np.errstate(over="ignore"):
        z = (x + np.uint64(0x9E3779B97F4A7C15)) & _MASK64
        z = ((z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)) & _MASK64
        z = ((z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)) & _MASK64
        return z ^ (z >> np.uint64(31))


def uniform(seed: int, n: int, stream: int = 0) -> np.ndarray:
    """n uniforms in [0, 1) for counters 0..n-1 of (seed, stream)."""
    base = (np.uint64(seed) << np.uint64(32)) + (np.uint64(stream) << np.uint64(56))
    ctr = base + np.arange(n, dtype=np.uint64)
    bits = splitmix64(ctr) >> np.uint64(11)
    return bits.astype(np.float64) * (1.0 / 9007199254740992.0)


def normal(seed: int, n: int) -> np.ndarray:
    """n standard normals (Box-Muller on streams 1 and 2)."""
    u1 = uniform(seed, n, stream=1)
    u2 = uniform(seed, n, stream=2)
    return np.sqrt(-2.0 * np.log1p(-u1)) * np.cos(2.0 * math.pi * u2)


def cell_centres(n: int) -> np.ndarray:
    return (np.arange(n, dtype=np.float64) + 0.5) / n


def conserved(rho, vel, p, gamma=1.4):
    """Stack primitives into conserved variables; vel is a list of arrays (x first)."""
    rho = np.asarray(rho, dtype=np.float64)
    comps = [rho]
    ke = np.zeros_like(rho)
    for u in vel:
        u = np.broadcast_to(np.asarray(u, dtype=np.float64), rho.shape)
        comps.append(rho * u)
        ke = ke + rho * u * u
    E = np.broadcast_to(np.asarray(p, dtype=np.float64), rho.shape) / (gamma - 1.0) + 0.5 * ke
    comps.append(E)
    return np.ascontiguousarray(np.stack(comps))


def euler2d_sine(n: int, amp: float = 0.2, u: float = 1.0, v: float = 0.5, p: float = 1.0,
                 gamma: float = 1.4, ny: int | None = None) -> np.ndarray:
    """(4, ny, n) state: rho = 1 + amp sin(2 pi x) sin(2 pi y), uniform u, v, p."""
    ny = n if ny is None else ny
    x = cell_centres(n)[None, :]
    y = cell_centres(ny)[:, None]
    rho = 1.0 + amp * np.sin(2.0 * math.pi * x) * np.sin(2.0 * math.pi * y)
    return conserved(rho, [u, v], p, gamma)


def euler3d_blast(n: int, seed: int = 1, gamma: float = 1.4, noise: float = 0.01,
                  radius: float = 0.2, dims: tuple | None = None) -> np.ndarray:
    """(5, nz, ny, nx) spherical blast with multiplicative uniform noise on rho."""
    nx, ny, nz = dims if dims is not None else (n, n, n)
    x = cell_centres(nx)[None, None, :]
    y = cell_centres(ny)[None, :, None]
    z = cell_centres(nz)[:, None, None]
    r = np.sqrt((x - 0.5) ** 2 + (y - 0.5) ** 2 + (z - 0.5) ** 2)
    inside = r < radius
    rho = np.where(inside, 1.0, 0.125)
    p = np.where(inside, 1.0, 0.1)
    if noise:
        xi = uniform(seed, nx * ny * nz).reshape(nz, ny, nx)
        rho = rho * (1.0 + noise * (2.0 * xi - 1.0))
    zero = np.zeros_like(rho)
    return conserved(rho, [zero, zero, zero], p, gamma)


def sod(ndim: int, n: int, axis: int = 0, ntrans: int = 4, gamma: float = 1.4) -> np.ndarray:
    """Sod tube along `axis` with `ntrans` cells on the other axes."""
    shape = [ntrans] * ndim  # (x, y[, z]) extents
    shape[axis] = n
    npshape = tuple(reversed(shape))
    xa = cell_centres(n)
    idx = [None] * ndim
    idx[ndim - 1 - axis] = slice(None)
    xs = np.broadcast_to(xa[tuple(idx)], npshape)
    left = xs < 0.5
    rho = np.where(left, 1.0, 0.125)
    p = np.where(left, 1.0, 0.1)
    zero = np.zeros(npshape)
    return conserved(rho, [zero] * ndim, p, gamma)


def uniform_state(dims, rho: float, vel, p: float, gamma: float = 1.4) -> np.ndarray:
    """dims = (nx, ny[, nz]); vel has one entry per axis."""
    npshape = tuple(reversed(dims))
    return conserved(np.full(npshape, rho), list(vel), p, gamma)


def eikonal_slowness(dims, seed: int = 1) -> np.ndarray:
    """s = exp(0.5 * box3(g)), g ~ N(0,1) i.i.d., periodic 3-wide box mean."""
    npshape = tuple(reversed(dims))
    g = normal(seed, int(np.prod(npshape))).reshape(npshape)
    acc = np.zeros_like(g)
    ndim = len(npshape)
    offsets = np.stack(np.meshgrid(*([np.arange(-1, 2)] * ndim), indexing="ij"), -1)
    offsets = offsets.reshape(-1, ndim)
    for off in offsets:
        acc += np.roll(g, shift=tuple(int(o) for o in off), axis=tuple(range(ndim)))
    return np.exp(0.5 * acc / len(offsets))


def eikonal_sources(dims, seed: int = 1, count: int | None = None):
    """1-4 distinct cells (count drawn from the seed unless given), as (x, y[, z])."""
    total = int(np.prod(dims))
    u = uniform(seed, 64, stream=3)
    if count is None:
        count = 1 + int(u[0] * 4.0)
    chosen = []
    k = 1
    while len(chosen) < count:
        lin = int(u[k] * total) % total
        k += 1
        if lin not in chosen:
            chosen.append(lin)
    out = []
    for lin in chosen:
        c = []
        rem = lin
        for d in dims:
            c.append(rem % d)
            rem //= d
        out.append(tuple(c))
    return out


def batch_problems(count: int = 512, seed: int = 1, lo: int = 32, hi: int = 512):
    """Per-instance (side, amplitude) with side = floor(exp(U(ln lo, ln hi)))."""
    u = uniform(seed, count, stream=4)
    a = uniform(seed, count, stream=5)
    sides = np.floor(np.exp(math.log(lo) + u * (math.log(hi) - math.log(lo)))).astype(np.int64)
    sides = np.clip(sides, lo, hi)
    amps = 0.05 + a * 0.25
    return [(int(s), float(x)) for s, x in zip(sides, amps)]


def serve_stream(rate: float, count: int, seed: int = 1):
    """Poisson arrivals of mixed requests (70 % Euler, 30 % eikonal).

    Returns a list of dicts: t (arrival s), kind ('euler'|'eikonal'), side,
    steps (Euler), amp (Euler), nsrc (eikonal), seed (per request).
    """
    ua = uniform(seed, count, stream=6)
    uk = uniform(seed, count, stream=7)
    us = uniform(seed, count, stream=8)
    un = uniform(seed, count, stream=9)
    um = uniform(seed, count, stream=10)
    t = np.cumsum(-np.log1p(-ua) / rate)
    reqs = []
    for i in range(count):
        if uk[i] < 0.7:
            side = int(math.floor(math.exp(math.log(64) + us[i] * (math.log(1024) - math.log(64)))))
            reqs.append(dict(t=float(t[i]), kind="euler", side=min(side, 1024),
                             steps=50 + int(un[i] * 451) % 451, amp=0.05 + 0.25 * um[i],
                             seed=seed * 100003 + i))
        else:
            side = int(math.floor(math.exp(math.log(128) + us[i] * (math.log(1024) - math.log(128)))))
            reqs.append(dict(t=float(t[i]), kind="eikonal", side=min(side, 1024),
                             nsrc=1 + int(un[i] * 4) % 4, seed=seed * 100003 + i))
    return reqs


def to_aos(U: np.ndarray) -> np.ndarray:
    """Component-major (ncomp, ...) -> cell-major (..., ncomp) contiguous."""
    return np.ascontiguousarray(np.moveaxis(U, 0, -1))


def from_aos(A: np.ndarray) -> np.ndarray:
    return np.ascontiguousarray(np.moveaxis(A, -1, 0))
