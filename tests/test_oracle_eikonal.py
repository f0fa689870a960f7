"""Pins of the FP64 eikonal oracle (Fast Marching with the Godunov upwind solver).

Independent checks, each catching a different plausible mistake:
  * Godunov closed forms (1-, 2-, 3-term cases)   -- wrong quadratic, wrong sort
  * 1-D strip: T = sum of h*s exactly             -- wrong f = s*h, off-by-one
  * axis lines through a point source: k*h        -- wrong neighbour along an axis
  * refinement towards |x - x0|                    -- wrong h, wrong geometry
  * Jacobi iteration to its bitwise fixed point     -- FMM ordering / acceptance bugs
  * 4-neighbour graph-Dijkstra upper bound          -- an update that overshoots
The Jacobi and Dijkstra references below are written independently of the
oracle (general m-term quadratic, plain heapq).
"""
import heapq
import math

import numpy as np
import pytest

import inputs


def _godunov_general(a, f):
    """Upwind solution of sum_{i<=m} (T - a_i)^2 = f^2 over the smallest m a's
    for which the root exceeds a_m (general form, test-side)."""
    a = sorted(a)
    best = a[0] + f
    for m in range(2, len(a) + 1):
        if best <= a[m - 1]:
            break
        s = sum(a[:m])
        q = sum(x * x for x in a[:m])
        disc = s * s - m * (q - f * f)
        best = (s + math.sqrt(max(disc, 0.0))) / m
    return best


def test_godunov_closed_forms(oracle_lib):
    f = 0.3
    # one-sided: |a - b| >= f
    assert oracle_lib.godunov([1.0, 5.0], f) == 1.0 + f
    assert oracle_lib.godunov([math.inf, 2.0], f) == 2.0 + f
    assert oracle_lib.godunov([math.inf, math.inf], f) == math.inf
    # symmetric two-sided: T = a + f / sqrt(2)
    assert oracle_lib.godunov([1.0, 1.0], f) == pytest.approx(1.0 + f / math.sqrt(2.0), rel=1e-15)
    # 3D all equal: T = a + f / sqrt(3)
    assert oracle_lib.godunov([2.0, 2.0, 2.0], f) == pytest.approx(2.0 + f / math.sqrt(3.0),
                                                                   rel=1e-15)
    # 3D: two equal and one far -> 2-term solution
    assert oracle_lib.godunov([2.0, 9.0, 2.0], f) == pytest.approx(2.0 + f / math.sqrt(2.0),
                                                                   rel=1e-15)
    # the result solves its quadratic: sum over upwind terms (T - a)^2 = f^2
    rng = inputs.uniform(5, 300).reshape(100, 3)
    for row in rng:
        a = list(row * 0.5)
        T = oracle_lib.godunov(a, f)
        assert T == pytest.approx(_godunov_general(a, f), rel=1e-13, abs=1e-15)
        up = [x for x in a if x < T]
        assert sum((T - x) ** 2 for x in up) == pytest.approx(f * f, rel=1e-12)


def test_strip_exact_unit_and_variable_speed(oracle_lib):
    n = 64
    h = 1.0 / n
    s = np.ones((1, n))
    T = oracle_lib.eikonal_fmm(s, h, [(17, 0)])
    k = np.abs(np.arange(n) - 17)
    assert np.array_equal(T[0], k * h)
    # variable slowness: T(i) = sum over the path of h * s(receiving cell)
    s = inputs.eikonal_slowness((n, 1), seed=3)
    T = oracle_lib.eikonal_fmm(s, h, [(40, 0)])
    ref = np.zeros(n)
    for i in range(41, n):
        ref[i] = ref[i - 1] + s[0, i] * h
    for i in range(39, -1, -1):
        ref[i] = ref[i + 1] + s[0, i] * h
    assert np.array_equal(T[0], ref)


@pytest.mark.parametrize("ndim,n", [(2, 33), (3, 17)])
def test_axis_lines_exact(oracle_lib, ndim, n):
    h = 1.0 / 32.0
    s = np.ones((n,) * ndim)
    c = n // 2
    T = oracle_lib.eikonal_fmm(s, h, [(c,) * ndim])
    k = np.abs(np.arange(n) - c) * h
    for axis in range(ndim):
        sl = [c] * ndim
        sl[ndim - 1 - axis] = slice(None)
        assert np.array_equal(T[tuple(sl)], k)


def test_refinement_towards_distance(oracle_lib):
    errs = []
    for n in (33, 65, 129):
        h = 1.0 / (n - 1)
        c = n // 2
        T = oracle_lib.eikonal_fmm(np.ones((n, n)), h, [(c, c)])
        x = (np.arange(n) - c) * h
        dist = np.sqrt(x[None, :] ** 2 + x[:, None] ** 2)
        err = np.max(np.abs(T - dist))
        # first-order upwind on a point source: error O(h log(1/h)), and T >= dist
        assert err <= 2.0 * h * math.log(1.0 / h) + h
        assert np.all(T >= dist - 1e-12)
        errs.append(err)
    assert errs[0] > errs[1] > errs[2]


def _jacobi_fixed_point(s, h, sources):
    ndim = s.ndim
    T = np.full(s.shape, np.inf)
    fixed = np.zeros(s.shape, bool)
    for c in sources:
        idx = tuple(reversed(c))
        T[idx] = 0.0
        fixed[idx] = True
    for _ in range(10 * s.size):
        new = T.copy()
        for idx in np.ndindex(s.shape):
            if fixed[idx]:
                continue
            a = []
            for ax in range(ndim):
                best = np.inf
                for sd in (-1, 1):
                    j = list(idx)
                    j[ax] += sd
                    if 0 <= j[ax] < s.shape[ax]:
                        best = min(best, T[tuple(j)])
                a.append(best)
            new[idx] = min(T[idx], _godunov_general(a, s[idx] * h))
        if np.array_equal(new, T):
            return T
        T = new
    raise AssertionError("Jacobi did not reach a fixed point")


@pytest.mark.parametrize("dims,seed", [((16, 16), 1), ((13, 9), 2), ((7, 6, 5), 3)])
def test_fmm_equals_jacobi_fixed_point(oracle_lib, dims, seed):
    s = inputs.eikonal_slowness(dims, seed=seed)
    src = inputs.eikonal_sources(dims, seed=seed)
    h = 1.0 / max(dims)
    T = oracle_lib.eikonal_fmm(s, h, src)
    J = _jacobi_fixed_point(s, h, src)
    np.testing.assert_allclose(T, J, rtol=1e-14, atol=1e-15)


def _graph_dijkstra(s, h, sources):
    shape = s.shape
    D = np.full(shape, np.inf)
    pq = []
    for c in sources:
        idx = tuple(reversed(c))
        D[idx] = 0.0
        heapq.heappush(pq, (0.0, idx))
    while pq:
        d, idx = heapq.heappop(pq)
        if d > D[idx]:
            continue
        for ax in range(len(shape)):
            for sd in (-1, 1):
                j = list(idx)
                j[ax] += sd
                if 0 <= j[ax] < shape[ax]:
                    j = tuple(j)
                    nd = d + h * s[j]
                    if nd < D[j]:
                        D[j] = nd
                        heapq.heappush(pq, (nd, j))
    return D


@pytest.mark.parametrize("dims,seed", [((16, 16), 4), ((12, 10, 6), 5)])
def test_below_graph_dijkstra(oracle_lib, dims, seed):
    s = inputs.eikonal_slowness(dims, seed=seed)
    src = inputs.eikonal_sources(dims, seed=seed)
    h = 1.0 / max(dims)
    T = oracle_lib.eikonal_fmm(s, h, src)
    D = _graph_dijkstra(s, h, src)
    assert np.all(T <= D * (1 + 1e-15))
    assert np.all(np.isfinite(T))
    for c in src:
        assert T[tuple(reversed(c))] == 0.0
