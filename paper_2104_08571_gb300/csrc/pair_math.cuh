// Packed FP32 pair arithmetic for sm_103a (add/sub/mul/fma.rn.f32x2) and the
// Euler physics written once for a scalar float or a pair of floats.
//
// A pair holds the same quantity of two neighbouring cells; every
// multiply/add of the flux, reconstruction and update arithmetic then issues
// once for both cells.  Comparisons, selects, reciprocal and square root act
// per lane.  With V = float the functions below are ordinary scalar code.
#pragma once
#include <cstdint>

namespace ripple {

struct f2 {
    float x, y;
};

__device__ __forceinline__ unsigned long long pk(f2 a)
{
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a.x), "f"(a.y));
    return r;
}
__device__ __forceinline__ f2 upk(unsigned long long r)
{
    f2 a;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a.x), "=f"(a.y) : "l"(r));
    return a;
}
__device__ __forceinline__ f2 operator+(f2 a, f2 b)
{
    unsigned long long r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(pk(a)), "l"(pk(b)));
    return upk(r);
}
__device__ __forceinline__ f2 operator-(f2 a, f2 b)
{
    unsigned long long r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(pk(a)), "l"(pk(b)));
    return upk(r);
}
__device__ __forceinline__ f2 operator*(f2 a, f2 b)
{
    unsigned long long r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(pk(a)), "l"(pk(b)));
    return upk(r);
}
__device__ __forceinline__ f2 fma_v(f2 a, f2 b, f2 c)
{
    unsigned long long r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(pk(a)), "l"(pk(b)), "l"(pk(c)));
    return upk(r);
}
__device__ __forceinline__ float fma_v(float a, float b, float c) { return fmaf(a, b, c); }

template <typename V>
__device__ __forceinline__ V splat(float s);
template <>
__device__ __forceinline__ float splat<float>(float s) { return s; }
template <>
__device__ __forceinline__ f2 splat<f2>(float s) { return f2{s, s}; }

__device__ __forceinline__ float rcp_v(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ f2 rcp_v(f2 a) { return f2{rcp_v(a.x), rcp_v(a.y)}; }
__device__ __forceinline__ float sqrt_v(float x)
{
    float r;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ f2 sqrt_v(f2 a) { return f2{sqrt_v(a.x), sqrt_v(a.y)}; }
__device__ __forceinline__ float abs_v(float a) { return fabsf(a); }
__device__ __forceinline__ f2 abs_v(f2 a) { return f2{fabsf(a.x), fabsf(a.y)}; }
__device__ __forceinline__ float max_v(float a, float b) { return fmaxf(a, b); }
__device__ __forceinline__ f2 max_v(f2 a, f2 b) { return f2{fmaxf(a.x, b.x), fmaxf(a.y, b.y)}; }
__device__ __forceinline__ float min_lanes(float a) { return a; }
__device__ __forceinline__ float min_lanes(f2 a) { return fminf(a.x, a.y); }
__device__ __forceinline__ float max_lanes(float a) { return a; }
__device__ __forceinline__ float max_lanes(f2 a) { return fmaxf(a.x, a.y); }

__device__ __forceinline__ float minmod_s(float a, float b)
{
    // minmod(a, b) (0 if the one-sided differences disagree in sign, else the
    // one of smaller magnitude) is the median of a, b and 0: three min/max
    // operations and no compare-and-select
    return fmaxf(fminf(a, b), fminf(fmaxf(a, b), 0.f));
}
__device__ __forceinline__ float minmod_v(float a, float b) { return minmod_s(a, b); }
__device__ __forceinline__ f2 minmod_v(f2 a, f2 b) { return f2{minmod_s(a.x, b.x), minmod_s(a.y, b.y)}; }

// Three-operand minimum (one ALU instruction on sm_100 and later).
__device__ __forceinline__ float min3f(float a, float b, float c)
{
    float r;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}

// Smallest density/pressure of four states into chk (both lanes).  Items that
// reach beyond a field's ghost layers read NaN (padding and out-of-tensor
// cells are NaN), which the minimum ignores, so no per-lane domain predicate
// is needed.  A NaN produced from in-domain data is skipped here too but
// reaches the updated cells, whose own check catches it.
__device__ __forceinline__ void track4(float& chk, float a, float b, float c, float d)
{
    chk = min3f(chk, min3f(a, b, c), d);
}
__device__ __forceinline__ void track4(float& chk, f2 a, f2 b, f2 c, f2 d)
{
    const float m0 = min3f(a.x, b.x, c.x), m1 = min3f(a.y, b.y, c.y);
    chk = min3f(chk, min3f(m0, m1, d.x), d.y);
}

// Physical flux along axis D; also returns 1/rho, the normal velocity, the pressure.
template <typename V, int DIM, int D>
__device__ __forceinline__ void pflux(const V (&q)[DIM + 2], V gm1, V (&F)[DIM + 2], V& inv_rho, V& un, V& p)
{
    inv_rho = rcp_v(q[0]);
    V mm = q[1] * q[1];
#pragma unroll
    for (int e = 1; e < DIM; ++e) mm = fma_v(q[1 + e], q[1 + e], mm);
    p = gm1 * fma_v(splat<V>(-0.5f), mm * inv_rho, q[DIM + 1]);
    un = q[1 + D] * inv_rho;
    F[0] = q[1 + D];
#pragma unroll
    for (int e = 0; e < DIM; ++e) F[1 + e] = e == D ? fma_v(q[1 + e], un, p) : q[1 + e] * un;
    F[DIM + 1] = (q[DIM + 1] + p) * un;
}

// Wave-speed sums sum_d (|u_d| + c)/dx_d of a pair of conserved states and
// their admissibility (density and pressure > 0) per lane.  Products and sums
// are separate roundings (packed mul/add are never contracted), so the sum
// does not depend on the order of the axes.
template <int DIM>
__device__ __forceinline__ f2 wave_sum2(const f2 (&q)[DIM + 2], f2 gamma, f2 gm1, const f2 (&inv_dx)[3], bool& ok0,
                                        bool& ok1)
{
    const f2 inv_rho = rcp_v(q[0]);
    f2 mm = q[1] * q[1];
#pragma unroll
    for (int e = 1; e < DIM; ++e) mm = fma_v(q[1 + e], q[1 + e], mm);
    const f2 p = gm1 * fma_v(splat<f2>(-0.5f), mm * inv_rho, q[DIM + 1]);
    ok0 = (q[0].x > 0.f) & (p.x > 0.f);
    ok1 = (q[0].y > 0.f) & (p.y > 0.f);
    const f2 c = sqrt_v(gamma * p * inv_rho);
    f2 s = (abs_v(q[1] * inv_rho) + c) * inv_dx[0];
#pragma unroll
    for (int d = 1; d < DIM; ++d) s = s + (abs_v(q[1 + d] * inv_rho) + c) * inv_dx[d];
    return s;
}

// Rusanov face flux along D between left states a and right states b;
// the smallest density/pressure of both goes to chk.
template <typename V, int DIM, int D>
__device__ __forceinline__ void rus(const V (&a)[DIM + 2], const V (&b)[DIM + 2], V gamma, V gm1, V (&F)[DIM + 2],
                                    float& chk)
{
    V Fa[DIM + 2], Fb[DIM + 2], ia, ua, pa, ib, ub, pb;
    pflux<V, DIM, D>(a, gm1, Fa, ia, ua, pa);
    pflux<V, DIM, D>(b, gm1, Fb, ib, ub, pb);
    track4(chk, a[0], pa, b[0], pb);
    const V ca = sqrt_v(gamma * pa * ia);
    const V cb = sqrt_v(gamma * pb * ib);
    const V s = max_v(abs_v(ua) + ca, abs_v(ub) + cb);
    const V half = splat<V>(0.5f);
#pragma unroll
    for (int m = 0; m < DIM + 2; ++m) F[m] = half * fma_v(s, a[m] - b[m], Fa[m] + Fb[m]);
}

// FORCE face flux along D (Toro): the mean of the Lax-Friedrichs flux and
// the flux of the Richtmyer state q = (a + b)/2 - (dt/dx)/2 (F(b) - F(a));
// dtdx = dt/dx, inv_dtdx = dx/dt.  Admissibility of a and b goes to chk (q is
// an intermediate of the formula).  Products and sums round separately, so
// the x and y faces of transposed data give transposed results.
template <typename V, int DIM, int D>
__device__ __forceinline__ void force(const V (&a)[DIM + 2], const V (&b)[DIM + 2], V gm1, V half_dtdx,
                                      V half_inv_dtdx, V (&F)[DIM + 2], float& chk)
{
    V Fa[DIM + 2], Fb[DIM + 2], q[DIM + 2], Fq[DIM + 2], ia, ua, pa, ib, ub, pb, iq, uq, pq;
    pflux<V, DIM, D>(a, gm1, Fa, ia, ua, pa);
    pflux<V, DIM, D>(b, gm1, Fb, ib, ub, pb);
    track4(chk, a[0], pa, b[0], pb);
    const V half = splat<V>(0.5f);
#pragma unroll
    for (int m = 0; m < DIM + 2; ++m) q[m] = half * (a[m] + b[m]) - half_dtdx * (Fb[m] - Fa[m]);
    pflux<V, DIM, D>(q, gm1, Fq, iq, uq, pq);
#pragma unroll
    for (int m = 0; m < DIM + 2; ++m) F[m] = half * (half * (Fa[m] + Fb[m]) - half_inv_dtdx * (b[m] - a[m]) + Fq[m]);
}

// MUSCL-Hancock face states of cells along D from (left, centre, right).
template <typename V, int DIM, int D>
__device__ __forceinline__ void muscl(const V (&qm)[DIM + 2], const V (&q)[DIM + 2], const V (&qp)[DIM + 2], V gm1,
                                      V half_dtdx, V (&L)[DIM + 2], V (&R)[DIM + 2], float& chk)
{
    const V half = splat<V>(0.5f), mhalf = splat<V>(-0.5f);
#pragma unroll
    for (int m = 0; m < DIM + 2; ++m) {
        const V slope = minmod_v(q[m] - qm[m], qp[m] - q[m]);
        L[m] = fma_v(mhalf, slope, q[m]);
        R[m] = fma_v(half, slope, q[m]);
    }
    V FL[DIM + 2], FR[DIM + 2], il, ir, u, pl, pr;
    pflux<V, DIM, D>(L, gm1, FL, il, u, pl);
    pflux<V, DIM, D>(R, gm1, FR, ir, u, pr);
    track4(chk, L[0], pl, R[0], pr);
#pragma unroll
    for (int m = 0; m < DIM + 2; ++m) {
        const V inc = half_dtdx * (FL[m] - FR[m]);
        L[m] = L[m] + inc;
        R[m] = R[m] + inc;
    }
}

}  // namespace ripple
