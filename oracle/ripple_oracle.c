/*
 * FP64 CPU oracle for the halo-padded stencil sweeps of Ripple (arXiv 2104.08571).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or call
 * this file: only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline
 * leg (and bench.py --impl reference) use it.  It shares no code, header,
 * table or helper with the CUDA library.
 *
 * Plain, slow, obviously correct: double precision, scalar loops, compiled
 * with -ffp-contract=off so that x86-64 and aarch64 give identical bits.  One
 * thread by default; oracle_set_threads(n) lets OpenMP split the independent
 * grid lines (and cells) of an Euler step over n threads.  Every cell's value
 * is computed by the same operations in the same order whatever the thread
 * count, and a maximum is exact, so the results do not depend on it.
 *
 * What it computes
 *  - Euler (2D/3D, conserved variables (rho, rho*u_1..rho*u_d, E), ideal gas):
 *    the step ordering of the paper's Euler solver graph (Section 7.4,
 *    Listing "euler_graph"): wave speeds -> max reduction -> dt -> boundary
 *    (padding) fill -> flux-difference update (the flux difference of
 *    Section 7.3) -> swap.  Readings where the paper is silent:
 *      * the update is unsplit (all directions summed in one pass, as in the
 *        flux-difference kernel of Section 7.3);
 *      * the face flux is Rusanov (local Lax-Friedrichs);
 *      * dt = CFL / max_cells sum_d (|u_d| + c) / dx_d from the state at the
 *        start of the step;
 *      * second order: MUSCL-Hancock in conserved variables, component-wise
 *        minmod slopes, per-direction half-step predictor;
 *      * the paper's own solver (Listing euler_graph) is also provided: a
 *        dimensionally split step (x, then y, then z sweeps, padding refilled
 *        before each) with the FORCE face flux of Section 7.3;
 *      * padding fills (Section 4.1 names "constant extrapolation"):
 *        periodic, or transmissive = every ghost layer copies the edge cell;
 *      * a non-positive (or NaN) density or pressure anywhere (cell,
 *        reconstructed or predicted state) stops the run with status 6.
 *  - Eikonal |grad T| s = 1 (Section 7.4, the Hamiltonian with speed f = 1/s):
 *    the Godunov upwind fixed point, computed directly by Fast Marching
 *    (Sethian 1996, cited in Section 7.4): Dijkstra-ordered acceptance with the
 *    Godunov local solver, outside-domain neighbours = +inf, sources fixed at 0.
 *
 * Array convention at the interface: interior cells only, component-major
 * ("strided"/SoA in the paper's Section 4.2 words), x fastest:
 *   U[((c * nz + k) * ny + j) * nx + i].
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_OK 0
#define ORACLE_INVALID 1
#define ORACLE_OOM 2
#define ORACLE_NUMERIC 6

#define SCHEME_RUSANOV1 0
#define SCHEME_MUSCL_HANCOCK 1
#define SCHEME_FORCE_SPLIT 2
#define BC_PERIODIC 0
#define BC_TRANSMISSIVE 1

#define MAXC 5 /* at most 3D: rho, 3 momenta, E */

/* ------------------------------------------------------------------------ */
/* Padded grid (Section 4.1: tensor with padding cells).                     */
/* ------------------------------------------------------------------------ */
typedef struct {
    int ndim;
    int64_t n[3]; /* interior cells per axis (1 on unused axes) */
    int h;        /* ghost layers on each side of every active axis */
    int64_t p[3]; /* padded extents */
    int64_t ncell;
} grid_t;

static int grid_init(grid_t* g, int ndim, const int64_t* n, int h)
{
    if (ndim < 2 || ndim > 3 || h < 0) return ORACLE_INVALID;
    g->ndim = ndim;
    g->h = h;
    g->ncell = 1;
    for (int d = 0; d < 3; d++) {
        g->n[d] = d < ndim ? n[d] : 1;
        if (g->n[d] < 1) return ORACLE_INVALID;
        g->p[d] = d < ndim ? g->n[d] + 2 * h : 1;
        g->ncell *= g->p[d];
    }
    return ORACLE_OK;
}

/* Linear padded index of interior coordinate c (each c[d] in [-h, n[d]+h)). */
static int64_t pidx(const grid_t* g, const int64_t* c)
{
    int64_t i = c[0] + g->h;
    int64_t j = c[1] + g->h;
    int64_t k = g->ndim > 2 ? c[2] + g->h : 0;
    return (k * g->p[1] + j) * g->p[0] + i;
}

static void load_cell(const grid_t* g, const double* U, int ncomp, const int64_t* c, double* q)
{
    int64_t id = pidx(g, c);
    for (int m = 0; m < ncomp; m++) q[m] = U[m * g->ncell + id];
}

/* Copy interior-only component-major array into a padded one (ghosts zeroed). */
static void to_padded(const grid_t* g, int ncomp, const double* Uint, double* U)
{
    memset(U, 0, sizeof(double) * (size_t)(g->ncell * ncomp));
    int64_t c[3] = {0, 0, 0};
    int64_t nint = g->n[0] * g->n[1] * g->n[2];
    for (int m = 0; m < ncomp; m++)
        for (c[2] = 0; c[2] < g->n[2]; c[2]++)
            for (c[1] = 0; c[1] < g->n[1]; c[1]++)
                for (c[0] = 0; c[0] < g->n[0]; c[0]++)
                    U[m * g->ncell + pidx(g, c)] =
                        Uint[m * nint + (c[2] * g->n[1] + c[1]) * g->n[0] + c[0]];
}

static void from_padded(const grid_t* g, int ncomp, const double* U, double* Uint)
{
    int64_t c[3] = {0, 0, 0};
    int64_t nint = g->n[0] * g->n[1] * g->n[2];
    for (int m = 0; m < ncomp; m++)
        for (c[2] = 0; c[2] < g->n[2]; c[2]++)
            for (c[1] = 0; c[1] < g->n[1]; c[1]++)
                for (c[0] = 0; c[0] < g->n[0]; c[0]++)
                    Uint[m * nint + (c[2] * g->n[1] + c[1]) * g->n[0] + c[0]] =
                        U[m * g->ncell + pidx(g, c)];
}

/*
 * Padding fill (Section 4.1; Listing "euler_graph" set_boundary).
 * Axis by axis; along axis d every ghost coordinate takes the value of its
 * source cell: periodic wrap, or the nearest edge cell (constant
 * extrapolation).  The other axes run over their full padded range, so that
 * after the last axis even edge/corner ghosts are defined.
 */
static void fill_padding(const grid_t* g, double* U, int ncomp, int bc)
{
    int64_t lo[3], hi[3];
    for (int e = 0; e < 3; e++) {
        lo[e] = e < g->ndim ? -g->h : 0;
        hi[e] = e < g->ndim ? g->n[e] + g->h : 1;
    }
    for (int d = 0; d < g->ndim; d++) {
        int64_t c[3];
        for (c[2] = lo[2]; c[2] < hi[2]; c[2]++)
            for (c[1] = lo[1]; c[1] < hi[1]; c[1]++)
                for (c[0] = lo[0]; c[0] < hi[0]; c[0]++) {
                    if (c[d] >= 0 && c[d] < g->n[d]) continue;
                    int64_t s[3] = {c[0], c[1], c[2]};
                    if (bc == BC_PERIODIC)
                        s[d] = ((c[d] % g->n[d]) + g->n[d]) % g->n[d];
                    else
                        s[d] = c[d] < 0 ? 0 : g->n[d] - 1;
                    int64_t dst = pidx(g, c), src = pidx(g, s);
                    for (int m = 0; m < ncomp; m++)
                        U[m * g->ncell + dst] = U[m * g->ncell + src];
                }
    }
}

/* ------------------------------------------------------------------------ */
/* Ideal-gas Euler physics.                                                  */
/* ------------------------------------------------------------------------ */

/* Primitive variables of a conserved state: rho, velocity, pressure. */
static void primitives(int ndim, const double* q, double gamma, double* rho, double* u, double* p)
{
    double kinetic = 0.0;
    *rho = q[0];
    for (int d = 0; d < ndim; d++) {
        u[d] = q[1 + d] / q[0];
        kinetic += q[1 + d] * u[d];
    }
    *p = (gamma - 1.0) * (q[ndim + 1] - 0.5 * kinetic);
}

static int admissible(double rho, double p) { return rho > 0.0 && p > 0.0; }

/* Physical flux of the Euler equations along axis d. */
static void physical_flux(int ndim, int d, const double* q, double gamma, double* F)
{
    double rho, u[3], p;
    primitives(ndim, q, gamma, &rho, u, &p);
    F[0] = q[1 + d];
    for (int e = 0; e < ndim; e++) F[1 + e] = q[1 + e] * u[d] + (e == d ? p : 0.0);
    F[ndim + 1] = (q[ndim + 1] + p) * u[d];
}

/*
 * Rusanov (local Lax-Friedrichs) face flux between left state qL and right
 * state qR along axis d:  F* = (F(qL) + F(qR))/2 - s_max (qR - qL)/2,
 * s_max = max(|u_d,L| + c_L, |u_d,R| + c_R).  Returns 0 if a state is not
 * admissible.
 */
static int rusanov(int ndim, int d, const double* qL, const double* qR, double gamma, double* F)
{
    int ncomp = ndim + 2;
    double rl, ul[3], pl, rr, ur[3], pr;
    primitives(ndim, qL, gamma, &rl, ul, &pl);
    primitives(ndim, qR, gamma, &rr, ur, &pr);
    if (!admissible(rl, pl) || !admissible(rr, pr)) return 0;
    double sl = fabs(ul[d]) + sqrt(gamma * pl / rl);
    double sr = fabs(ur[d]) + sqrt(gamma * pr / rr);
    double s = sl > sr ? sl : sr;
    double FL[MAXC], FR[MAXC];
    physical_flux(ndim, d, qL, gamma, FL);
    physical_flux(ndim, d, qR, gamma, FR);
    for (int m = 0; m < ncomp; m++) F[m] = 0.5 * (FL[m] + FR[m]) - 0.5 * s * (qR[m] - qL[m]);
    return 1;
}

/*
 * FORCE face flux (Toro's first-order centred scheme, the face flux the paper
 * uses in Section 7.3) for a time step dt over cells of width dx along axis d,
 * with dtdx = dt/dx: the mean of the Lax-Friedrichs flux
 *   F_LF = (F(qL) + F(qR))/2 - (qR - qL)/(2 dtdx)
 * and the Richtmyer flux F_RI = F(q_RI) of the intermediate state
 *   q_RI = (qL + qR)/2 - dtdx (F(qR) - F(qL))/2.
 * Returns 0 if qL or qR is not admissible (q_RI is an intermediate of the
 * formula and is not required to be).
 */
static int force_flux(int ndim, int d, const double* qL, const double* qR, double gamma, double dtdx,
                      double* F)
{
    int ncomp = ndim + 2;
    double rho, u[3], p;
    primitives(ndim, qL, gamma, &rho, u, &p);
    if (!admissible(rho, p)) return 0;
    primitives(ndim, qR, gamma, &rho, u, &p);
    if (!admissible(rho, p)) return 0;
    double FL[MAXC], FR[MAXC], qRI[MAXC], FRI[MAXC];
    physical_flux(ndim, d, qL, gamma, FL);
    physical_flux(ndim, d, qR, gamma, FR);
    for (int m = 0; m < ncomp; m++) qRI[m] = 0.5 * (qL[m] + qR[m]) - 0.5 * dtdx * (FR[m] - FL[m]);
    physical_flux(ndim, d, qRI, gamma, FRI);
    for (int m = 0; m < ncomp; m++) {
        double flf = 0.5 * (FL[m] + FR[m]) - 0.5 * (qR[m] - qL[m]) / dtdx;
        F[m] = 0.5 * (flf + FRI[m]);
    }
    return 1;
}

static double minmod(double a, double b)
{
    if (a * b <= 0.0) return 0.0;
    return fabs(a) < fabs(b) ? a : b;
}

/*
 * Face states of cell c along axis d: the values the cell presents at its
 * low face (qbL) and its high face (qbR).
 *  first order: both are the cell average;
 *  MUSCL-Hancock: slope D = minmod(U_c - U_{c-1}, U_{c+1} - U_c), boundary
 *  extrapolated values U_c -/+ D/2, each advanced half a step with the
 *  direction-d flux difference (dt/dx)(F(U^L) - F(U^R))/2.
 */
static int face_states(const grid_t* g, const double* U, int ncomp, int d, const int64_t* c,
                       double dtdx, int scheme, double gamma, double* qbL, double* qbR)
{
    double q[MAXC];
    load_cell(g, U, ncomp, c, q);
    if (scheme == SCHEME_RUSANOV1) {
        for (int m = 0; m < ncomp; m++) qbL[m] = qbR[m] = q[m];
        return 1;
    }
    int64_t cm[3] = {c[0], c[1], c[2]}, cp[3] = {c[0], c[1], c[2]};
    cm[d] -= 1;
    cp[d] += 1;
    double qm[MAXC], qp[MAXC], qL[MAXC], qR[MAXC];
    load_cell(g, U, ncomp, cm, qm);
    load_cell(g, U, ncomp, cp, qp);
    for (int m = 0; m < ncomp; m++) {
        double slope = minmod(q[m] - qm[m], qp[m] - q[m]);
        qL[m] = q[m] - 0.5 * slope;
        qR[m] = q[m] + 0.5 * slope;
    }
    int ndim = ncomp - 2;
    double rho, u[3], p;
    primitives(ndim, qL, gamma, &rho, u, &p);
    if (!admissible(rho, p)) return 0;
    primitives(ndim, qR, gamma, &rho, u, &p);
    if (!admissible(rho, p)) return 0;
    double FL[MAXC], FR[MAXC];
    physical_flux(ndim, d, qL, gamma, FL);
    physical_flux(ndim, d, qR, gamma, FR);
    for (int m = 0; m < ncomp; m++) {
        double half_step = 0.5 * dtdx * (FL[m] - FR[m]);
        qbL[m] = qL[m] + half_step;
        qbR[m] = qR[m] + half_step;
    }
    return 1;
}

/* Flux through the face between cell c and cell c + e_d. */
static int face_flux(const grid_t* g, const double* U, int ncomp, int d, const int64_t* c,
                     double dtdx, int scheme, double gamma, double* F)
{
    double lo_L[MAXC], lo_R[MAXC], hi_L[MAXC], hi_R[MAXC];
    int64_t cn[3] = {c[0], c[1], c[2]};
    cn[d] += 1;
    if (!face_states(g, U, ncomp, d, c, dtdx, scheme, gamma, lo_L, lo_R)) return 0;
    if (!face_states(g, U, ncomp, d, cn, dtdx, scheme, gamma, hi_L, hi_R)) return 0;
    /* left side of the face = high-face value of c; right = low-face value of c+e_d */
    return rusanov(ncomp - 2, d, lo_R, hi_L, gamma, F);
}

/* Max over interior cells of sum_d (|u_d| + c)/dx_d  (set_wavespeeds + MaxReducer). */
static int max_wavespeed(const grid_t* g, const double* U, int ncomp, double gamma,
                         const double* dx, double* smax)
{
    int ndim = ncomp - 2;
    double best = 0.0;
    int ok = 1;
    /* cells are independent and a maximum does not depend on the order in
       which it is taken, so the planes may be split over threads */
#pragma omp parallel for schedule(static) reduction(max : best) reduction(&& : ok)
    for (int64_t k = 0; k < g->n[2]; k++) {
        int64_t c[3] = {0, 0, k};
        for (c[1] = 0; c[1] < g->n[1]; c[1]++)
            for (c[0] = 0; c[0] < g->n[0]; c[0]++) {
                double q[MAXC], rho, u[3], p;
                load_cell(g, U, ncomp, c, q);
                primitives(ndim, q, gamma, &rho, u, &p);
                if (!admissible(rho, p)) {
                    ok = 0;
                    continue;
                }
                double cs = sqrt(gamma * p / rho);
                double s = 0.0;
                for (int d = 0; d < ndim; d++) s += (fabs(u[d]) + cs) / dx[d];
                if (s > best) best = s;
            }
    }
    if (!ok) return 0;
    *smax = best;
    return 1;
}

/*
 * New value of interior cell c:  U_c - dt * sum_d (F_{d,c+1/2} - F_{d,c-1/2}) / dx_d.
 * Both faces are evaluated with face_flux, so a face shared by two cells has
 * the same bits whichever cell asks for it.
 */
static int cell_update(const grid_t* g, const double* U, int ncomp, const int64_t* c, double dt,
                       const double* dx, int scheme, double gamma, double* qnew)
{
    double acc[MAXC] = {0, 0, 0, 0, 0};
    for (int d = 0; d < g->ndim; d++) {
        double Fp[MAXC], Fm[MAXC];
        int64_t cm[3] = {c[0], c[1], c[2]};
        cm[d] -= 1;
        if (!face_flux(g, U, ncomp, d, c, dt / dx[d], scheme, gamma, Fp)) return 0;
        if (!face_flux(g, U, ncomp, d, cm, dt / dx[d], scheme, gamma, Fm)) return 0;
        for (int m = 0; m < ncomp; m++) acc[m] += (Fp[m] - Fm[m]) / dx[d];
    }
    double q[MAXC];
    load_cell(g, U, ncomp, c, q);
    for (int m = 0; m < ncomp; m++) qnew[m] = q[m] - dt * acc[m];
    double rho, u[3], p;
    primitives(ncomp - 2, qnew, gamma, &rho, u, &p);
    return admissible(rho, p);
}

/*
 * One time step on a padded array, out of place (Section 5.4 double
 * buffering: in -> out, then swap).  Faces are computed once per face along
 * each grid line and differenced; the bits equal those of cell_update.
 */
static int euler_step(const grid_t* g, double* U, double* Unew, int ncomp, double gamma,
                      double cfl, const double* dx, int scheme, int bc, double* dt_out)
{
    double smax;
    if (!max_wavespeed(g, U, ncomp, gamma, dx, &smax)) return ORACLE_NUMERIC;
    double dt = cfl / smax;
    fill_padding(g, U, ncomp, bc);

    int64_t nint = g->n[0] * g->n[1] * g->n[2];
    double* acc = (double*)calloc((size_t)(nint * ncomp), sizeof(double));
    int64_t nmax = g->n[0];
    if (g->n[1] > nmax) nmax = g->n[1];
    if (g->n[2] > nmax) nmax = g->n[2];
    if (!acc) return ORACLE_OOM;
    int status = ORACLE_OK;
    for (int d = 0; d < g->ndim && status == ORACLE_OK; d++) {
        /* all grid lines along axis d; a line writes only its own cells of
           acc, so lines may run on different threads without changing a bit */
        int64_t ext[3] = {g->n[0], g->n[1], g->n[2]};
        ext[d] = 1;
        int64_t nlines = ext[0] * ext[1] * ext[2];
        int bad = 0, oom = 0;
#pragma omp parallel reduction(|| : bad, oom)
        {
            double* line = (double*)malloc(sizeof(double) * (size_t)((nmax + 1) * ncomp));
            if (!line) oom = 1;
#pragma omp for schedule(static)
            for (int64_t l = 0; l < nlines; l++) {
                if (!line || bad) continue;
                int64_t c[3] = {l % ext[0], (l / ext[0]) % ext[1], l / (ext[0] * ext[1])};
                /* faces between cells f-1 and f for f = 0..n_d; slot f */
                for (int64_t f = 0; f <= g->n[d]; f++) {
                    c[d] = f - 1;
                    if (!face_flux(g, U, ncomp, d, c, dt / dx[d], scheme, gamma, line + f * ncomp)) {
                        bad = 1;
                        break;
                    }
                }
                for (int64_t i = 0; i < g->n[d] && !bad; i++) {
                    c[d] = i;
                    int64_t lin = (c[2] * g->n[1] + c[1]) * g->n[0] + c[0];
                    for (int m = 0; m < ncomp; m++)
                        acc[m * nint + lin] += (line[(i + 1) * ncomp + m] - line[i * ncomp + m]) / dx[d];
                }
            }
            free(line);
        }
        if (oom) status = ORACLE_OOM;
        else if (bad) status = ORACLE_NUMERIC;
    }
    if (status == ORACLE_OK) {
        memcpy(Unew, U, sizeof(double) * (size_t)(g->ncell * ncomp));
#pragma omp parallel for schedule(static)
        for (int64_t k = 0; k < g->n[2]; k++) {
            int64_t c[3] = {0, 0, k};
            for (c[1] = 0; c[1] < g->n[1]; c[1]++)
                for (c[0] = 0; c[0] < g->n[0]; c[0]++) {
                    int64_t id = pidx(g, c);
                    int64_t lin = (c[2] * g->n[1] + c[1]) * g->n[0] + c[0];
                    for (int m = 0; m < ncomp; m++)
                        Unew[m * g->ncell + id] = U[m * g->ncell + id] - dt * acc[m * nint + lin];
                }
        }
    }
    free(acc);
    if (dt_out) *dt_out = dt;
    return status;
}

/*
 * One dimensionally split step, the paper's Euler solver (Listing euler_graph:
 * set_wavespeeds -> MaxReducer -> set_dt -> set_boundary -> update_state_x ->
 * set_boundary -> update_state_y [-> set_boundary -> update_state_z] ->
 * swap_in_out) with the FORCE face flux.  dt comes from the state at the start
 * of the step (the same rule as the unsplit step); each sweep fills the
 * padding of its input and applies the flux difference along its own axis:
 *   U^(d+1)_i = U^(d)_i - (dt/dx_d) (F_{i+1/2} - F_{i-1/2}).
 * Every updated cell must be admissible.  The result is written to Unew.
 */
static int euler_split_step(const grid_t* g, double* U, double* Unew, int ncomp, double gamma, double cfl,
                            const double* dx, int bc, double* dt_out)
{
    double smax;
    if (!max_wavespeed(g, U, ncomp, gamma, dx, &smax)) return ORACLE_NUMERIC;
    double dt = cfl / smax;
    if (dt_out) *dt_out = dt;
    int64_t nmax = g->n[0];
    if (g->n[1] > nmax) nmax = g->n[1];
    if (g->n[2] > nmax) nmax = g->n[2];
    double* src = U;
    double* dst = Unew;
    int status = ORACLE_OK;
    for (int d = 0; d < g->ndim && status == ORACLE_OK; d++) {
        fill_padding(g, src, ncomp, bc);
        memcpy(dst, src, sizeof(double) * (size_t)(g->ncell * ncomp));
        /* all grid lines along axis d; a line reads src and writes only its
           own cells of dst, so lines may run on different threads */
        int64_t ext[3] = {g->n[0], g->n[1], g->n[2]};
        ext[d] = 1;
        int64_t nlines = ext[0] * ext[1] * ext[2];
        int bad = 0, oom = 0;
#pragma omp parallel reduction(|| : bad, oom)
        {
            double* line = (double*)malloc(sizeof(double) * (size_t)((nmax + 1) * ncomp));
            if (!line) oom = 1;
#pragma omp for schedule(static)
            for (int64_t l = 0; l < nlines; l++) {
                if (!line || bad) continue;
                int64_t c[3] = {l % ext[0], (l / ext[0]) % ext[1], l / (ext[0] * ext[1])};
                /* faces between cells f-1 and f for f = 0..n_d; slot f */
                for (int64_t f = 0; f <= g->n[d] && !bad; f++) {
                    double qL[MAXC], qR[MAXC];
                    c[d] = f - 1;
                    load_cell(g, src, ncomp, c, qL);
                    c[d] = f;
                    load_cell(g, src, ncomp, c, qR);
                    if (!force_flux(ncomp - 2, d, qL, qR, gamma, dt / dx[d], line + f * ncomp)) bad = 1;
                }
                for (int64_t i = 0; i < g->n[d] && !bad; i++) {
                    c[d] = i;
                    int64_t id = pidx(g, c);
                    double q[MAXC], rho, u[3], p;
                    for (int m = 0; m < ncomp; m++) {
                        q[m] = src[m * g->ncell + id] -
                               dt / dx[d] * (line[(i + 1) * ncomp + m] - line[i * ncomp + m]);
                        dst[m * g->ncell + id] = q[m];
                    }
                    primitives(ncomp - 2, q, gamma, &rho, u, &p);
                    if (!admissible(rho, p)) bad = 1;
                }
            }
            free(line);
        }
        if (oom) status = ORACLE_OOM;
        else if (bad) status = ORACLE_NUMERIC;
        double* tmp = src;
        src = dst;
        dst = tmp;
    }
    if (status == ORACLE_OK && src != Unew) memcpy(Unew, src, sizeof(double) * (size_t)(g->ncell * ncomp));
    return status;
}

static int check_euler_args(int ndim, int ncomp, int scheme, int bc)
{
    if (ndim < 2 || ndim > 3 || ncomp != ndim + 2) return 0;
    if (scheme != SCHEME_RUSANOV1 && scheme != SCHEME_MUSCL_HANCOCK && scheme != SCHEME_FORCE_SPLIT) return 0;
    if (bc != BC_PERIODIC && bc != BC_TRANSMISSIVE) return 0;
    return 1;
}

/* Threads used by the Euler steps (1 unless set; 1 if built without OpenMP). */
static int g_threads = 1;

int oracle_set_threads(int n)
{
#ifdef _OPENMP
    g_threads = n < 1 ? 1 : n;
#else
    (void)n;
    g_threads = 1;
#endif
    return g_threads;
}

int oracle_threads(void) { return g_threads; }

/*
 * Run nsteps steps in place on an interior-only component-major array.
 * Returns ORACLE_NUMERIC (and leaves U at the last admissible state) if a
 * state loses positivity.  t_out = sum of dt; dt_last = the last dt used.
 */
int oracle_euler_run(int ndim, const int64_t* n, double* U, double gamma, double cfl,
                     const double* dx, int scheme, int bc, int64_t nsteps, double* t_out,
                     double* dt_last, int64_t* steps_done)
{
    int ncomp = ndim + 2;
    if (!check_euler_args(ndim, ncomp, scheme, bc) || nsteps < 0) return ORACLE_INVALID;
    grid_t g;
    int h = scheme == SCHEME_MUSCL_HANCOCK ? 2 : 1;
    if (grid_init(&g, ndim, n, h) != ORACLE_OK) return ORACLE_INVALID;
    if (bc == BC_PERIODIC)
        for (int d = 0; d < ndim; d++)
            if (g.n[d] < h) return ORACLE_INVALID;
    size_t bytes = sizeof(double) * (size_t)(g.ncell * ncomp);
    double* A = (double*)malloc(bytes);
    double* B = (double*)malloc(bytes);
    if (!A || !B) {
        free(A);
        free(B);
        return ORACLE_OOM;
    }
    to_padded(&g, ncomp, U, A);
#ifdef _OPENMP
    omp_set_num_threads(g_threads);
#endif
    double t = 0.0, dt = 0.0;
    int status = ORACLE_OK;
    int64_t s = 0;
    for (; s < nsteps; s++) {
        status = scheme == SCHEME_FORCE_SPLIT ? euler_split_step(&g, A, B, ncomp, gamma, cfl, dx, bc, &dt)
                                              : euler_step(&g, A, B, ncomp, gamma, cfl, dx, scheme, bc, &dt);
        if (status != ORACLE_OK) break;
        t += dt;
        double* tmp = A; /* swap_in_out */
        A = B;
        B = tmp;
    }
    from_padded(&g, ncomp, A, U);
    free(A);
    free(B);
    if (t_out) *t_out = t;
    if (dt_last) *dt_last = dt;
    if (steps_done) *steps_done = s;
    return status;
}

/* dt = CFL / max wave-speed sum of an interior array (0 on a non-admissible state). */
int oracle_euler_dt(int ndim, const int64_t* n, const double* U, double gamma, double cfl,
                    const double* dx, double* dt_out)
{
    int ncomp = ndim + 2;
    grid_t g;
    if (grid_init(&g, ndim, n, 0) != ORACLE_OK) return ORACLE_INVALID;
    double smax;
    if (!max_wavespeed(&g, U, ncomp, gamma, dx, &smax)) return ORACLE_NUMERIC;
    *dt_out = cfl / smax;
    return ORACLE_OK;
}

/*
 * One step evaluated only at selected interior cells (linear interior
 * indices), from a full interior state U.  dt <= 0 means "compute dt from U".
 * out[s * ncomp + m] = new value of component m at cells[s].
 */
int oracle_euler_step_cells(int ndim, const int64_t* n, const double* U, double gamma, double cfl,
                            const double* dx, int scheme, int bc, double dt, int64_t ncells,
                            const int64_t* cells, double* out, double* dt_out)
{
    int ncomp = ndim + 2;
    /* a split step's value at a cell needs the whole first sweep: full runs only */
    if (!check_euler_args(ndim, ncomp, scheme, bc) || scheme == SCHEME_FORCE_SPLIT) return ORACLE_INVALID;
    grid_t g;
    int h = scheme == SCHEME_RUSANOV1 ? 1 : 2;
    if (grid_init(&g, ndim, n, h) != ORACLE_OK) return ORACLE_INVALID;
    double* A = (double*)malloc(sizeof(double) * (size_t)(g.ncell * ncomp));
    if (!A) return ORACLE_OOM;
    to_padded(&g, ncomp, U, A);
    if (dt <= 0.0) {
        double smax;
        if (!max_wavespeed(&g, A, ncomp, gamma, dx, &smax)) {
            free(A);
            return ORACLE_NUMERIC;
        }
        dt = cfl / smax;
    }
    fill_padding(&g, A, ncomp, bc);
    int status = ORACLE_OK;
    for (int64_t s = 0; s < ncells; s++) {
        int64_t lin = cells[s];
        int64_t c[3];
        c[0] = lin % g.n[0];
        c[1] = (lin / g.n[0]) % g.n[1];
        c[2] = lin / (g.n[0] * g.n[1]);
        if (c[2] >= g.n[2] || lin < 0) {
            status = ORACLE_INVALID;
            break;
        }
        if (!cell_update(&g, A, ncomp, c, dt, dx, scheme, gamma, out + s * ncomp))
            status = ORACLE_NUMERIC;
    }
    free(A);
    if (dt_out) *dt_out = dt;
    return status;
}

/* ------------------------------------------------------------------------ */
/* Eikonal: Godunov upwind local solver and Fast Marching.                   */
/* ------------------------------------------------------------------------ */

/*
 * Godunov upwind update of one cell.  a[d] = smaller of the two neighbour
 * values along axis d (+inf when unknown / outside), f = s*h.
 * 2D: |a-b| >= f -> min(a,b) + f, else (a + b + sqrt(2 f^2 - (a-b)^2)) / 2.
 * 3D: sort a1 <= a2 <= a3 and add terms while the candidate exceeds the next
 * a: the m-term candidate solves sum_{i<=m} (T - a_i)^2 = f^2.
 */
double oracle_godunov(int ndim, const double* a_in, double f)
{
    double a[3];
    for (int d = 0; d < ndim; d++) a[d] = a_in[d];
    if (ndim == 2) {
        double x = a[0], y = a[1];
        double lo = x < y ? x : y;
        if (!(fabs(x - y) < f)) return lo + f; /* also both +inf */
        return 0.5 * (x + y + sqrt(2.0 * f * f - (x - y) * (x - y)));
    }
    /* insertion sort, ascending */
    for (int i = 1; i < 3; i++)
        for (int j = i; j > 0 && a[j] < a[j - 1]; j--) {
            double t = a[j];
            a[j] = a[j - 1];
            a[j - 1] = t;
        }
    double T = a[0] + f;
    if (!(T > a[1])) return T;
    /* two terms */
    T = 0.5 * (a[0] + a[1] + sqrt(2.0 * f * f - (a[0] - a[1]) * (a[0] - a[1])));
    if (!(T > a[2])) return T;
    /* three terms: 3T^2 - 2 S T + (Q - f^2) = 0 */
    double S = a[0] + a[1] + a[2];
    double Q = a[0] * a[0] + a[1] * a[1] + a[2] * a[2];
    double disc = S * S - 3.0 * (Q - f * f);
    if (disc < 0.0) disc = 0.0; /* rounding guard: exact arithmetic gives disc > 0 here */
    return (S + sqrt(disc)) / 3.0;
}

typedef struct {
    double key;
    int64_t idx;
} heap_item;

typedef struct {
    heap_item* v;
    int64_t size, cap;
} heap_t;

static int heap_push(heap_t* hp, double key, int64_t idx)
{
    if (hp->size == hp->cap) {
        int64_t cap = hp->cap ? 2 * hp->cap : 1024;
        heap_item* nv = (heap_item*)realloc(hp->v, sizeof(heap_item) * (size_t)cap);
        if (!nv) return 0;
        hp->v = nv;
        hp->cap = cap;
    }
    int64_t i = hp->size++;
    hp->v[i].key = key;
    hp->v[i].idx = idx;
    while (i > 0) {
        int64_t parent = (i - 1) / 2;
        if (!(hp->v[i].key < hp->v[parent].key)) break;
        heap_item t = hp->v[i];
        hp->v[i] = hp->v[parent];
        hp->v[parent] = t;
        i = parent;
    }
    return 1;
}

static heap_item heap_pop(heap_t* hp)
{
    heap_item top = hp->v[0];
    hp->v[0] = hp->v[--hp->size];
    int64_t i = 0;
    for (;;) {
        int64_t l = 2 * i + 1, r = l + 1, m = i;
        if (l < hp->size && hp->v[l].key < hp->v[m].key) m = l;
        if (r < hp->size && hp->v[r].key < hp->v[m].key) m = r;
        if (m == i) break;
        heap_item t = hp->v[i];
        hp->v[i] = hp->v[m];
        hp->v[m] = t;
        i = m;
    }
    return top;
}

/*
 * Fast Marching.  s: slowness per cell (interior array, x fastest), h: grid
 * spacing, src: linear cell indices held at T = 0.  T receives the travel
 * time of every cell (+inf if unreachable).
 */
int oracle_eikonal_fmm(int ndim, const int64_t* n, const double* s, double h, int nsrc,
                       const int64_t* src, double* T)
{
    if (ndim < 2 || ndim > 3 || nsrc < 1) return ORACLE_INVALID;
    int64_t N[3] = {1, 1, 1}, total = 1;
    for (int d = 0; d < ndim; d++) {
        N[d] = n[d];
        if (N[d] < 1) return ORACLE_INVALID;
        total *= N[d];
    }
    int64_t stride[3] = {1, N[0], N[0] * N[1]};
    unsigned char* known = (unsigned char*)calloc((size_t)total, 1);
    unsigned char* fixed = (unsigned char*)calloc((size_t)total, 1);
    heap_t hp = {0, 0, 0};
    if (!known || !fixed) {
        free(known);
        free(fixed);
        return ORACLE_OOM;
    }
    for (int64_t i = 0; i < total; i++) T[i] = INFINITY;
    int status = ORACLE_OK;
    for (int k = 0; k < nsrc; k++) {
        if (src[k] < 0 || src[k] >= total) {
            status = ORACLE_INVALID;
            goto done;
        }
        T[src[k]] = 0.0;
        fixed[src[k]] = 1;
        if (!heap_push(&hp, 0.0, src[k])) {
            status = ORACLE_OOM;
            goto done;
        }
    }
    while (hp.size > 0) {
        heap_item it = heap_pop(&hp);
        if (known[it.idx]) continue;       /* stale entry */
        if (it.key != T[it.idx]) continue; /* superseded by a smaller value */
        known[it.idx] = 1;
        int64_t c[3] = {it.idx % N[0], (it.idx / N[0]) % N[1], it.idx / (N[0] * N[1])};
        for (int d = 0; d < ndim; d++)
            for (int side = -1; side <= 1; side += 2) {
                int64_t cd = c[d] + side;
                if (cd < 0 || cd >= N[d]) continue;
                int64_t nb = it.idx + side * stride[d];
                if (known[nb] || fixed[nb]) continue;
                /* Godunov value of nb from its known neighbours */
                int64_t cn[3] = {c[0], c[1], c[2]};
                cn[d] = cd;
                double a[3];
                for (int e = 0; e < ndim; e++) {
                    a[e] = INFINITY;
                    for (int s2 = -1; s2 <= 1; s2 += 2) {
                        int64_t ce = cn[e] + s2;
                        if (ce < 0 || ce >= N[e]) continue;
                        int64_t m = nb + s2 * stride[e];
                        if (known[m] && T[m] < a[e]) a[e] = T[m];
                    }
                }
                double val = oracle_godunov(ndim, a, s[nb] * h);
                if (val < T[nb]) {
                    T[nb] = val;
                    if (!heap_push(&hp, val, nb)) {
                        status = ORACLE_OOM;
                        goto done;
                    }
                }
            }
    }
done:
    free(known);
    free(fixed);
    free(hp.v);
    return status;
}
