/*
 * oklb.c -- plain FP64 CPU oracle of the finite-difference lattice Boltzmann
 * (FDLB) time step of Gan, Xu, Zhang & Li, "Lattice Boltzmann study on
 * Kelvin-Helmholtz instability: the roles of velocity and density gradients"
 * (arXiv:1010.4124).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this library.  It shares no code,
 * header, table or helper with the CUDA path; it is written as loops over
 * nodes and velocities, in the order in which the paper states the method,
 * with no tiling, fusion or reordering.
 *
 * Compiled twice from this one source:
 *   liboklb.so     real = double
 *   liboklb_cs.so  real = double _Complex  (-DOKLB_COMPLEX): the same step run
 *                  on complex numbers gives exact forward-mode derivatives by
 *                  the complex-step method (Im f(x+ih)/h), used as the tangent
 *                  of the step for the adjoint's dot-product test.  Every
 *                  operation of the step is analytic (the upwind side depends
 *                  only on the sign of a constant velocity component), so the
 *                  complex-step derivative is exact up to rounding.
 *
 * Build: gcc -O2 -fPIC -shared -fopenmp -ffp-contract=off (see build.py).
 *
 * Layout of a distribution array handed to this library: f[q][j][i],
 * q = 0..18 velocity, j = 0..ny-1 row (y), i = 0..nx-1 column (x, fastest).
 * Only interior nodes are passed; ghost nodes are rebuilt inside each step.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include <stdint.h>

#ifdef OKLB_COMPLEX
#include <complex.h>
typedef double _Complex real;
#define RE(x) creal(x)
#else
typedef double real;
#define RE(x) (x)
#endif

#define NQ 19
#define NG 3 /* ghost layers per side: indices -2,-1,0 and Nx+1..Nx+3 (Sec. III.B) */

enum { OKLB_PERIODIC = 0, OKLB_OUTFLOW = 1, OKLB_FIXED_EQ = 2 };

typedef struct {
    int32_t nx, ny;
    double dx, dy, dt, tau;
    double v[3];
    int32_t bc_x_lo, bc_x_hi, bc_y_lo, bc_y_hi;
    double eps; /* WENO epsilon; the paper's value is 1e-6 (Eq. 52) */
    int32_t scheme; /* convection scheme: 0 WENO5 (Sec. III.A), 1 first-order upwind,
                       2 second-order upwind, 3 second-order TVD (minmod); Sec. III.B, Fig. 2 */
} oklb_params;

/* ------------------------------------------------------------------------ */
/* Discrete velocity model, Sec. II.A, Eq. (5) with N = 6:                  */
/* v_0 = 0, v_ki = v_k (cos(2 pi i/6), sin(2 pi i/6)), i = 1..6, k = 1..3.   */
/* Index q = 0 is the rest velocity; q = 1 + 6(k-1) + (i-1).                 */
/* The cosines and sines of multiples of 60 degrees are written as exact     */
/* constants (+-1, +-1/2, +-sqrt(3)/2) instead of calls to cos/sin.          */
/* ------------------------------------------------------------------------ */
void oklb_velocity_set(const double v[3], double vx[NQ], double vy[NQ])
{
    const double h = 0.5 * sqrt(3.0);
    /* i = 1..6 -> angles 60, 120, 180, 240, 300, 360 degrees */
    const double c[6] = {0.5, -0.5, -1.0, -0.5, 0.5, 1.0};
    const double s[6] = {h, h, 0.0, -h, -h, 0.0};
    vx[0] = 0.0;
    vy[0] = 0.0;
    for (int k = 0; k < 3; ++k)
        for (int i = 0; i < 6; ++i) {
            vx[1 + 6 * k + i] = v[k] * c[i];
            vy[1 + 6 * k + i] = v[k] * s[i];
        }
}

/* ring index k (0 = rest, 1..3) of velocity q */
static int ring_of(int q) { return q == 0 ? 0 : 1 + (q - 1) / 6; }

/* ------------------------------------------------------------------------ */
/* Global coefficients F_k(T), Sec. II.C, Eqs. (44)-(46): the solution of    */
/* the four requirements (FK-11)-(FK-14) with v_0 = 0 and three rings,       */
/*   F_k = [24T^3 - 4(v_{k+1}^2 + v_{k+2}^2) T^2 + v_{k+1}^2 v_{k+2}^2 T]     */
/*         / [3 v_k^2 (v_k^2 - v_{k+1}^2)(v_k^2 - v_{k+2}^2)],               */
/*   F_0 = 1 - 6 (F_1 + F_2 + F_3),  ring index k+l taken cyclically in 1..3. */
/* ------------------------------------------------------------------------ */
static void Fk_of_T(real T, const double v[3], real F[4])
{
    for (int k = 1; k <= 3; ++k) {
        int k1 = k + 1 > 3 ? k + 1 - 3 : k + 1;
        int k2 = k + 2 > 3 ? k + 2 - 3 : k + 2;
        double ak = v[k - 1] * v[k - 1];
        double a1 = v[k1 - 1] * v[k1 - 1];
        double a2 = v[k2 - 1] * v[k2 - 1];
        real num = 24.0 * T * T * T - 4.0 * (a1 + a2) * T * T + a1 * a2 * T;
        double den = 3.0 * ak * (ak - a1) * (ak - a2);
        F[k] = num / den;
    }
    F[0] = 1.0 - 6.0 * (F[1] + F[2] + F[3]);
}

void oklb_Fk(const real* T, const double v[3], real F[4]) { Fk_of_T(*T, v, F); }

/* ------------------------------------------------------------------------ */
/* Truncated equilibrium, Sec. II.C, Eq. (28):                               */
/*   f_ki^(0) = rho F_k [ (1 - u^2/2T) + (v.u/T)(1 - u^2/2T)                 */
/*                        + (v.u)^2/(2T^2) + (v.u)^3/(6T^3) ].               */
/* ------------------------------------------------------------------------ */
static void feq_of(real rho, real ux, real uy, real T, const double v[3],
                   const double vx[NQ], const double vy[NQ], real out[NQ])
{
    real F[4];
    Fk_of_T(T, v, F);
    real u2 = ux * ux + uy * uy;
    real A = 1.0 - u2 / (2.0 * T);
    for (int q = 0; q < NQ; ++q) {
        real vu = vx[q] * ux + vy[q] * uy;
        real bracket = A + (vu / T) * A + (vu * vu) / (2.0 * T * T)
                     + (vu * vu * vu) / (6.0 * T * T * T);
        out[q] = rho * F[ring_of(q)] * bracket;
    }
}

void oklb_feq(const real* rho, const real* ux, const real* uy, const real* T,
              const double v[3], real out[NQ])
{
    double vx[NQ], vy[NQ];
    oklb_velocity_set(v, vx, vy);
    feq_of(*rho, *ux, *uy, *T, v, vx, vy, out);
}

/* ------------------------------------------------------------------------ */
/* Macroscopic moments, Sec. II.B, Eq. (10):                                 */
/*   rho = sum f,  rho u = sum f v,  rho T = sum f (v - u)^2 / 2.            */
/* (Eq. (10) is stated for f^(0); the step conserves these moments, so they  */
/* are taken from f.)                                                         */
/* ------------------------------------------------------------------------ */
static void moments_of(const real f[NQ], const double vx[NQ], const double vy[NQ],
                       real* rho, real* ux, real* uy, real* T)
{
    real r = 0.0, jx = 0.0, jy = 0.0;
    for (int q = 0; q < NQ; ++q) {
        r += f[q];
        jx += f[q] * vx[q];
        jy += f[q] * vy[q];
    }
    real u = jx / r, w = jy / r;
    real e = 0.0;
    for (int q = 0; q < NQ; ++q) {
        real cx = vx[q] - u, cy = vy[q] - w;
        e += f[q] * (cx * cx + cy * cy) / 2.0;
    }
    *rho = r;
    *ux = u;
    *uy = w;
    *T = e / r;
}

void oklb_moments(const real f[NQ], const double v[3], real* rho, real* ux, real* uy, real* T)
{
    double vx[NQ], vy[NQ];
    oklb_velocity_set(v, vx, vy);
    moments_of(f, vx, vy, rho, ux, uy, T);
}

/* ------------------------------------------------------------------------ */
/* Fifth-order WENO numerical flux h_{I+1/2}, Sec. III.A, Eqs. (48)-(55)     */
/* (Jiang & Shu), for a non-negative velocity component:                     */
/*   a..e = F_{I-2}, F_{I-1}, F_I, F_{I+1}, F_{I+2}, with F = v_alpha f.     */
/* For a negative component the caller passes the mirror stencil             */
/*   a..e = F_{I+3}, F_{I+2}, F_{I+1}, F_I, F_{I-1}  (Sec. III.A, last par.). */
/* ------------------------------------------------------------------------ */
static real weno5(real a, real b, real c, real d, real e, double eps)
{
    /* candidate fluxes, Eqs. (49)-(51) */
    real h1 = (1.0 / 3.0) * a - (7.0 / 6.0) * b + (11.0 / 6.0) * c;
    real h2 = -(1.0 / 6.0) * b + (5.0 / 6.0) * c + (1.0 / 3.0) * d;
    real h3 = (1.0 / 3.0) * c + (5.0 / 6.0) * d - (1.0 / 6.0) * e;
    /* smoothness indicators, Eqs. (53)-(55) */
    real t1 = a - 2.0 * b + c, r1 = a - 4.0 * b + 3.0 * c;
    real t2 = b - 2.0 * c + d, r2 = b - d;
    real t3 = c - 2.0 * d + e, r3 = 3.0 * c - 4.0 * d + e;
    real s1 = (13.0 / 12.0) * t1 * t1 + 0.25 * r1 * r1;
    real s2 = (13.0 / 12.0) * t2 * t2 + 0.25 * r2 * r2;
    real s3 = (13.0 / 12.0) * t3 * t3 + 0.25 * r3 * r3;
    /* nonlinear weights, Eq. (52), optimal weights 1/10, 3/5, 3/10 */
    real w1 = 0.1 / ((eps + s1) * (eps + s1));
    real w2 = 0.6 / ((eps + s2) * (eps + s2));
    real w3 = 0.3 / ((eps + s3) * (eps + s3));
    real ws = w1 + w2 + w3;
    /* convex combination, Eq. (48) */
    return (w1 / ws) * h1 + (w2 / ws) * h2 + (w3 / ws) * h3;
}

/* exported for unit tests: F[0..4] = the five stencil values, in the order
 * weno5 takes them (already mirrored by the caller for negative velocity). */
void oklb_weno5_face(const real F[5], double eps, real* h)
{
    *h = weno5(F[0], F[1], F[2], F[3], F[4], eps);
}

/* ------------------------------------------------------------------------ */
/* The lower-order convection schemes the paper compares with WENO5 near the  */
/* Sod shock (Sec. III.B, Fig. 2).  The paper names them and gives no         */
/* formulas; these are the textbook forms, on the same upwind-ordered stencil */
/* as weno5 (c = F_I the upwind node, b = F_{I-1}, d = F_{I+1}):              */
/*   first-order upwind   h = F_I                                             */
/*   second-order upwind  h = F_I + (F_I - F_{I-1}) / 2                       */
/*   second-order TVD     h = F_I + minmod(F_I - F_{I-1}, F_{I+1} - F_I) / 2  */
/* The TVD form is the minmod-limited (NND-type) scheme of the paper's        */
/* reference for it.  For a negative velocity the mirrored stencil gives the  */
/* upwind node I+1 and the differences towards I+2 and I, as for weno5.       */
/* ------------------------------------------------------------------------ */
static real minmod(real x, real y)
{
    /* the argument of smaller magnitude when both have the same sign, else 0
       (decided on the real parts: the complex-step build differentiates the
       branch that is taken) */
    if (RE(x) > 0.0 && RE(y) > 0.0) return RE(x) < RE(y) ? x : y;
    if (RE(x) < 0.0 && RE(y) < 0.0) return RE(x) > RE(y) ? x : y;
    return 0.0;
}

static real face_flux(int scheme, real a, real b, real c, real d, real e, double eps)
{
    switch (scheme) {
    case 1: return c;
    case 2: return c + 0.5 * (c - b);
    case 3: return c + 0.5 * minmod(c - b, d - c);
    default: return weno5(a, b, c, d, e, eps);
    }
}

/* exported for unit tests: the face flux of `scheme` (same stencil order) */
void oklb_face_flux(int32_t scheme, const real F[5], double eps, real* h)
{
    *h = face_flux(scheme, F[0], F[1], F[2], F[3], F[4], eps);
}

/* ------------------------------------------------------------------------ */
/* Ghost nodes.  Three ghost layers per side (Sec. III.B, Eq. (57)).          */
/*  periodic  : wrap-around (Sec. III.B and Sec. IV.A, y direction).          */
/*  outflow   : zeroth-order extrapolation, Eqs. (63)-(64): every ghost node */
/*              carries the macroscopic state of the edge interior node; with */
/*              the non-equilibrium part also extrapolated at zeroth order    */
/*              (Sec. III.B, paragraph after Eq. (58)) the ghost f equals the */
/*              edge node's f.                                                */
/*  fixed_eq  : Eq. (57): f_ghost = f^(0) of the edge node at t = 0, supplied */
/*              in the fixed-ghost array (see oklb_fixed_ghosts).             */
/* Padded array layout: P[q][j+NG][i+NG], j in [-NG, ny+NG), i in [-NG, nx+NG). */
/* Corner ghosts are never read by the dimension-by-dimension stencils; they  */
/* are set to NaN so that any stray read poisons the result.                  */
/* ------------------------------------------------------------------------ */
static void fill_padded(const oklb_params* p, const real* f, const real* fixed, real* P)
{
    const int nx = p->nx, ny = p->ny;
    const int PX = nx + 2 * NG, PY = ny + 2 * NG;
    const real nanv = NAN;
    for (int q = 0; q < NQ; ++q) {
        real* Pq = P + (size_t)q * PY * PX;
        const real* fq = f + (size_t)q * ny * nx;
        for (int j = -NG; j < ny + NG; ++j)
            for (int i = -NG; i < nx + NG; ++i) {
                int inx = (i >= 0 && i < nx), iny = (j >= 0 && j < ny);
                real val = nanv;
                if (inx && iny) {
                    val = fq[(size_t)j * nx + i];
                } else if (iny) { /* x ghost of an interior row */
                    int bc = i < 0 ? p->bc_x_lo : p->bc_x_hi;
                    if (bc == OKLB_PERIODIC) {
                        int ii = ((i % nx) + nx) % nx;
                        val = fq[(size_t)j * nx + ii];
                    } else if (bc == OKLB_OUTFLOW) {
                        int ii = i < 0 ? 0 : nx - 1;
                        val = fq[(size_t)j * nx + ii];
                    } else { /* fixed: xlo block [19][ny], then xhi block */
                        size_t off = (i < 0 ? 0 : (size_t)NQ * ny) + (size_t)q * ny + j;
                        val = fixed[off];
                    }
                } else if (inx) { /* y ghost of an interior column */
                    int bc = j < 0 ? p->bc_y_lo : p->bc_y_hi;
                    if (bc == OKLB_PERIODIC) {
                        int jj = ((j % ny) + ny) % ny;
                        val = fq[(size_t)jj * nx + i];
                    } else if (bc == OKLB_OUTFLOW) {
                        int jj = j < 0 ? 0 : ny - 1;
                        val = fq[(size_t)jj * nx + i];
                    } else { /* ylo block [19][nx] after the two x blocks */
                        size_t off = (size_t)2 * NQ * ny + (j < 0 ? 0 : (size_t)NQ * nx)
                                   + (size_t)q * nx + i;
                        val = fixed[off];
                    }
                }
                Pq[(size_t)(j + NG) * PX + (i + NG)] = val;
            }
    }
}

/* Fixed-equilibrium ghost values from the initial macroscopic fields
 * (Eq. (57)): for each boundary row/column, f^(0) of the edge node's state.
 * Layout of `fixed`: xlo[19][ny], xhi[19][ny], ylo[19][nx], yhi[19][nx]. */
void oklb_fixed_ghosts(const oklb_params* p, const real* rho, const real* ux,
                       const real* uy, const real* T, real* fixed)
{
    const int nx = p->nx, ny = p->ny;
    double vx[NQ], vy[NQ];
    oklb_velocity_set(p->v, vx, vy);
    real fe[NQ];
    for (int side = 0; side < 2; ++side)
        for (int j = 0; j < ny; ++j) {
            size_t n = (size_t)j * nx + (side == 0 ? 0 : nx - 1);
            feq_of(rho[n], ux[n], uy[n], T[n], p->v, vx, vy, fe);
            for (int q = 0; q < NQ; ++q)
                fixed[(size_t)side * NQ * ny + (size_t)q * ny + j] = fe[q];
        }
    for (int side = 0; side < 2; ++side)
        for (int i = 0; i < nx; ++i) {
            size_t n = (size_t)(side == 0 ? 0 : ny - 1) * nx + i;
            feq_of(rho[n], ux[n], uy[n], T[n], p->v, vx, vy, fe);
            for (int q = 0; q < NQ; ++q)
                fixed[(size_t)2 * NQ * ny + (size_t)side * NQ * nx + (size_t)q * nx + i] = fe[q];
        }
}

/* f := f^(0)(rho, u, T) at every node (initial state of every run). */
void oklb_init_feq(const oklb_params* p, const real* rho, const real* ux,
                   const real* uy, const real* T, real* f)
{
    const size_t n = (size_t)p->nx * p->ny;
    double vx[NQ], vy[NQ];
    oklb_velocity_set(p->v, vx, vy);
#pragma omp parallel for schedule(static)
    for (size_t k = 0; k < n; ++k) {
        real fe[NQ];
        feq_of(rho[k], ux[k], uy[k], T[k], p->v, vx, vy, fe);
        for (int q = 0; q < NQ; ++q) f[(size_t)q * n + k] = fe[q];
    }
}

/* Macroscopic fields of a whole distribution array. */
void oklb_fields(const oklb_params* p, const real* f, real* rho, real* ux, real* uy, real* T)
{
    const size_t n = (size_t)p->nx * p->ny;
    double vx[NQ], vy[NQ];
    oklb_velocity_set(p->v, vx, vy);
#pragma omp parallel for schedule(static)
    for (size_t k = 0; k < n; ++k) {
        real fl[NQ];
        for (int q = 0; q < NQ; ++q) fl[q] = f[(size_t)q * n + k];
        moments_of(fl, vx, vy, &rho[k], &ux[k], &uy[k], &T[k]);
    }
}

/* ------------------------------------------------------------------------ */
/* One time step, Sec. III.A, Eq. (47):                                      */
/*   f^{n+1} = f^n - dt sum_alpha (h_{I+1/2} - h_{I-1/2}) / dr_alpha          */
/*                 - (dt/tau) (f^n - f^{n,(0)}),                              */
/* forward Euler in time, the alpha sum over x and y, h from weno5 (or the    */
/* scheme chosen in p->scheme) applied to F = v_alpha f with the upwind side  */
/* given by the sign of v_alpha.  A zero velocity component carries no flux   */
/* and is skipped.                                                             */
/* Steps in order: ghost fill; moments -> F_k(T) -> f^(0) per node; WENO face  */
/* fluxes in x and y; the update.                                              */
/* ------------------------------------------------------------------------ */
void oklb_step(const oklb_params* p, const real* f, const real* fixed, real* fout)
{
    const int nx = p->nx, ny = p->ny;
    const int PX = nx + 2 * NG, PY = ny + 2 * NG;
    const size_t n = (size_t)nx * ny;
    double vx[NQ], vy[NQ];
    oklb_velocity_set(p->v, vx, vy);

    real* P = (real*)malloc(sizeof(real) * NQ * PY * PX);
    real* feq = (real*)malloc(sizeof(real) * NQ * n);
    real* hx = (real*)malloc(sizeof(real) * NQ * ny * (nx + 1)); /* face i: between nodes i-1 and i */
    real* hy = (real*)malloc(sizeof(real) * NQ * (ny + 1) * nx); /* face j: between rows j-1 and j */
    fill_padded(p, f, fixed, P);

#define PAD(q, j, i) P[(size_t)(q) * PY * PX + (size_t)((j) + NG) * PX + (size_t)((i) + NG)]

    /* moments -> F_k(T) -> equilibrium at every interior node */
#pragma omp parallel for schedule(static)
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            real fl[NQ], fe[NQ], rho, ux, uy, T;
            for (int q = 0; q < NQ; ++q) fl[q] = PAD(q, j, i);
            moments_of(fl, vx, vy, &rho, &ux, &uy, &T);
            feq_of(rho, ux, uy, T, p->v, vx, vy, fe);
            for (int q = 0; q < NQ; ++q) feq[(size_t)q * n + (size_t)j * nx + i] = fe[q];
        }

    /* x-direction face fluxes */
#pragma omp parallel for schedule(static)
    for (int j = 0; j < ny; ++j)
        for (int q = 0; q < NQ; ++q) {
            const double c = vx[q];
            for (int i = 0; i <= nx; ++i) {
                real h = 0.0;
                if (c > 0.0) { /* face between I = i-1 and i; stencil I-2..I+2 */
                    h = face_flux(p->scheme, c * PAD(q, j, i - 3), c * PAD(q, j, i - 2), c * PAD(q, j, i - 1),
                              c * PAD(q, j, i), c * PAD(q, j, i + 1), p->eps);
                } else if (c < 0.0) { /* mirror stencil I+3..I-1 */
                    h = face_flux(p->scheme, c * PAD(q, j, i + 2), c * PAD(q, j, i + 1), c * PAD(q, j, i),
                              c * PAD(q, j, i - 1), c * PAD(q, j, i - 2), p->eps);
                }
                hx[(size_t)q * ny * (nx + 1) + (size_t)j * (nx + 1) + i] = h;
            }
        }

    /* y-direction face fluxes */
#pragma omp parallel for schedule(static)
    for (int j = 0; j <= ny; ++j)
        for (int q = 0; q < NQ; ++q) {
            const double c = vy[q];
            for (int i = 0; i < nx; ++i) {
                real h = 0.0;
                if (c > 0.0) {
                    h = face_flux(p->scheme, c * PAD(q, j - 3, i), c * PAD(q, j - 2, i), c * PAD(q, j - 1, i),
                              c * PAD(q, j, i), c * PAD(q, j + 1, i), p->eps);
                } else if (c < 0.0) {
                    h = face_flux(p->scheme, c * PAD(q, j + 2, i), c * PAD(q, j + 1, i), c * PAD(q, j, i),
                              c * PAD(q, j - 1, i), c * PAD(q, j - 2, i), p->eps);
                }
                hy[(size_t)q * (ny + 1) * nx + (size_t)j * nx + i] = h;
            }
        }

    /* forward-Euler update with BGK relaxation */
#pragma omp parallel for schedule(static)
    for (int j = 0; j < ny; ++j)
        for (int q = 0; q < NQ; ++q)
            for (int i = 0; i < nx; ++i) {
                size_t k = (size_t)q * n + (size_t)j * nx + i;
                real fo = PAD(q, j, i);
                real dhx = hx[(size_t)q * ny * (nx + 1) + (size_t)j * (nx + 1) + i + 1]
                         - hx[(size_t)q * ny * (nx + 1) + (size_t)j * (nx + 1) + i];
                real dhy = hy[(size_t)q * (ny + 1) * nx + (size_t)(j + 1) * nx + i]
                         - hy[(size_t)q * (ny + 1) * nx + (size_t)j * nx + i];
                fout[k] = fo - p->dt * (dhx / p->dx + dhy / p->dy)
                             - (p->dt / p->tau) * (fo - feq[k]);
            }
#undef PAD
    free(P);
    free(feq);
    free(hx);
    free(hy);
}

/* ------------------------------------------------------------------------ */
/* Averaged density profile of the mixing layer (Sec. IV.A, the profile of   */
/* Fig. 4): the density averaged along the direction of the interface.  In   */
/* this code the interface lies along x (the periodic axis), so              */
/*   rho_bar(y_j) = (1/nx) sum_i rho(x_i, y_j),  rho = sum_q f_q (Eq. 10),   */
/* the integral over one period by the rectangle rule.                       */
/* ------------------------------------------------------------------------ */
void oklb_mean_density(const oklb_params* p, const real* f, real* out)
{
    const int nx = p->nx, ny = p->ny;
    const size_t n = (size_t)nx * ny;
    for (int j = 0; j < ny; ++j) {
        real s = 0.0;
        for (int i = 0; i < nx; ++i) {
            real rho = 0.0;
            for (int q = 0; q < NQ; ++q) rho += f[(size_t)q * n + (size_t)j * nx + i];
            s += rho;
        }
        out[j] = s / nx;
    }
}

/* ------------------------------------------------------------------------ */
/* Diagnostics of one state (Sec. IV: E_x = rho u^2 / 2 of the cross-stream   */
/* component and its maximum over the domain; conservation sums):            */
/*  d[0] = sum rho, d[1] = sum rho u_x, d[2] = sum rho u_y,                   */
/*  d[3] = sum rho (T + |u|^2/2), d[4] = max |u_y|, d[5] = max rho u_y^2 / 2,  */
/*  d[6] = sum rho u_y^2 / 2.  Sums are over interior nodes, unweighted.       */
/*  In the complex build the two maxima are taken over real parts.             */
/* Row partials are summed in row order, so the result is deterministic.      */
/* ------------------------------------------------------------------------ */
void oklb_diag(const oklb_params* p, const real* f, real d[7])
{
    const int nx = p->nx, ny = p->ny;
    const size_t n = (size_t)nx * ny;
    double vx[NQ], vy[NQ];
    oklb_velocity_set(p->v, vx, vy);
    real* rows = (real*)malloc(sizeof(real) * 5 * ny);
    double* rmax = (double*)malloc(sizeof(double) * 2 * ny);
#pragma omp parallel for schedule(static)
    for (int j = 0; j < ny; ++j) {
        real s[5] = {0, 0, 0, 0, 0};
        double m4 = 0.0, m5 = 0.0;
        for (int i = 0; i < nx; ++i) {
            real fl[NQ], rho, ux, uy, T;
            for (int q = 0; q < NQ; ++q) fl[q] = f[(size_t)q * n + (size_t)j * nx + i];
            moments_of(fl, vx, vy, &rho, &ux, &uy, &T);
            s[0] += rho;
            s[1] += rho * ux;
            s[2] += rho * uy;
            s[3] += rho * (T + (ux * ux + uy * uy) / 2.0);
            s[4] += rho * uy * uy / 2.0;
            double a = fabs(RE(uy));
            double ex = RE(rho * uy * uy / 2.0);
            if (a > m4) m4 = a;
            if (ex > m5) m5 = ex;
        }
        for (int t = 0; t < 5; ++t) rows[(size_t)5 * j + t] = s[t];
        rmax[2 * j] = m4;
        rmax[2 * j + 1] = m5;
    }
    real s[5] = {0, 0, 0, 0, 0};
    double m4 = 0.0, m5 = 0.0;
    for (int j = 0; j < ny; ++j) {
        for (int t = 0; t < 5; ++t) s[t] += rows[(size_t)5 * j + t];
        if (rmax[2 * j] > m4) m4 = rmax[2 * j];
        if (rmax[2 * j + 1] > m5) m5 = rmax[2 * j + 1];
    }
    d[0] = s[0];
    d[1] = s[1];
    d[2] = s[2];
    d[3] = s[3];
    d[4] = m4;
    d[5] = m5;
    d[6] = s[4];
    free(rows);
    free(rmax);
}

/* n steps from f (overwritten with the final state).  If sample_every > 0,
 * the diagnostics of the states after 0, s, 2s, ... steps are written to
 * diag[7*m] (m-th sample), at most cap samples; *count receives the number. */
void oklb_run(const oklb_params* p, real* f, const real* fixed, int64_t nsteps,
              int32_t sample_every, real* diag, int64_t cap, int64_t* count)
{
    const size_t n = (size_t)NQ * p->nx * p->ny;
    real* g = (real*)malloc(sizeof(real) * n);
    int64_t m = 0;
    if (sample_every > 0 && m < cap) oklb_diag(p, f, diag + 7 * m++);
    for (int64_t s = 1; s <= nsteps; ++s) {
        oklb_step(p, f, fixed, g);
        memcpy(f, g, sizeof(real) * n);
        if (sample_every > 0 && s % sample_every == 0 && m < cap) oklb_diag(p, f, diag + 7 * m++);
    }
    if (count) *count = m;
    free(g);
}
