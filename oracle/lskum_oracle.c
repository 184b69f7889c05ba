/*
 * lskum_oracle.c -- plain, slow FP64 CPU oracle of the q-LSKUM hot path.
 *
 * TEST INFRASTRUCTURE ONLY. Only tests/, the smoke check and the benchmark's
 * CPU-baseline leg may load this library. It shares no code, header, table
 * or constant generator with the CUDA path, and the CUDA path never calls it.
 *
 * Method: Mamidi et al., "On the performance of GPU accelerated q-LSKUM based
 * meshfree solvers in Fortran, C++, Python, and Julia" (2021).
 *   - conserved vector, Euler fluxes and specific energy: Section 2, Eqs. 1-3
 *   - kinetic (Maxwellian) basis and CIR splitting: Section 2, Eqs. 4-9
 *   - stencil N(P0) and first-order least squares: Section 2, Eqs. 10-11
 *   - semi-discrete LSKUM, split-stencil flux derivatives and the split
 *     stencils: Eqs. 12-14
 *   - four-stage third-order SSP-RK with local time stepping: Section 2
 *     (paragraph after Eq. 14)
 *   - second-order split-flux derivatives: Section 2.1, Eq. 24 with the
 *     q-variable perturbation of Eq. 27
 *   - q-variables: Eq. 26; modified q-variables q~: Eq. 28
 *   - implicit q-derivatives with inner iterations: Eq. 29 (three inner
 *     iterations in the paper; a parameter here)
 *   - solver loop (timestep, 4 x {q_variables, q_derivatives, flux_residual,
 *     state_update(rk)}, residue): Algorithm 1
 *
 * The paper does not print the split-flux closed forms, the boundary fluxes,
 * the time-step formula, the residue norm or the force integral. The readings
 * taken here (all identical on the CUDA side) are:
 *   - gamma = 1.4 (parameter). Free stream rho = 1, p = 1/gamma,
 *     u = M (cos a, sin a).
 *   - Split fluxes: half-range moments of the 2D Maxwellian with internal
 *     energy; with beta = rho/(2p), S = u_a sqrt(beta),
 *     A(+/-) = erfc(-/+ S)/2, B = exp(-S^2) / (2 sqrt(pi beta)):
 *        G1 = rho (u_a A +/- B)
 *        G_a = (p + rho u_a^2) A +/- rho u_a B
 *        G_b = rho u_b (u_a A +/- B)
 *        G4 = (p + rho e) u_a A +/- (rho e + p/2) B
 *     (a = split direction, b = transverse direction).
 *   - Frame: interior points use the global (x, y) frame; wall and outer
 *     points use the local frame t = (n_y, -n_x), n. Split stencils:
 *     dG+/ds over {ds < 0}, dG-/ds over {ds > 0}, likewise in n; ds == 0 is in
 *     neither. q-derivatives always use the full stencil, global frame.
 *   - Wall (normal into the fluid): R = dGs+/ds + dGs-/ds + 2 dGn-/dn over
 *     {dn > 0}: molecules arriving from the fluid plus their specular
 *     reflection, which for mass, tangential momentum and energy contributes
 *     the same normal-flux derivative again (wall_factor = 2); after every
 *     stage the wall-normal momentum is removed.
 *   - Outer (normal out of the domain), default: the far-field points hold
 *     the free-stream state (they are not updated and their residual is 0).
 *     Optional kinetic reading: R = dGs+/ds + dGs-/ds + dGn+/dn over {dn < 0}
 *     with the incoming (free-stream) part taken as uniform; it never feeds
 *     the free-stream values back and lets the far field drift, so it is not
 *     the default.
 *   - Inner iterations are Jacobi sweeps started from the first-order
 *     derivatives in every stage.
 *   - Least squares as printed (Eqs. 11, 24, 29) are unweighted. Optional
 *     weights w_j = |P_j - P_i|^(-weight_power) multiply every term of every
 *     least-squares sum (the weighted normal equations); weight_power = 0 is
 *     the printed form.
 *   - dt_i = CFL min_j |P_j - P_i| / (|u_i| + a_i), once per iteration.
 *   - residue = sqrt(sum_i R_rho,i^2) / N, from the stage-1 residual.
 *   - forces: F = -sum_wall (p_i - p_inf) n_i ds_i, ds_i half the sum of the
 *     two adjacent wall-loop segment lengths; chord 1, q_inf = rho_inf M^2 / 2.
 *
 * Compiled with -O2 -ffp-contract=off (no fused multiply-add contraction) and
 * optional OpenMP over points (each point's outputs are written by one
 * thread; reductions are serial, so results do not depend on thread count).
 *
 * Precision. The arithmetic is written once, on the type `real`: double by
 * default (the FP64 oracle), IEEE binary128 (_Float128, a 113-bit significand,
 * libm's *f128 functions) when compiled with -DORC_QUAD. The binary128 build
 * evaluates the same formulas in the same order on the same double inputs
 * (coordinates, normals, states, gamma), converted exactly; it is the
 * extended-precision reference that measures how far an FP64 evaluation of
 * the method lies from the exact result of its formulas. Arrays of `real`
 * cross the library boundary as opaque buffers of orc_real_bytes() bytes per
 * value, filled and read with orc_to_real / orc_from_real (value = hi + lo).
 */

#ifdef ORC_QUAD
#define __STDC_WANT_IEC_60559_TYPES_EXT__ 1
#endif
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef ORC_QUAD
typedef _Float128 real;
#define R_LIT(v) v##F128
#define R_EXP expf128
#define R_LOG logf128
#define R_ERFC erfcf128
#define R_SQRT sqrtf128
#define R_POW powf128
#define R_SIN sinf128
#define R_COS cosf128
#else
typedef double real;
#define R_LIT(v) v
#define R_EXP exp
#define R_LOG log
#define R_ERFC erfc
#define R_SQRT sqrt
#define R_POW pow
#define R_SIN sin
#define R_COS cos
#endif

#define ORC_PI R_LIT(3.14159265358979323846264338327950288)

enum { ORC_INTERIOR = 0, ORC_WALL = 1, ORC_OUTER = 2 };

typedef struct {
    int64_t n;
    const double* x;
    const double* y;
    const double* nx;
    const double* ny;
    const int8_t* flag;
    const int32_t* off;
    const int32_t* nbr;
    double gamma;
    double wall_factor; /* weight of dGn-/dn at wall points (2: mirror wall) */
    int order;          /* 2: q~ defect correction (Eq. 27-28); 1: first order (Eq. 13) */
    int outer_mode;     /* 1: outer points held at the free stream; 0: kinetic reading */
    double weight_power; /* least-squares weight |P_j - P_i|^-weight_power; 0: unweighted */
} orc_cloud;

/* ------------------------------------------------------------ real buffers */

/* Bytes of one `real` value (8 in the FP64 build, 16 in the binary128 build). */
int orc_real_bytes(void) { return (int)sizeof(real); }

/* out[i] = hi[i] + lo[i] (lo may be NULL), rounded to `real`. */
void orc_to_real(int64_t n, const double* hi, const double* lo, real* out) {
    for (int64_t i = 0; i < n; ++i) out[i] = lo ? (real)hi[i] + (real)lo[i] : (real)hi[i];
}

/* hi[i] = in[i] rounded to double; lo[i] (lo may be NULL) = the remainder,
 * rounded to double. */
void orc_from_real(int64_t n, const real* in, double* hi, double* lo) {
    for (int64_t i = 0; i < n; ++i) {
        double h = (double)in[i];
        hi[i] = h;
        if (lo) lo[i] = (double)(in[i] - (real)h);
    }
}

/* Offset P_j - P_i of neighbour j seen from point i (exact in binary128). */
static real offset_x(const orc_cloud* c, int64_t i, int64_t j) { return (real)c->x[j] - (real)c->x[i]; }
static real offset_y(const orc_cloud* c, int64_t i, int64_t j) { return (real)c->y[j] - (real)c->y[i]; }

/* Weight of neighbour offset (dx, dy) in the least-squares sums. */
static real ls_weight(const orc_cloud* c, real dx, real dy) {
    if (c->weight_power == 0.0) return 1;
    return R_POW(dx * dx + dy * dy, (real)-0.5 * (real)c->weight_power);
}

/* ---------------------------------------------------------------- state maps */

/* Eqs. 2-3: conserved U = (rho, rho u1, rho u2, rho e) from W = (rho, u1, u2, p). */
void orc_prim_to_cons(const real* W, double gamma, real* U) {
    real rho = W[0], u1 = W[1], u2 = W[2], p = W[3];
    U[0] = rho;
    U[1] = rho * u1;
    U[2] = rho * u2;
    U[3] = p / ((real)gamma - 1) + (real)0.5 * rho * (u1 * u1 + u2 * u2);
}

void orc_cons_to_prim(const real* U, double gamma, real* W) {
    real rho = U[0];
    real u1 = U[1] / rho, u2 = U[2] / rho;
    W[0] = rho;
    W[1] = u1;
    W[2] = u2;
    W[3] = ((real)gamma - 1) * (U[3] - (real)0.5 * rho * (u1 * u1 + u2 * u2));
}

/* Eq. 26: q = (ln rho + ln beta/(gamma-1) - beta |u|^2, 2 beta u1, 2 beta u2, -2 beta),
 * beta = 1/(2RT) = rho/(2p). */
void orc_prim_to_q(const real* W, double gamma, real* q) {
    real rho = W[0], u1 = W[1], u2 = W[2], p = W[3];
    real beta = rho / (2 * p);
    q[0] = R_LOG(rho) + R_LOG(beta) / ((real)gamma - 1) - beta * (u1 * u1 + u2 * u2);
    q[1] = 2 * beta * u1;
    q[2] = 2 * beta * u2;
    q[3] = -2 * beta;
}

/* Inverse of Eq. 26 (the map U <-> q is one to one, Section 2.1). Returns 0,
 * or 1 when q4 >= 0 (no positive temperature). */
int orc_q_to_prim(const real* q, double gamma, real* W) {
    real beta = (real)-0.5 * q[3];
    if (!(beta > 0)) {
        W[0] = W[1] = W[2] = W[3] = NAN;
        return 1;
    }
    real u1 = q[1] / (2 * beta);
    real u2 = q[2] / (2 * beta);
    real rho = R_EXP(q[0] - R_LOG(beta) / ((real)gamma - 1) + beta * (u1 * u1 + u2 * u2));
    W[0] = rho;
    W[1] = u1;
    W[2] = u2;
    W[3] = rho / (2 * beta);
    return 0;
}

/* ------------------------------------------------------------- split fluxes */

/* Kinetic split flux G^sign along direction dir (0: x, the split velocity is
 * W[1]; 1: y, the split velocity is W[2]) for W = (rho, u1, u2, p); output in
 * the components of W's frame (mass, momentum 1, momentum 2, energy).
 * Half-range moments of the Maxwellian of Eq. 5 over v_dir > 0 (sign = +1) or
 * v_dir < 0 (sign = -1), the CIR split of Eqs. 8-9. */
void orc_split_flux(const real* W, int dir, int sign, double gamma, real* G) {
    real rho = W[0], p = W[3];
    real ua = dir == 0 ? W[1] : W[2];
    real ub = dir == 0 ? W[2] : W[1];
    real beta = rho / (2 * p);
    real S = ua * R_SQRT(beta);
    real sg = sign > 0 ? 1 : -1;
    real A = (real)0.5 * R_ERFC(-sg * S);
    real B = R_EXP(-S * S) / (2 * R_SQRT(ORC_PI * beta));
    real rhoe = p / ((real)gamma - 1) + (real)0.5 * rho * (ua * ua + ub * ub);
    real g_mass = rho * (ua * A + sg * B);
    real g_a = (p + rho * ua * ua) * A + sg * rho * ua * B;
    real g_b = rho * ub * (ua * A + sg * B);
    real g_e = (p + rhoe) * ua * A + sg * (rhoe + (real)0.5 * p) * B;
    G[0] = g_mass;
    G[1] = dir == 0 ? g_a : g_b;
    G[2] = dir == 0 ? g_b : g_a;
    G[3] = g_e;
}

/* Array forms of the point maps (n rows of 4). */
void orc_prim_to_q_n(int64_t n, const real* W, double gamma, real* q) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) orc_prim_to_q(W + 4 * i, gamma, q + 4 * i);
}
void orc_q_to_prim_n(int64_t n, const real* q, double gamma, real* W) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) orc_q_to_prim(q + 4 * i, gamma, W + 4 * i);
}
void orc_prim_to_cons_n(int64_t n, const real* W, double gamma, real* U) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) orc_prim_to_cons(W + 4 * i, gamma, U + 4 * i);
}
void orc_cons_to_prim_n(int64_t n, const real* U, double gamma, real* W) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) orc_cons_to_prim(U + 4 * i, gamma, W + 4 * i);
}
void orc_split_flux_n(int64_t n, const real* W, int dir, int sign, double gamma, real* G) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) orc_split_flux(W + 4 * i, dir, sign, gamma, G + 4 * i);
}

/* ---------------------------------------------------------- q-derivatives */

/* One least-squares sweep over the full stencil, global frame. With px, py
 * NULL it is the first-order formula of Eq. 11 applied to q; otherwise it is
 * Eq. 29 with the perturbations dq~ = q~_j - q~_0 of Eq. 28 built from the
 * previous derivative iterate (px, py). q, px, py, qx, qy are n x 4. */
void orc_ls_sweep(const orc_cloud* c, const real* q, const real* px, const real* py,
                  real* qx, real* qy) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < c->n; ++i) {
        real sxx = 0, sxy = 0, syy = 0;
        real sxq[4] = {0, 0, 0, 0}, syq[4] = {0, 0, 0, 0};
        for (int32_t e = c->off[i]; e < c->off[i + 1]; ++e) {
            int32_t j = c->nbr[e];
            real dx = offset_x(c, i, j);
            real dy = offset_y(c, i, j);
            real w = ls_weight(c, dx, dy);
            sxx += w * dx * dx;
            sxy += w * dx * dy;
            syy += w * dy * dy;
            for (int m = 0; m < 4; ++m) {
                real dq;
                if (px == NULL) {
                    dq = q[4 * j + m] - q[4 * i + m];
                } else {
                    real qtj = q[4 * j + m] - (real)0.5 * (dx * px[4 * j + m] + dy * py[4 * j + m]);
                    real qt0 = q[4 * i + m] - (real)0.5 * (dx * px[4 * i + m] + dy * py[4 * i + m]);
                    dq = qtj - qt0;
                }
                sxq[m] += w * dx * dq;
                syq[m] += w * dy * dq;
            }
        }
        real det = sxx * syy - sxy * sxy;
        for (int m = 0; m < 4; ++m) {
            qx[4 * i + m] = (sxq[m] * syy - sxy * syq[m]) / det;
            qy[4 * i + m] = (sxx * syq[m] - sxy * sxq[m]) / det;
        }
    }
}

/* q_derivatives(): the first-order sweep, then `inner` Jacobi sweeps of the
 * implicit defect-corrected formula (Eqs. 28-29), each using only the
 * previous sweep's derivatives. */
void orc_q_derivatives(const orc_cloud* c, const real* q, int inner, real* qx, real* qy) {
    size_t sz = sizeof(real) * 4 * (size_t)c->n;
    real* px = (real*)malloc(sz);
    real* py = (real*)malloc(sz);
    orc_ls_sweep(c, q, NULL, NULL, qx, qy);
    for (int sweep = 1; sweep <= inner; ++sweep) {
        memcpy(px, qx, sz);
        memcpy(py, qy, sz);
        orc_ls_sweep(c, q, px, py, qx, qy);
    }
    free(px);
    free(py);
}

/* ------------------------------------------------------------ flux residual */

static void frame_of(const orc_cloud* c, int64_t i, real* tx, real* ty, real* nx, real* ny) {
    if (c->flag[i] == ORC_INTERIOR) {
        *tx = 1; *ty = 0; *nx = 0; *ny = 1;
    } else {
        *nx = c->nx[i]; *ny = c->ny[i];
        *tx = c->ny[i]; *ty = -(real)c->nx[i];
    }
}

/* Residual R_i = sum of the split-flux derivatives at point i (Eq. 12), each
 * from Eq. 24 over its split stencil (Eq. 14) with the q~ perturbation of
 * Eqs. 27-28, conserved
 * components in the global frame; dU/dt + R = 0. Returns the number of
 * split stencils whose determinant was not positive (their derivative is
 * taken as 0). */
static int residual_point(const orc_cloud* c, int64_t i, const real* q, const real* qx,
                          const real* qy, real* R) {
    if (c->outer_mode == 1 && c->flag[i] == ORC_OUTER) {
        /* far-field points held at the free stream are not unknowns */
        R[0] = R[1] = R[2] = R[3] = 0;
        return 0;
    }
    real tx, ty, nx, ny;
    frame_of(c, i, &tx, &ty, &nx, &ny);
    int flag = c->flag[i];
    /* stencil slots: 0 s+ (ds<0), 1 s- (ds>0), 2 n+ (dn<0), 3 n- (dn>0) */
    int use[4] = {1, 1, flag != ORC_WALL, flag != ORC_OUTER};
    real sss[4] = {0}, ssn[4] = {0}, snn[4] = {0};
    real sdg_s[4][4] = {{0}}, sdg_n[4][4] = {{0}};
    double gamma = c->gamma;
    for (int32_t e = c->off[i]; e < c->off[i + 1]; ++e) {
        int32_t j = c->nbr[e];
        real dx = offset_x(c, i, j);
        real dy = offset_y(c, i, j);
        real ds = dx * tx + dy * ty;
        real dn = dx * nx + dy * ny;
        real qtj[4], qt0[4], Wj[4], W0[4], Lj[4], L0[4];
        for (int m = 0; m < 4; ++m) {
            if (c->order == 1) {
                qtj[m] = q[4 * j + m];
                qt0[m] = q[4 * i + m];
            } else {
                qtj[m] = q[4 * j + m] - (real)0.5 * (dx * qx[4 * j + m] + dy * qy[4 * j + m]);
                qt0[m] = q[4 * i + m] - (real)0.5 * (dx * qx[4 * i + m] + dy * qy[4 * i + m]);
            }
        }
        orc_q_to_prim(qtj, gamma, Wj);
        orc_q_to_prim(qt0, gamma, W0);
        /* velocities into the local frame: (rho, u_s, u_n, p) */
        Lj[0] = Wj[0]; Lj[1] = Wj[1] * tx + Wj[2] * ty; Lj[2] = Wj[1] * nx + Wj[2] * ny; Lj[3] = Wj[3];
        L0[0] = W0[0]; L0[1] = W0[1] * tx + W0[2] * ty; L0[2] = W0[1] * nx + W0[2] * ny; L0[3] = W0[3];
        int slot_s = ds < 0 ? 0 : (ds > 0 ? 1 : -1);
        int slot_n = dn < 0 ? 2 : (dn > 0 ? 3 : -1);
        int slots[2] = {slot_s, slot_n};
        for (int k = 0; k < 2; ++k) {
            int sl = slots[k];
            if (sl < 0 || !use[sl]) continue;
            int dir = sl < 2 ? 0 : 1;
            int sign = (sl == 0 || sl == 2) ? 1 : -1;
            real Gj[4], G0[4];
            orc_split_flux(Lj, dir, sign, gamma, Gj);
            orc_split_flux(L0, dir, sign, gamma, G0);
            real w = ls_weight(c, dx, dy);
            sss[sl] += w * ds * ds;
            ssn[sl] += w * ds * dn;
            snn[sl] += w * dn * dn;
            for (int m = 0; m < 4; ++m) {
                real dG = Gj[m] - G0[m];
                sdg_s[sl][m] += w * ds * dG;
                sdg_n[sl][m] += w * dn * dG;
            }
        }
    }
    int bad = 0;
    real Rl[4] = {0, 0, 0, 0};
    for (int sl = 0; sl < 4; ++sl) {
        if (!use[sl]) continue;
        real det = sss[sl] * snn[sl] - ssn[sl] * ssn[sl];
        if (!(det > 0)) { ++bad; continue; }
        for (int m = 0; m < 4; ++m) {
            real d;
            if (sl < 2) /* d/ds: Cramer's rule, first unknown */
                d = (sdg_s[sl][m] * snn[sl] - ssn[sl] * sdg_n[sl][m]) / det;
            else        /* d/dn: second unknown */
                d = (sss[sl] * sdg_n[sl][m] - ssn[sl] * sdg_s[sl][m]) / det;
            if (sl == 3 && flag == ORC_WALL) d = (real)c->wall_factor * d;
            Rl[m] += d;
        }
    }
    R[0] = Rl[0];
    R[1] = Rl[1] * tx + Rl[2] * nx;
    R[2] = Rl[1] * ty + Rl[2] * ny;
    R[3] = Rl[3];
    return bad;
}

int orc_flux_residual(const orc_cloud* c, const real* q, const real* qx, const real* qy,
                      real* R) {
    int bad = 0;
#pragma omp parallel for schedule(static) reduction(+ : bad)
    for (int64_t i = 0; i < c->n; ++i) bad += residual_point(c, i, q, qx, qy, R + 4 * i);
    return bad;
}

/* Residual at a subset of points only (for sampled checks on large clouds). */
int orc_flux_residual_subset(const orc_cloud* c, const real* q, const real* qx,
                             const real* qy, const int64_t* idx, int64_t m, real* R) {
    int bad = 0;
#pragma omp parallel for schedule(static) reduction(+ : bad)
    for (int64_t k = 0; k < m; ++k) bad += residual_point(c, idx[k], q, qx, qy, R + 4 * k);
    return bad;
}

/* --------------------------------------------------------- time step, RK */

/* Local time step dt_i = CFL min_j d_ij / (|u_i| + a_i), a = sqrt(gamma p / rho). */
void orc_timestep(const orc_cloud* c, const real* W, double cfl, real* dt) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < c->n; ++i) {
        real dmin = INFINITY;
        for (int32_t e = c->off[i]; e < c->off[i + 1]; ++e) {
            int32_t j = c->nbr[e];
            real dx = offset_x(c, i, j);
            real dy = offset_y(c, i, j);
            real d = R_SQRT(dx * dx + dy * dy);
            if (d < dmin) dmin = d;
        }
        const real* w = W + 4 * i;
        real speed = R_SQRT(w[1] * w[1] + w[2] * w[2]) + R_SQRT((real)c->gamma * w[3] / w[0]);
        dt[i] = (real)cfl * dmin / speed;
    }
}

/* One stage of the four-stage third-order SSP Runge-Kutta scheme with local
 * time step dt (dU/dt = -R), for one point's conserved 4-vector:
 *   stage 1: U1 = U0 - dt/2 R(U0)
 *   stage 2: U2 = U1 - dt/2 R(U1)
 *   stage 3: U3 = 2/3 U0 + 1/3 (U2 - dt/2 R(U2))
 *   stage 4: U4 = U3 - dt/2 R(U3)                                          */
void orc_rk_stage(int stage, const real* U0, const real* U, const real* R, real dt,
                  real* Unew) {
    for (int m = 0; m < 4; ++m) {
        if (stage == 3)
            Unew[m] = ((real)2 / 3) * U0[m] + ((real)1 / 3) * (U[m] - (real)0.5 * dt * R[m]);
        else
            Unew[m] = U[m] - (real)0.5 * dt * R[m];
    }
}

/* Wall condition on the state: keep rho, the tangential momentum and rho e;
 * the momentum normal to the wall is set to zero. */
void orc_wall_project(real* U, double nx, double ny) {
    real tx = ny, ty = -(real)nx;
    real ms = U[1] * tx + U[2] * ty;
    U[1] = ms * tx;
    U[2] = ms * ty;
}

/* residue = sqrt(sum_i R_rho,i^2) / N (serial sum in point order). */
real orc_residue(int64_t n, const real* R) {
    real s = 0;
    for (int64_t i = 0; i < n; ++i) s += R[4 * i] * R[4 * i];
    return R_SQRT(s) / (real)n;
}

/* Pressure force on the wall loop and the lift/drag coefficients. The loop
 * lists the wall points in order (closed: the last connects to the first). */
void orc_forces(const orc_cloud* c, const real* W, const int64_t* loop, int64_t m,
                double mach, double alpha_deg, real* cl, real* cd) {
    real p_inf = 1 / (real)c->gamma;
    real fx = 0, fy = 0;
    for (int64_t k = 0; k < m; ++k) {
        int64_t i = loop[k];
        int64_t ip = loop[(k + 1) % m];
        int64_t im = loop[(k + m - 1) % m];
        real next_x = offset_x(c, i, ip), next_y = offset_y(c, i, ip);
        real prev_x = offset_x(c, im, i), prev_y = offset_y(c, im, i);
        real lp = R_SQRT(next_x * next_x + next_y * next_y);
        real lm = R_SQRT(prev_x * prev_x + prev_y * prev_y);
        real ds = (real)0.5 * (lp + lm);
        real dp = W[4 * i + 3] - p_inf;
        fx -= dp * (real)c->nx[i] * ds;
        fy -= dp * (real)c->ny[i] * ds;
    }
    real a = (real)alpha_deg * ORC_PI / 180;
    real qinf = (real)0.5 * (real)mach * (real)mach;
    *cl = (-fx * R_SIN(a) + fy * R_COS(a)) / qinf;
    *cd = (fx * R_COS(a) + fy * R_SIN(a)) / qinf;
}

void orc_freestream(double gamma, double mach, double alpha_deg, real* W) {
    real a = (real)alpha_deg * ORC_PI / 180;
    W[0] = 1;
    W[1] = (real)mach * R_COS(a);
    W[2] = (real)mach * R_SIN(a);
    W[3] = 1 / (real)gamma;
}

/* --------------------------------------------------------------- solver */

/* Algorithm 1: `iters` pseudo-time iterations from primitive state W (n x 4,
 * updated in place). Each iteration: timestep; four stages of q_variables,
 * q_derivatives, flux_residual, state_update(rk); residue. res[n_it] receives
 * the residue of each iteration (may be NULL). R1 (may be NULL) receives the
 * stage-1 residual of the last iteration. Returns 0, or the iteration number
 * (1-based) at which a non-positive density/pressure or a non-finite value
 * appeared. */
int orc_iterate(const orc_cloud* c, real* W, int iters, double cfl, int inner, real* res,
                real* R1) {
    int64_t n = c->n;
    double gamma = c->gamma;
    size_t sz = sizeof(real) * 4 * (size_t)n;
    real* U0 = (real*)malloc(sz);
    real* U = (real*)malloc(sz);
    real* q = (real*)malloc(sz);
    real* qx = (real*)malloc(sz);
    real* qy = (real*)malloc(sz);
    real* R = (real*)malloc(sz);
    real* dt = (real*)malloc(sizeof(real) * (size_t)n);
    int status = 0;
    for (int it = 0; it < iters && status == 0; ++it) {
        orc_timestep(c, W, cfl, dt);
        for (int64_t i = 0; i < n; ++i) orc_prim_to_cons(W + 4 * i, gamma, U0 + 4 * i);
        memcpy(U, U0, sz);
        real r = 0;
        for (int stage = 1; stage <= 4; ++stage) {
            for (int64_t i = 0; i < n; ++i) orc_prim_to_q(W + 4 * i, gamma, q + 4 * i);
            orc_q_derivatives(c, q, inner, qx, qy);
            orc_flux_residual(c, q, qx, qy, R);
            if (stage == 1) {
                r = orc_residue(n, R);
                if (R1 && it == iters - 1) memcpy(R1, R, sz);
            }
            for (int64_t i = 0; i < n; ++i) {
                real un[4];
                if (c->outer_mode == 1 && c->flag[i] == ORC_OUTER) continue;
                orc_rk_stage(stage, U0 + 4 * i, U + 4 * i, R + 4 * i, dt[i], un);
                if (c->flag[i] == ORC_WALL) orc_wall_project(un, c->nx[i], c->ny[i]);
                memcpy(U + 4 * i, un, sizeof(un));
                orc_cons_to_prim(un, gamma, W + 4 * i);
                const real* w = W + 4 * i;
                if (!(w[0] > 0) || !(w[3] > 0) || !isfinite(w[1]) || !isfinite(w[2]))
                    status = it + 1;
            }
        }
        if (res) res[it] = r;
        if (!isfinite(r)) status = it + 1;
    }
    free(U0); free(U); free(q); free(qx); free(qy); free(R); free(dt);
    return status;
}

/* R(W): the stage-1 residual of the state W (q_variables, q_derivatives,
 * flux_residual) without updating it. */
int orc_residual_of_state(const orc_cloud* c, const real* W, int inner, real* R) {
    int64_t n = c->n;
    size_t sz = sizeof(real) * 4 * (size_t)n;
    real* q = (real*)malloc(sz);
    real* qx = (real*)malloc(sz);
    real* qy = (real*)malloc(sz);
    for (int64_t i = 0; i < n; ++i) orc_prim_to_q(W + 4 * i, c->gamma, q + 4 * i);
    orc_q_derivatives(c, q, inner, qx, qy);
    int bad = orc_flux_residual(c, q, qx, qy, R);
    free(q); free(qx); free(qy);
    return bad;
}

int orc_num_threads(void) {
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}
