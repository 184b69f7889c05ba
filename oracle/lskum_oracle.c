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
 */

#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_PI 3.14159265358979323846

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

/* Weight of neighbour offset (dx, dy) in the least-squares sums. */
static double ls_weight(const orc_cloud* c, double dx, double dy) {
    if (c->weight_power == 0.0) return 1.0;
    return pow(dx * dx + dy * dy, -0.5 * c->weight_power);
}

/* ---------------------------------------------------------------- state maps */

/* Eqs. 2-3: conserved U = (rho, rho u1, rho u2, rho e) from W = (rho, u1, u2, p). */
void orc_prim_to_cons(const double* W, double gamma, double* U) {
    double rho = W[0], u1 = W[1], u2 = W[2], p = W[3];
    U[0] = rho;
    U[1] = rho * u1;
    U[2] = rho * u2;
    U[3] = p / (gamma - 1.0) + 0.5 * rho * (u1 * u1 + u2 * u2);
}

void orc_cons_to_prim(const double* U, double gamma, double* W) {
    double rho = U[0];
    double u1 = U[1] / rho, u2 = U[2] / rho;
    W[0] = rho;
    W[1] = u1;
    W[2] = u2;
    W[3] = (gamma - 1.0) * (U[3] - 0.5 * rho * (u1 * u1 + u2 * u2));
}

/* Eq. 26: q = (ln rho + ln beta/(gamma-1) - beta |u|^2, 2 beta u1, 2 beta u2, -2 beta),
 * beta = 1/(2RT) = rho/(2p). */
void orc_prim_to_q(const double* W, double gamma, double* q) {
    double rho = W[0], u1 = W[1], u2 = W[2], p = W[3];
    double beta = rho / (2.0 * p);
    q[0] = log(rho) + log(beta) / (gamma - 1.0) - beta * (u1 * u1 + u2 * u2);
    q[1] = 2.0 * beta * u1;
    q[2] = 2.0 * beta * u2;
    q[3] = -2.0 * beta;
}

/* Inverse of Eq. 26 (the map U <-> q is one to one, Section 2.1). Returns 0,
 * or 1 when q4 >= 0 (no positive temperature). */
int orc_q_to_prim(const double* q, double gamma, double* W) {
    double beta = -0.5 * q[3];
    if (!(beta > 0.0)) {
        W[0] = W[1] = W[2] = W[3] = NAN;
        return 1;
    }
    double u1 = q[1] / (2.0 * beta);
    double u2 = q[2] / (2.0 * beta);
    double rho = exp(q[0] - log(beta) / (gamma - 1.0) + beta * (u1 * u1 + u2 * u2));
    W[0] = rho;
    W[1] = u1;
    W[2] = u2;
    W[3] = rho / (2.0 * beta);
    return 0;
}

/* ------------------------------------------------------------- split fluxes */

/* Kinetic split flux G^sign along direction dir (0: x, the split velocity is
 * W[1]; 1: y, the split velocity is W[2]) for W = (rho, u1, u2, p); output in
 * the components of W's frame (mass, momentum 1, momentum 2, energy).
 * Half-range moments of the Maxwellian of Eq. 5 over v_dir > 0 (sign = +1) or
 * v_dir < 0 (sign = -1), the CIR split of Eqs. 8-9. */
void orc_split_flux(const double* W, int dir, int sign, double gamma, double* G) {
    double rho = W[0], p = W[3];
    double ua = dir == 0 ? W[1] : W[2];
    double ub = dir == 0 ? W[2] : W[1];
    double beta = rho / (2.0 * p);
    double S = ua * sqrt(beta);
    double sg = sign > 0 ? 1.0 : -1.0;
    double A = 0.5 * erfc(-sg * S);
    double B = exp(-S * S) / (2.0 * sqrt(ORC_PI * beta));
    double rhoe = p / (gamma - 1.0) + 0.5 * rho * (ua * ua + ub * ub);
    double g_mass = rho * (ua * A + sg * B);
    double g_a = (p + rho * ua * ua) * A + sg * rho * ua * B;
    double g_b = rho * ub * (ua * A + sg * B);
    double g_e = (p + rhoe) * ua * A + sg * (rhoe + 0.5 * p) * B;
    G[0] = g_mass;
    G[1] = dir == 0 ? g_a : g_b;
    G[2] = dir == 0 ? g_b : g_a;
    G[3] = g_e;
}

/* Array forms of the point maps (n rows of 4). */
void orc_prim_to_q_n(int64_t n, const double* W, double gamma, double* q) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) orc_prim_to_q(W + 4 * i, gamma, q + 4 * i);
}
void orc_q_to_prim_n(int64_t n, const double* q, double gamma, double* W) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) orc_q_to_prim(q + 4 * i, gamma, W + 4 * i);
}
void orc_prim_to_cons_n(int64_t n, const double* W, double gamma, double* U) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) orc_prim_to_cons(W + 4 * i, gamma, U + 4 * i);
}
void orc_cons_to_prim_n(int64_t n, const double* U, double gamma, double* W) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) orc_cons_to_prim(U + 4 * i, gamma, W + 4 * i);
}
void orc_split_flux_n(int64_t n, const double* W, int dir, int sign, double gamma, double* G) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) orc_split_flux(W + 4 * i, dir, sign, gamma, G + 4 * i);
}

/* ---------------------------------------------------------- q-derivatives */

/* One least-squares sweep over the full stencil, global frame. With px, py
 * NULL it is the first-order formula of Eq. 11 applied to q; otherwise it is
 * Eq. 29 with the perturbations dq~ = q~_j - q~_0 of Eq. 28 built from the
 * previous derivative iterate (px, py). q, px, py, qx, qy are n x 4. */
void orc_ls_sweep(const orc_cloud* c, const double* q, const double* px, const double* py,
                  double* qx, double* qy) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < c->n; ++i) {
        double sxx = 0, sxy = 0, syy = 0;
        double sxq[4] = {0, 0, 0, 0}, syq[4] = {0, 0, 0, 0};
        for (int32_t e = c->off[i]; e < c->off[i + 1]; ++e) {
            int32_t j = c->nbr[e];
            double dx = c->x[j] - c->x[i];
            double dy = c->y[j] - c->y[i];
            double w = ls_weight(c, dx, dy);
            sxx += w * dx * dx;
            sxy += w * dx * dy;
            syy += w * dy * dy;
            for (int m = 0; m < 4; ++m) {
                double dq;
                if (px == NULL) {
                    dq = q[4 * j + m] - q[4 * i + m];
                } else {
                    double qtj = q[4 * j + m] - 0.5 * (dx * px[4 * j + m] + dy * py[4 * j + m]);
                    double qt0 = q[4 * i + m] - 0.5 * (dx * px[4 * i + m] + dy * py[4 * i + m]);
                    dq = qtj - qt0;
                }
                sxq[m] += w * dx * dq;
                syq[m] += w * dy * dq;
            }
        }
        double det = sxx * syy - sxy * sxy;
        for (int m = 0; m < 4; ++m) {
            qx[4 * i + m] = (sxq[m] * syy - sxy * syq[m]) / det;
            qy[4 * i + m] = (sxx * syq[m] - sxy * sxq[m]) / det;
        }
    }
}

/* q_derivatives(): the first-order sweep, then `inner` Jacobi sweeps of the
 * implicit defect-corrected formula (Eqs. 28-29), each using only the
 * previous sweep's derivatives. */
void orc_q_derivatives(const orc_cloud* c, const double* q, int inner, double* qx, double* qy) {
    size_t sz = sizeof(double) * 4 * (size_t)c->n;
    double* px = (double*)malloc(sz);
    double* py = (double*)malloc(sz);
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

static void frame_of(const orc_cloud* c, int64_t i, double* tx, double* ty, double* nx, double* ny) {
    if (c->flag[i] == ORC_INTERIOR) {
        *tx = 1.0; *ty = 0.0; *nx = 0.0; *ny = 1.0;
    } else {
        *nx = c->nx[i]; *ny = c->ny[i];
        *tx = c->ny[i]; *ty = -c->nx[i];
    }
}

/* Residual R_i = sum of the split-flux derivatives at point i (Eq. 12), each
 * from Eq. 24 over its split stencil (Eq. 14) with the q~ perturbation of
 * Eqs. 27-28, conserved
 * components in the global frame; dU/dt + R = 0. Returns the number of
 * split stencils whose determinant was not positive (their derivative is
 * taken as 0). */
static int residual_point(const orc_cloud* c, int64_t i, const double* q, const double* qx,
                          const double* qy, double* R) {
    if (c->outer_mode == 1 && c->flag[i] == ORC_OUTER) {
        /* far-field points held at the free stream are not unknowns */
        R[0] = R[1] = R[2] = R[3] = 0.0;
        return 0;
    }
    double tx, ty, nx, ny;
    frame_of(c, i, &tx, &ty, &nx, &ny);
    int flag = c->flag[i];
    /* stencil slots: 0 s+ (ds<0), 1 s- (ds>0), 2 n+ (dn<0), 3 n- (dn>0) */
    int use[4] = {1, 1, flag != ORC_WALL, flag != ORC_OUTER};
    double sss[4] = {0}, ssn[4] = {0}, snn[4] = {0};
    double sdg_s[4][4] = {{0}}, sdg_n[4][4] = {{0}};
    double gamma = c->gamma;
    for (int32_t e = c->off[i]; e < c->off[i + 1]; ++e) {
        int32_t j = c->nbr[e];
        double dx = c->x[j] - c->x[i];
        double dy = c->y[j] - c->y[i];
        double ds = dx * tx + dy * ty;
        double dn = dx * nx + dy * ny;
        double qtj[4], qt0[4], Wj[4], W0[4], Lj[4], L0[4];
        for (int m = 0; m < 4; ++m) {
            if (c->order == 1) {
                qtj[m] = q[4 * j + m];
                qt0[m] = q[4 * i + m];
            } else {
                qtj[m] = q[4 * j + m] - 0.5 * (dx * qx[4 * j + m] + dy * qy[4 * j + m]);
                qt0[m] = q[4 * i + m] - 0.5 * (dx * qx[4 * i + m] + dy * qy[4 * i + m]);
            }
        }
        orc_q_to_prim(qtj, gamma, Wj);
        orc_q_to_prim(qt0, gamma, W0);
        /* velocities into the local frame: (rho, u_s, u_n, p) */
        Lj[0] = Wj[0]; Lj[1] = Wj[1] * tx + Wj[2] * ty; Lj[2] = Wj[1] * nx + Wj[2] * ny; Lj[3] = Wj[3];
        L0[0] = W0[0]; L0[1] = W0[1] * tx + W0[2] * ty; L0[2] = W0[1] * nx + W0[2] * ny; L0[3] = W0[3];
        int slot_s = ds < 0.0 ? 0 : (ds > 0.0 ? 1 : -1);
        int slot_n = dn < 0.0 ? 2 : (dn > 0.0 ? 3 : -1);
        int slots[2] = {slot_s, slot_n};
        for (int k = 0; k < 2; ++k) {
            int sl = slots[k];
            if (sl < 0 || !use[sl]) continue;
            int dir = sl < 2 ? 0 : 1;
            int sign = (sl == 0 || sl == 2) ? 1 : -1;
            double Gj[4], G0[4];
            orc_split_flux(Lj, dir, sign, gamma, Gj);
            orc_split_flux(L0, dir, sign, gamma, G0);
            double w = ls_weight(c, dx, dy);
            sss[sl] += w * ds * ds;
            ssn[sl] += w * ds * dn;
            snn[sl] += w * dn * dn;
            for (int m = 0; m < 4; ++m) {
                double dG = Gj[m] - G0[m];
                sdg_s[sl][m] += w * ds * dG;
                sdg_n[sl][m] += w * dn * dG;
            }
        }
    }
    int bad = 0;
    double Rl[4] = {0, 0, 0, 0};
    for (int sl = 0; sl < 4; ++sl) {
        if (!use[sl]) continue;
        double det = sss[sl] * snn[sl] - ssn[sl] * ssn[sl];
        if (!(det > 0.0)) { ++bad; continue; }
        for (int m = 0; m < 4; ++m) {
            double d;
            if (sl < 2) /* d/ds: Cramer's rule, first unknown */
                d = (sdg_s[sl][m] * snn[sl] - ssn[sl] * sdg_n[sl][m]) / det;
            else        /* d/dn: second unknown */
                d = (sss[sl] * sdg_n[sl][m] - ssn[sl] * sdg_s[sl][m]) / det;
            if (sl == 3 && flag == ORC_WALL) d = c->wall_factor * d;
            Rl[m] += d;
        }
    }
    R[0] = Rl[0];
    R[1] = Rl[1] * tx + Rl[2] * nx;
    R[2] = Rl[1] * ty + Rl[2] * ny;
    R[3] = Rl[3];
    return bad;
}

int orc_flux_residual(const orc_cloud* c, const double* q, const double* qx, const double* qy,
                      double* R) {
    int bad = 0;
#pragma omp parallel for schedule(static) reduction(+ : bad)
    for (int64_t i = 0; i < c->n; ++i) bad += residual_point(c, i, q, qx, qy, R + 4 * i);
    return bad;
}

/* Residual at a subset of points only (for sampled checks on large clouds). */
int orc_flux_residual_subset(const orc_cloud* c, const double* q, const double* qx,
                             const double* qy, const int64_t* idx, int64_t m, double* R) {
    int bad = 0;
#pragma omp parallel for schedule(static) reduction(+ : bad)
    for (int64_t k = 0; k < m; ++k) bad += residual_point(c, idx[k], q, qx, qy, R + 4 * k);
    return bad;
}

/* --------------------------------------------------------- time step, RK */

/* Local time step dt_i = CFL min_j d_ij / (|u_i| + a_i), a = sqrt(gamma p / rho). */
void orc_timestep(const orc_cloud* c, const double* W, double cfl, double* dt) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < c->n; ++i) {
        double dmin = INFINITY;
        for (int32_t e = c->off[i]; e < c->off[i + 1]; ++e) {
            int32_t j = c->nbr[e];
            double dx = c->x[j] - c->x[i];
            double dy = c->y[j] - c->y[i];
            double d = sqrt(dx * dx + dy * dy);
            if (d < dmin) dmin = d;
        }
        const double* w = W + 4 * i;
        double speed = sqrt(w[1] * w[1] + w[2] * w[2]) + sqrt(c->gamma * w[3] / w[0]);
        dt[i] = cfl * dmin / speed;
    }
}

/* One stage of the four-stage third-order SSP Runge-Kutta scheme with local
 * time step dt (dU/dt = -R), for one point's conserved 4-vector:
 *   stage 1: U1 = U0 - dt/2 R(U0)
 *   stage 2: U2 = U1 - dt/2 R(U1)
 *   stage 3: U3 = 2/3 U0 + 1/3 (U2 - dt/2 R(U2))
 *   stage 4: U4 = U3 - dt/2 R(U3)                                          */
void orc_rk_stage(int stage, const double* U0, const double* U, const double* R, double dt,
                  double* Unew) {
    for (int m = 0; m < 4; ++m) {
        if (stage == 3)
            Unew[m] = (2.0 / 3.0) * U0[m] + (1.0 / 3.0) * (U[m] - 0.5 * dt * R[m]);
        else
            Unew[m] = U[m] - 0.5 * dt * R[m];
    }
}

/* Wall condition on the state: keep rho, the tangential momentum and rho e;
 * the momentum normal to the wall is set to zero. */
void orc_wall_project(double* U, double nx, double ny) {
    double tx = ny, ty = -nx;
    double ms = U[1] * tx + U[2] * ty;
    U[1] = ms * tx;
    U[2] = ms * ty;
}

/* residue = sqrt(sum_i R_rho,i^2) / N (serial sum in point order). */
double orc_residue(int64_t n, const double* R) {
    double s = 0.0;
    for (int64_t i = 0; i < n; ++i) s += R[4 * i] * R[4 * i];
    return sqrt(s) / (double)n;
}

/* Pressure force on the wall loop and the lift/drag coefficients. The loop
 * lists the wall points in order (closed: the last connects to the first). */
void orc_forces(const orc_cloud* c, const double* W, const int64_t* loop, int64_t m,
                double mach, double alpha_deg, double* cl, double* cd) {
    double p_inf = 1.0 / c->gamma;
    double fx = 0.0, fy = 0.0;
    for (int64_t k = 0; k < m; ++k) {
        int64_t i = loop[k];
        int64_t ip = loop[(k + 1) % m];
        int64_t im = loop[(k + m - 1) % m];
        double lp = sqrt((c->x[ip] - c->x[i]) * (c->x[ip] - c->x[i]) +
                         (c->y[ip] - c->y[i]) * (c->y[ip] - c->y[i]));
        double lm = sqrt((c->x[i] - c->x[im]) * (c->x[i] - c->x[im]) +
                         (c->y[i] - c->y[im]) * (c->y[i] - c->y[im]));
        double ds = 0.5 * (lp + lm);
        double dp = W[4 * i + 3] - p_inf;
        fx -= dp * c->nx[i] * ds;
        fy -= dp * c->ny[i] * ds;
    }
    double a = alpha_deg * ORC_PI / 180.0;
    double qinf = 0.5 * mach * mach;
    *cl = (-fx * sin(a) + fy * cos(a)) / qinf;
    *cd = (fx * cos(a) + fy * sin(a)) / qinf;
}

void orc_freestream(double gamma, double mach, double alpha_deg, double* W) {
    double a = alpha_deg * ORC_PI / 180.0;
    W[0] = 1.0;
    W[1] = mach * cos(a);
    W[2] = mach * sin(a);
    W[3] = 1.0 / gamma;
}

/* --------------------------------------------------------------- solver */

/* Algorithm 1: `iters` pseudo-time iterations from primitive state W (n x 4,
 * updated in place). Each iteration: timestep; four stages of q_variables,
 * q_derivatives, flux_residual, state_update(rk); residue. res[n_it] receives
 * the residue of each iteration (may be NULL). R1 (may be NULL) receives the
 * stage-1 residual of the last iteration. Returns 0, or the iteration number
 * (1-based) at which a non-positive density/pressure or a non-finite value
 * appeared. */
int orc_iterate(const orc_cloud* c, double* W, int iters, double cfl, int inner, double* res,
                double* R1) {
    int64_t n = c->n;
    double gamma = c->gamma;
    size_t sz = sizeof(double) * 4 * (size_t)n;
    double* U0 = (double*)malloc(sz);
    double* U = (double*)malloc(sz);
    double* q = (double*)malloc(sz);
    double* qx = (double*)malloc(sz);
    double* qy = (double*)malloc(sz);
    double* R = (double*)malloc(sz);
    double* dt = (double*)malloc(sizeof(double) * (size_t)n);
    int status = 0;
    for (int it = 0; it < iters && status == 0; ++it) {
        orc_timestep(c, W, cfl, dt);
        for (int64_t i = 0; i < n; ++i) orc_prim_to_cons(W + 4 * i, gamma, U0 + 4 * i);
        memcpy(U, U0, sz);
        double r = 0.0;
        for (int stage = 1; stage <= 4; ++stage) {
            for (int64_t i = 0; i < n; ++i) orc_prim_to_q(W + 4 * i, gamma, q + 4 * i);
            orc_q_derivatives(c, q, inner, qx, qy);
            orc_flux_residual(c, q, qx, qy, R);
            if (stage == 1) {
                r = orc_residue(n, R);
                if (R1 && it == iters - 1) memcpy(R1, R, sz);
            }
            for (int64_t i = 0; i < n; ++i) {
                double un[4];
                if (c->outer_mode == 1 && c->flag[i] == ORC_OUTER) continue;
                orc_rk_stage(stage, U0 + 4 * i, U + 4 * i, R + 4 * i, dt[i], un);
                if (c->flag[i] == ORC_WALL) orc_wall_project(un, c->nx[i], c->ny[i]);
                memcpy(U + 4 * i, un, sizeof(un));
                orc_cons_to_prim(un, gamma, W + 4 * i);
                const double* w = W + 4 * i;
                if (!(w[0] > 0.0) || !(w[3] > 0.0) || !isfinite(w[1]) || !isfinite(w[2]))
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
int orc_residual_of_state(const orc_cloud* c, const double* W, int inner, double* R) {
    int64_t n = c->n;
    size_t sz = sizeof(double) * 4 * (size_t)n;
    double* q = (double*)malloc(sz);
    double* qx = (double*)malloc(sz);
    double* qy = (double*)malloc(sz);
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
