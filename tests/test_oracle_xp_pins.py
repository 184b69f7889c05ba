"""Pins of the oracle's binary128 build, the extended-precision reference.

The binary128 build runs the FP64 oracle's source (whose formulas the pins in
test_oracle_pins.py tie to the paper and the mathematics) with every value
carried in IEEE binary128. What these tests pin is that it really delivers
that precision -- a double literal, a double libm call or a lost low part
anywhere would cap it near 1e-16 -- against computations outside the oracle:
half-range moments of the Maxwellian by mpmath quadrature at 40 digits, the
entropy variables by mpmath differentiation, exactness for linear and
quadratic fields at binary128 level, and point residuals re-assembled in
40-digit arithmetic with mpmath's own least-squares solver. They also pin the
sub-cloud evaluation that makes the reference affordable on large clouds:
in FP64 it equals the whole-cloud evaluation bit for bit.
"""

import numpy as np
import pytest

from oracle import oracle as O
from paper_2108_07031_gb300 import cloud as Cl

mp = pytest.importorskip("mpmath")

GAMMA = 1.4


@pytest.fixture(scope="module")
def small():
    return Cl.naca0012_cloud(64, 24, shuffle=True, seed=5)


def _split_exact(vals):
    """mpmath values -> (hi, lo) doubles with hi + lo equal to them to ~1e-32."""
    flat = [mp.mpf(v) for v in np.ravel(vals)]
    hi = np.array([float(v) for v in flat])
    lo = np.array([float(v - mp.mpf(h)) for v, h in zip(flat, hi)])
    return hi.reshape(np.shape(vals)), lo.reshape(np.shape(vals))


def _to_mp(hi, lo):
    return mp.mpf(float(hi)) + mp.mpf(float(lo))


# -------------------------------------------------- the sub-cloud evaluation

@pytest.mark.parametrize("inner,opts", [(2, {}), (0, {}), (3, {"weight_power": 1.5}),
                                        (2, {"outer_mode": 0, "wall_factor": 1.0}),
                                        (0, {"order": 1})])
def test_fp64_subcloud_evaluation_equals_whole_cloud(small, inner, opts):
    """R and the q-derivatives at sampled points from their (inner + 2)-hop
    neighbourhood equal the whole-cloud evaluation bit for bit."""
    oc = O.OracleCloud.from_cloud(small, **opts)
    W = Cl.perturbed_state(small, 0.7, 1.5)
    idx = np.concatenate([np.arange(10), np.random.default_rng(2).choice(small.n, 150, replace=False),
                          np.flatnonzero(small.flags == 2)[:10]])
    R, bad = O.residual_of_state(oc, W, inner=inner)
    assert bad == 0
    qx, qy = O.q_derivatives(oc, O.prim_to_q(W), inner)
    got = O.residual_at(oc, W, idx, inner, quad=False)
    assert got["bad"] == 0
    assert np.array_equal(got["R"][0], R[idx]) and not np.any(got["R"][1])
    assert np.array_equal(got["qx"][0], qx[idx]) and np.array_equal(got["qy"][0], qy[idx])


def test_subcloud_rings(small):
    """Hop rings: the seeds at 0, their neighbours at 1, and so on; every point
    inside the outermost ring keeps its whole stencil."""
    oc = O.OracleCloud.from_cloud(small)
    seeds = np.array([3, 500, 1200])
    level = oc.neighbourhood(seeds, 3)
    assert np.all(level[seeds] == 0)
    for i in range(small.n):
        if 0 <= level[i] < 3:
            nb = small.neighbours(i)
            assert np.all((level[nb] >= 0) & (level[nb] <= level[i] + 1))
    sub, members, loc = oc.subcloud(seeds, 3)
    assert np.array_equal(members[loc], seeds)
    for k, g in enumerate(members):
        if level[g] < 3:
            assert np.array_equal(members[sub.nbr[sub.off[k]:sub.off[k + 1]]], small.neighbours(g))


# ------------------------------------------------------ pointwise maps at 40 digits

def test_quad_split_flux_equals_half_range_moments():
    """Split fluxes (binary128) against the half-range moments of the
    Maxwellian (Eqs. 5-9) integrated by mpmath at 40 digits; the transverse
    velocity and internal energy moments are the Gaussian's closed forms."""
    mp.mp.dps = 40
    rng = np.random.Generator(np.random.PCG64(17))
    W = np.stack([rng.uniform(0.4, 2.0, 4), rng.uniform(-1.2, 1.2, 4), rng.uniform(-1.2, 1.2, 4),
                  rng.uniform(0.3, 1.5, 4)], 1)
    g = mp.mpf(GAMMA)
    for direction in (0, 1):
        for sign in (+1, -1):
            hi, lo = O.split_flux_real(W, direction, sign, quad=True)
            for i in range(W.shape[0]):
                rho, u1, u2, p = (mp.mpf(float(v)) for v in W[i])
                beta = rho / (2 * p)
                I0 = (2 - g) / (g - 1) / (2 * beta)
                ua, ub = (u1, u2) if direction == 0 else (u2, u1)
                f1 = lambda v: rho * mp.sqrt(beta / mp.pi) * mp.exp(-beta * (v - ua) ** 2)
                rng_v = [0, mp.inf] if sign > 0 else [-mp.inf, 0]
                m0 = mp.quad(lambda v: v * f1(v), rng_v)
                m1 = mp.quad(lambda v: v * v * f1(v), rng_v)
                m3 = mp.quad(lambda v: v * (v * v / 2 + (ub * ub + 1 / (2 * beta)) / 2 + I0) * f1(v),
                             rng_v)
                ref = [m0, m1, ub * m0, m3] if direction == 0 else [m0, ub * m0, m1, m3]
                scale = max(abs(r) for r in ref)
                for k in range(4):
                    err = abs(_to_mp(hi[i, k], lo[i, k]) - ref[k]) / scale
                    assert err < 1e-29, (direction, sign, i, k, err)


def test_quad_q_variables_are_entropy_variables():
    """Eq. 26 in binary128 equals dEta/dU (Eta = -rho s/(gamma - 1)) computed
    by mpmath's numerical differentiation at 40 digits, up to the constant."""
    mp.mp.dps = 40
    rng = np.random.Generator(np.random.PCG64(19))
    W = np.stack([rng.uniform(0.4, 2.0, 5), rng.uniform(-1, 1, 5), rng.uniform(-1, 1, 5),
                  rng.uniform(0.3, 1.5, 5)], 1)
    hi, lo = O.prim_to_q_real(W, quad=True)
    g = mp.mpf(GAMMA)
    for i in range(W.shape[0]):
        rho, u1, u2, p = (mp.mpf(float(v)) for v in W[i])
        U = [rho, rho * u1, rho * u2, p / (g - 1) + rho * (u1 * u1 + u2 * u2) / 2]

        def eta(*Uc):
            pr = (g - 1) * (Uc[3] - (Uc[1] ** 2 + Uc[2] ** 2) / (2 * Uc[0]))
            return -Uc[0] * (mp.log(pr) - g * mp.log(Uc[0])) / (g - 1)

        const = -(mp.log(2) + g) / (g - 1)
        for k in range(4):
            order = [0, 0, 0, 0]
            order[k] = 1
            ref = mp.diff(eta, U, tuple(order)) + (const if k == 0 else 0)
            assert abs(_to_mp(hi[i, k], lo[i, k]) - ref) < 1e-30 * max(1, abs(ref))


def test_quad_state_map_round_trip():
    rng = np.random.Generator(np.random.PCG64(23))
    W = np.stack([rng.uniform(0.4, 2.0, 50), rng.uniform(-1, 1, 50), rng.uniform(-1, 1, 50),
                  rng.uniform(0.3, 1.5, 50)], 1)
    qh, ql = O.prim_to_q_real(W, quad=True)
    Wh, Wl = O.q_to_prim_real(qh, ql, quad=True)
    err = np.abs((Wh - W) + Wl) / np.abs(W)
    assert err.max() < 1e-31


# ------------------------------------------------ least squares at binary128 level

def _poly_field(cloud, degree, seed):
    """A random polynomial field of the given degree, its value as (hi, lo)
    (exact to ~1e-32) and its exact derivatives."""
    mp.mp.dps = 40
    rng = np.random.Generator(np.random.PCG64(seed))
    co = rng.normal(size=(6, 4))
    vals, dx, dy = [], [], []
    for (x, y) in cloud.xy:
        X, Y = mp.mpf(float(x)) - mp.mpf("0.5"), mp.mpf(float(y))
        mons = [1, X, Y, X * X, X * Y, Y * Y][: 3 if degree == 1 else 6]
        dmx = [0, 1, 0, 2 * X, Y, 0][: len(mons)]
        dmy = [0, 0, 1, 0, X, 2 * Y][: len(mons)]
        vals.append([mp.fsum(co[m, c] * mons[m] for m in range(len(mons))) for c in range(4)])
        dx.append([mp.fsum(co[m, c] * dmx[m] for m in range(len(mons))) for c in range(4)])
        dy.append([mp.fsum(co[m, c] * dmy[m] for m in range(len(mons))) for c in range(4)])
    return _split_exact(vals), _split_exact(dx), _split_exact(dy)


def test_quad_first_order_ls_is_exact_for_linear_fields(small):
    """Eq. 11 in binary128 returns a linear field's gradient to ~1e-28 (the
    FP64 build only to ~1e-12 of it)."""
    oc = O.OracleCloud.from_cloud(small)
    q, gx, gy = _poly_field(small, 1, 29)
    (qxh, qxl), (qyh, qyl) = O.q_derivatives_real(oc, q[0], q[1], inner=0, quad=True)
    assert np.abs((qxh - gx[0]) + (qxl - gx[1])).max() < 1e-26 * np.abs(gx[0]).max()
    assert np.abs((qyh - gy[0]) + (qyl - gy[1])).max() < 1e-26 * np.abs(gy[0]).max()
    (fx, _), _ = O.q_derivatives_real(oc, q[0], q[1], inner=0, quad=False)
    assert np.abs(fx - gx[0]).max() > 1e-20 * np.abs(gx[0]).max()


def test_quad_defect_correction_is_exact_for_quadratics(small):
    """k-exactness (degree <= 2, Section 2.1 after Eq. 23) at binary128 level:
    fed a quadratic's exact derivatives, one sweep of Eq. 29 returns them."""
    oc = O.OracleCloud.from_cloud(small)
    q, gx, gy = _poly_field(small, 2, 31)
    (nxh, nxl), (nyh, nyl) = O.ls_sweep_real(oc, q, gx, gy, quad=True)
    scale = max(np.abs(gx[0]).max(), np.abs(gy[0]).max())
    assert np.abs((nxh - gx[0]) + (nxl - gx[1])).max() < 1e-25 * scale
    assert np.abs((nyh - gy[0]) + (nyl - gy[1])).max() < 1e-25 * scale


def test_quad_uniform_state_gives_zero_residual(small):
    oc = O.OracleCloud.from_cloud(small)
    W = np.tile(O.freestream(0.85, 1.0), (small.n, 1))
    got = O.residual_at(oc, W, np.arange(small.n), 2, quad=True)
    assert got["bad"] == 0
    assert not np.any(got["R"][0]) and not np.any(got["R"][1])


# -------------------------------------- residuals re-assembled in 40 digits

def _mp_residual(cloud, W, i, inner, wall_factor=2.0):
    """R_i in 40-digit arithmetic: Eq. 26, then least squares (mpmath's QR
    solver, not the normal equations) for Eq. 11 and the inner sweeps of
    Eqs. 28-29 on the points the result depends on, then the split-flux
    derivatives of Eq. 24 over the split stencils of Eq. 14 in the point's
    frame, with the wall and held far-field readings."""
    mp.mp.dps = 40
    g = mp.mpf(GAMMA)
    oc = O.OracleCloud.from_cloud(cloud)
    level = oc.neighbourhood([i], inner + 2)
    pts = np.flatnonzero(level >= 0)
    X = {int(p): (mp.mpf(float(cloud.xy[p, 0])), mp.mpf(float(cloud.xy[p, 1]))) for p in pts}

    def q_of(w):
        rho, u1, u2, p = (mp.mpf(float(v)) for v in w)
        beta = rho / (2 * p)
        return [mp.log(rho) + mp.log(beta) / (g - 1) - beta * (u1 * u1 + u2 * u2),
                2 * beta * u1, 2 * beta * u2, -2 * beta]

    def prim_of(q):
        beta = -q[3] / 2
        u1, u2 = q[1] / (2 * beta), q[2] / (2 * beta)
        rho = mp.exp(q[0] - mp.log(beta) / (g - 1) + beta * (u1 * u1 + u2 * u2))
        return [rho, u1, u2, rho / (2 * beta)]

    q = {int(p): q_of(W[p]) for p in pts}

    def lsq(rows, rhs):
        A = mp.matrix(rows)
        return [mp.qr_solve(A, mp.matrix(col))[0] for col in zip(*rhs)]

    def sweep(prev, ring):
        out = {}
        for p in pts[level[pts] <= ring]:
            p = int(p)
            rows, rhs = [], []
            for j in cloud.neighbours(p):
                j = int(j)
                dx, dy = X[j][0] - X[p][0], X[j][1] - X[p][1]
                rows.append([dx, dy])
                if prev is None:
                    rhs.append([q[j][m] - q[p][m] for m in range(4)])
                else:
                    rhs.append([(q[j][m] - q[p][m]) - (dx * (prev[j][0][m] - prev[p][0][m])
                                                      + dy * (prev[j][1][m] - prev[p][1][m])) / 2
                                for m in range(4)])
            sol = lsq(rows, rhs)
            out[p] = ([sol[m][0] for m in range(4)], [sol[m][1] for m in range(4)])
        return out

    d = sweep(None, inner + 1)
    for k in range(1, inner + 1):
        d = sweep(d, inner + 1 - k)

    def flux(L, direction, sign):
        rho, p = L[0], L[3]
        ua, ub = (L[1], L[2]) if direction == 0 else (L[2], L[1])
        beta = rho / (2 * p)
        S = ua * mp.sqrt(beta)
        A = mp.erfc(-sign * S) / 2
        B = mp.exp(-S * S) / (2 * mp.sqrt(mp.pi * beta))
        rhoe = p / (g - 1) + rho * (ua * ua + ub * ub) / 2
        ga = (p + rho * ua * ua) * A + sign * rho * ua * B
        gb = rho * ub * (ua * A + sign * B)
        G = [rho * (ua * A + sign * B), ga if direction == 0 else gb,
             gb if direction == 0 else ga, (p + rhoe) * ua * A + sign * (rhoe + p / 2) * B]
        return G

    f = int(cloud.flags[i])
    if f == 2:
        return [mp.mpf(0)] * 4, d[i]
    if f == 0:
        t, n = (mp.mpf(1), mp.mpf(0)), (mp.mpf(0), mp.mpf(1))
    else:
        n = (mp.mpf(float(cloud.normals[i, 0])), mp.mpf(float(cloud.normals[i, 1])))
        t = (n[1], -n[0])
    members = {0: [], 1: [], 2: [], 3: []}
    for j in cloud.neighbours(i):
        j = int(j)
        dx, dy = X[j][0] - X[i][0], X[j][1] - X[i][1]
        ds, dn = dx * t[0] + dy * t[1], dx * n[0] + dy * n[1]
        Wt = [prim_of([q[a][m] - (dx * d[a][0][m] + dy * d[a][1][m]) / 2 for m in range(4)])
              for a in (j, i)]
        Ls = [[w[0], w[1] * t[0] + w[2] * t[1], w[1] * n[0] + w[2] * n[1], w[3]] for w in Wt]
        if ds != 0:
            members[0 if ds < 0 else 1].append((ds, dn, Ls))
        if dn != 0:
            members[2 if dn < 0 else 3].append((ds, dn, Ls))
    use = [0, 1] + ([] if f == 1 else [2]) + [3]
    Rl = [mp.mpf(0)] * 4
    for sl in use:
        direction, sign = (0 if sl < 2 else 1), (1 if sl in (0, 2) else -1)
        rows = [[ds, dn] for ds, dn, _ in members[sl]]
        rhs = [[a - b for a, b in zip(flux(Ls[0], direction, sign), flux(Ls[1], direction, sign))]
               for _, _, Ls in members[sl]]
        sol = lsq(rows, rhs)
        fac = wall_factor if (f == 1 and sl == 3) else 1
        for m in range(4):
            Rl[m] += fac * sol[m][direction]
    R = [Rl[0], Rl[1] * t[0] + Rl[2] * n[0], Rl[1] * t[1] + Rl[2] * n[1], Rl[3]]
    return R, d[i]


def test_quad_residual_matches_40_digit_reassembly(small):
    """Point residuals and q-derivatives of the binary128 build against the
    40-digit re-assembly (wall, interior and far-field-adjacent points); the
    FP64 build is ~1e-13 away, the binary128 build ~1e-28."""
    oc = O.OracleCloud.from_cloud(small)
    W = Cl.perturbed_state(small, 0.7, 1.5)
    lay = small.l
    pts = [0, 5, int(np.flatnonzero(lay == 1)[3]), int(np.flatnonzero(lay == 11)[7]),
           int(np.flatnonzero(lay == small.n_r - 2)[2])]
    got = O.residual_at(oc, W, pts, 2, quad=True)
    f64 = O.residual_at(oc, W, pts, 2, quad=False)
    worst64 = 0.0
    for k, i in enumerate(pts):
        R, (qx, qy) = _mp_residual(small, W, i, 2)
        scale = max(abs(r) for r in R)
        for m in range(4):
            err = abs(_to_mp(got["R"][0][k, m], got["R"][1][k, m]) - R[m]) / scale
            assert err < 1e-27, (i, m, err)
            worst64 = max(worst64, float(abs(mp.mpf(float(f64["R"][0][k, m])) - R[m]) / scale))
            for name, ref in (("qx", qx[m]), ("qy", qy[m])):
                e = abs(_to_mp(got[name][0][k, m], got[name][1][k, m]) - ref)
                assert e < 1e-27 * max(1, abs(ref)), (i, name, m, e)
    assert 1e-18 < worst64 < 1e-11  # FP64 rounding is visible against the reference
