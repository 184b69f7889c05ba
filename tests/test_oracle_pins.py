"""Pins of the CPU oracle to facts outside itself (no GPU needed).

Each test ties one oracle function to something the paper or the mathematics
fixes independently of the oracle's own code: half-range moments of the
Maxwellian computed by quadrature, the textbook entropy variables, library
least squares, exactness properties, the SSP-RK stability polynomial,
closed-form integrals and the method's invariants.
"""

import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2108_07031_gb300 import cloud as Cl

GAMMA = 1.4
RNG = np.random.Generator(np.random.PCG64(2108))


def random_states(n, rng=RNG):
    rho = rng.uniform(0.3, 2.5, n)
    u1 = rng.uniform(-1.5, 1.5, n)
    u2 = rng.uniform(-1.5, 1.5, n)
    p = rng.uniform(0.2, 2.0, n)
    return np.stack([rho, u1, u2, p], axis=1)


def euler_flux(W, direction):
    """Eq. 2: Gx (direction 0) or Gy (direction 1), written out from the paper."""
    rho, u1, u2, p = W.T
    rhoe = p / (GAMMA - 1.0) + 0.5 * rho * (u1 * u1 + u2 * u2)  # Eq. 3
    if direction == 0:
        return np.stack([rho * u1, p + rho * u1 * u1, rho * u1 * u2, (p + rhoe) * u1], axis=1)
    return np.stack([rho * u2, rho * u1 * u2, p + rho * u2 * u2, (p + rhoe) * u2], axis=1)


# --------------------------------------------------------------- split fluxes

def test_split_fluxes_add_up_to_euler_flux():
    """G+ + G- = G (the CIR split of Eq. 9 partitions velocity space)."""
    W = random_states(200)
    for d in (0, 1):
        Gp = O.split_flux(W, d, +1)
        Gm = O.split_flux(W, d, -1)
        G = euler_flux(W, d)
        scale = np.abs(G).max(axis=1, keepdims=True) + np.abs(Gp).max(axis=1, keepdims=True)
        assert np.all(np.abs(Gp + Gm - G) <= 8 * np.finfo(float).eps * scale)


def _half_range_moments(W, direction, sign):
    """Half-range moments <Psi, v_d F> over sign*v_d > 0 by quadrature.

    F is the Maxwellian of Eq. 5 read as rho/I0 (beta/pi) exp(-beta|v-u|^2 - I/I0)
    with the mean non-translational energy I0 = (2 - gamma)/(gamma - 1) / (2 beta);
    Psi is Eq. 6. The internal-energy integral is done in closed form (it only
    contributes I0 to the energy moment), the transverse velocity by
    Gauss-Hermite and the split velocity by adaptive quadrature.
    """
    from scipy import integrate

    rho, u1, u2, p = W
    beta = rho / (2.0 * p)
    I0 = (2.0 - GAMMA) / (GAMMA - 1.0) / (2.0 * beta)
    ua, ub = (u1, u2) if direction == 0 else (u2, u1)
    xh, wh = np.polynomial.hermite.hermgauss(40)
    vb = ub + xh / math.sqrt(beta)
    wb = wh / math.sqrt(math.pi)  # weights of the normalised transverse Gaussian

    def f1(va):
        return rho * math.sqrt(beta / math.pi) * math.exp(-beta * (va - ua) ** 2)

    def moment(k):
        def integrand(va):
            if k == 0:
                psi = 1.0
            elif k == 1:
                psi = va
            elif k == 2:
                psi = float(np.sum(wb * vb))
            else:
                psi = 0.5 * va * va + 0.5 * float(np.sum(wb * vb * vb)) + I0
            return va * psi * f1(va)
        lo, hi = (0.0, np.inf) if sign > 0 else (-np.inf, 0.0)
        val, _ = integrate.quad(integrand, lo, hi, epsabs=1e-14, epsrel=1e-13, limit=200)
        return val

    m = [moment(k) for k in range(4)]
    # order (mass, momentum along the split direction, transverse momentum, energy)
    if direction == 0:
        return np.array([m[0], m[1], m[2], m[3]])
    return np.array([m[0], m[2], m[1], m[3]])


@pytest.mark.parametrize("direction", [0, 1])
@pytest.mark.parametrize("sign", [+1, -1])
def test_split_flux_equals_half_range_moments(direction, sign):
    """Each split flux is the half-range moment of the Maxwellian (Eqs. 5-9)."""
    pytest.importorskip("scipy")
    W = random_states(6, np.random.Generator(np.random.PCG64(11 + direction + 3 * sign)))
    G = O.split_flux(W, direction, sign)
    for i in range(W.shape[0]):
        ref = _half_range_moments(W[i], direction, sign)
        assert np.allclose(G[i], ref, rtol=1e-9, atol=1e-11), (W[i], G[i], ref)


def test_split_flux_limits():
    """Hypersonic limits: G+ -> G and G- -> 0 for S >> 1, and the reverse."""
    W = np.array([[1.0, 30.0, 0.3, 0.5], [1.0, -30.0, 0.3, 0.5]])
    G = euler_flux(W, 0)
    Gp = O.split_flux(W, 0, +1)
    Gm = O.split_flux(W, 0, -1)
    assert np.allclose(Gp[0], G[0], rtol=1e-14) and np.all(np.abs(Gm[0]) < 1e-200)
    assert np.allclose(Gm[1], G[1], rtol=1e-14) and np.all(np.abs(Gp[1]) < 1e-200)


def test_split_flux_at_rest():
    """u = 0: mass flux +/- rho/(2 sqrt(pi beta)), momentum flux p/2."""
    W = np.array([[1.3, 0.0, 0.0, 0.9]])
    beta = 1.3 / 1.8
    Gp = O.split_flux(W, 0, +1)[0]
    assert Gp[0] == pytest.approx(1.3 / (2 * math.sqrt(math.pi * beta)), rel=1e-15)
    assert Gp[1] == pytest.approx(0.45, rel=1e-15)
    assert Gp[2] == 0.0


# ------------------------------------------------------------------ q-variables

def test_q_variables_are_entropy_variables():
    """Eq. 26 equals the textbook entropy variables dEta/dU (Eta = -rho s/(gamma-1),
    s = ln(p rho^-gamma)) up to a constant in the first component."""
    W = random_states(50)
    U = O.prim_to_cons(W)
    q = O.prim_to_q(W)

    def eta(Uc):
        rho = Uc[0]
        p = (GAMMA - 1.0) * (Uc[3] - 0.5 * (Uc[1] ** 2 + Uc[2] ** 2) / rho)
        s = np.log(p) - GAMMA * np.log(rho)
        return -rho * s / (GAMMA - 1.0)

    h = 1e-30
    for i in range(U.shape[0]):
        grad = np.empty(4)
        for k in range(4):
            Uc = U[i].astype(complex)
            Uc[k] += 1j * h
            grad[k] = eta(Uc).imag / h  # complex-step derivative, exact to rounding
        const = -(math.log(2.0) + GAMMA) / (GAMMA - 1.0)
        assert np.allclose(q[i], grad + np.array([const, 0, 0, 0]), rtol=1e-12, atol=1e-12)


def test_q_prim_cons_roundtrips():
    W = random_states(100)
    assert np.allclose(O.q_to_prim(O.prim_to_q(W)), W, rtol=1e-13, atol=1e-14)
    assert np.allclose(O.cons_to_prim(O.prim_to_cons(W)), W, rtol=1e-13, atol=1e-14)
    U = O.prim_to_cons(W)
    rho, u1, u2, p = W.T
    assert np.allclose(U[:, 3], p / (GAMMA - 1) + 0.5 * rho * (u1 ** 2 + u2 ** 2), rtol=1e-15)


def test_q_to_prim_rejects_nonpositive_temperature():
    W = O.q_to_prim(np.array([[0.1, 0.2, 0.3, 0.5]]))
    assert np.all(np.isnan(W))


# ------------------------------------------------------------- least squares

@pytest.fixture(scope="module")
def oc5k(cloud5k):
    return O.OracleCloud.from_cloud(cloud5k)


@pytest.mark.parametrize("weight_power", [0.0, 2.0])
def test_first_order_ls_exact_for_linear_fields(cloud5k, weight_power):
    """Eq. 11 (plain or distance-weighted) reproduces the gradient of any
    linear field exactly."""
    oc = O.OracleCloud.from_cloud(cloud5k, weight_power=weight_power)
    x, y = cloud5k.xy[:, 0], cloud5k.xy[:, 1]
    a, b, c = RNG.normal(size=(3, 4))
    q = a[None, :] + b[None, :] * x[:, None] + c[None, :] * y[:, None]
    qx, qy = O.q_derivatives(oc, q, 0)
    assert np.allclose(qx, np.broadcast_to(b, qx.shape), rtol=1e-8, atol=1e-8)
    assert np.allclose(qy, np.broadcast_to(c, qy.shape), rtol=1e-8, atol=1e-8)


def _row_scale(d, weight_power):
    """sqrt of the least-squares weight |d|^-p of each offset row: scaling the
    rows of a least-squares system by it gives the weighted normal equations."""
    return np.hypot(d[:, 0], d[:, 1]) ** (-0.5 * weight_power)


@pytest.mark.parametrize("weight_power", [0.0, 1.0, 2.0])
def test_first_order_ls_matches_library_lstsq(cloud5k, weight_power):
    """Eq. 11's 2x2 normal equations (optionally weighted by |P_j - P_i|^-p)
    equal numpy's least-squares solution of the row-scaled system."""
    oc = O.OracleCloud.from_cloud(cloud5k, weight_power=weight_power)
    q = RNG.normal(size=(cloud5k.n, 4))
    qx, qy = O.q_derivatives(oc, q, 0)
    for i in RNG.choice(cloud5k.n, 60, replace=False):
        nb = cloud5k.neighbours(i)
        A = cloud5k.xy[nb] - cloud5k.xy[i]
        r = _row_scale(A, weight_power)[:, None]
        sol, *_ = np.linalg.lstsq(r * A, r * (q[nb] - q[i]), rcond=None)
        assert np.allclose(sol[0], qx[i], rtol=1e-9, atol=1e-9 * np.abs(sol).max())
        assert np.allclose(sol[1], qy[i], rtol=1e-9, atol=1e-9 * np.abs(sol).max())


def test_weights_change_the_derivative_of_a_nonlinear_field(cloud5k, oc5k):
    """The weight option is live: for a field that is not linear the weighted
    and unweighted fits differ (and agree again for p = 0)."""
    q, _, _ = _quadratic(cloud5k, np.random.Generator(np.random.PCG64(8)))
    qx0, _ = O.q_derivatives(oc5k, q, 0)
    qx2, _ = O.q_derivatives(O.OracleCloud.from_cloud(cloud5k, weight_power=2.0), q, 0)
    qxz, _ = O.q_derivatives(O.OracleCloud.from_cloud(cloud5k, weight_power=0.0), q, 0)
    assert np.array_equal(qxz, qx0)
    assert np.abs(qx2 - qx0).max() > 1e-6 * np.abs(qx0).max()


def _quadratic(cloud, rng):
    x, y = cloud.xy[:, 0] - 0.5, cloud.xy[:, 1]
    co = rng.normal(size=(6, 4))
    q = (co[0] + co[1] * x[:, None] + co[2] * y[:, None] + co[3] * (x * x)[:, None]
         + co[4] * (x * y)[:, None] + co[5] * (y * y)[:, None])
    qx = co[1] + 2 * co[3] * x[:, None] + co[4] * y[:, None]
    qy = co[2] + co[4] * x[:, None] + 2 * co[5] * y[:, None]
    return q, qx, qy


@pytest.mark.parametrize("weight_power", [0.0, 2.0])
def test_defect_correction_is_exact_for_quadratics(cloud5k, oc5k, weight_power):
    """k-exactness for degree <= 2 (Section 2.1, after Eq. 23): fed the exact
    derivatives of a quadratic, one sweep of Eq. 29 returns them (with or
    without least-squares weights)."""
    q, qx, qy = _quadratic(cloud5k, np.random.Generator(np.random.PCG64(5)))
    if weight_power:
        oc5k = O.OracleCloud.from_cloud(cloud5k, weight_power=weight_power)
    nx, ny = O.ls_sweep(oc5k, q, qx, qy)
    scale = max(np.abs(qx).max(), np.abs(qy).max())
    assert np.abs(nx - qx).max() < 1e-9 * scale
    assert np.abs(ny - qy).max() < 1e-9 * scale
    # the first-order formula alone is not exact for a quadratic
    fx, _ = O.ls_sweep(oc5k, q)
    assert np.abs(fx - qx).max() > 1e-4 * scale


def test_inner_iterations_approach_exact_derivatives(cloud5k, oc5k):
    """Jacobi sweeps of Eq. 29 move the first-order derivatives towards the
    exact ones of a quadratic field (its fixed point)."""
    q, qx, qy = _quadratic(cloud5k, np.random.Generator(np.random.PCG64(6)))
    interior = (cloud5k.flags == 0) & (cloud5k.l > 2) & (cloud5k.l < 30)
    errs = []
    for inner in (0, 1, 2, 3):
        dx, _ = O.q_derivatives(oc5k, q, inner)
        errs.append(np.sqrt(np.mean((dx - qx)[interior] ** 2)))
    assert errs[1] < errs[0] and errs[2] < errs[1] and errs[3] < errs[2]


# ------------------------------------------------------------- flux residual

def test_uniform_state_gives_zero_residual(cloud5k, oc5k):
    """Free-stream preservation: every perturbation vanishes for a uniform state."""
    for mach, alpha in ((0.63, 2.0), (0.85, 1.0), (0.3, -4.0)):
        W = np.tile(O.freestream(mach, alpha), (cloud5k.n, 1))
        R, bad = O.residual_of_state(oc5k, W, inner=2)
        assert bad == 0
        assert np.all(R == 0.0)


def _smooth_field(x, y):
    rho = 1 + 0.1 * np.sin(x + 0.3) * np.cos(0.5 * y)
    u = 0.5 + 0.1 * np.cos(0.7 * x) * np.sin(y + 0.2)
    v = 0.1 + 0.1 * np.sin(0.4 * x + y)
    p = 1 / GAMMA + 0.05 * np.cos(x - 0.5 * y)
    return np.stack([rho, u, v, p], 1)


def _div_euler(x, y, field, h=1e-5):
    return ((euler_flux(field(x + h, y), 0) - euler_flux(field(x - h, y), 0)) / (2 * h)
            + (euler_flux(field(x, y + h), 1) - euler_flux(field(x, y - h), 1)) / (2 * h))


@pytest.mark.parametrize("order,inner,ratio", [(1, 0, 0.6), (2, 2, 0.7)])
def test_residual_is_consistent_with_euler_divergence(order, inner, ratio):
    """At interior points R -> dGx/dx + dGy/dy (Eqs. 1, 12) as the cloud is refined."""
    errs = []
    for n_c, n_r in ((128, 40), (256, 80), (512, 160)):
        c = Cl.naca0012_cloud(n_c, n_r)
        oc = O.OracleCloud.from_cloud(c, order=order)
        x, y = c.xy[:, 0], c.xy[:, 1]
        R, bad = O.residual_of_state(oc, _smooth_field(x, y), inner=inner)
        assert bad == 0
        m = (c.flags == 0) & (c.l > 2) & (c.l < n_r // 2)
        errs.append(np.abs(R - _div_euler(x, y, _smooth_field))[m].max())
    assert errs[1] < ratio * errs[0] and errs[2] < ratio * errs[1], errs
    if order == 2:
        assert errs[2] < 4e-3


def _flat_wall_cloud(nx, ny, seed=3):
    """Jittered rectangle [0, 1] x [0, 0.5]; bottom row is a wall (normal +y)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    h = 1.0 / (nx - 1)
    ii, jj = np.meshgrid(np.arange(nx), np.arange(ny))
    x = ii * h + rng.uniform(-0.1, 0.1, ii.shape) * h
    y = jj * h + rng.uniform(-0.1, 0.1, jj.shape) * h
    y[0, :] = 0.0
    x, y = x.ravel(), y.ravel()
    n = x.size
    flags = np.zeros(n, np.int8)
    flags[:nx] = 1
    normals = np.tile([0.0, 1.0], (n, 1))
    offs, idx = [0], []
    for p in range(n):
        i, j = p % nx, p // nx
        cand = [(jj2 * nx + ii2) for jj2 in range(max(0, j - 2), min(ny, j + 3))
                for ii2 in range(max(0, i - 2), min(nx, i + 3)) if (ii2, jj2) != (i, j)]
        cand = [c for c in cand if math.hypot(x[c] - x[p], y[c] - y[p]) < 1.6 * h]
        idx += cand
        offs.append(len(idx))
    xy = np.stack([x, y], 1)
    return xy, normals, flags, np.array(offs, np.int32), np.array(idx, np.int32)


def _mirror_field(x, y):
    rho = 1 + 0.1 * np.sin(2 * x) + 0.2 * y * y
    u = 0.5 + 0.1 * np.cos(x) * (1 + y * y)
    v = 0.3 * y * np.cos(x)
    p = 1 / GAMMA + 0.05 * np.cos(2 * x) + 0.1 * y * y
    return np.stack([rho, u, v, p], 1)


def test_kinetic_wall_is_consistent_for_mirror_symmetric_flow():
    """With specular reflection at a flat wall the reflected molecules add a
    second dGn-/dn for mass, tangential momentum and energy; with that factor 2
    the wall residual tends to the Euler divergence (the kinetic wall condition
    of Section 2.1, last paragraph), and without it it does not."""
    errs2, errs1 = [], []
    for nx in (41, 81, 161):
        xy, nrm, fl, off, idx = _flat_wall_cloud(nx, (nx - 1) // 2 + 1)
        x, y = xy[:, 0], xy[:, 1]
        W = _mirror_field(x, y)
        ex = _div_euler(x, y, _mirror_field)
        wall = (fl == 1) & (x > 0.2) & (x < 0.8)
        for fac, errs in ((2.0, errs2), (1.0, errs1)):
            oc = O.OracleCloud(xy, nrm, fl, off, idx, wall_factor=fac)
            R, bad = O.residual_of_state(oc, W, inner=2)
            errs.append(np.abs(R - ex)[wall][:, [0, 1, 3]].max())
    assert errs2[2] < 0.6 * errs2[0] and errs2[2] < 0.02, errs2
    assert errs1[2] > 0.05, errs1


@pytest.mark.parametrize("outer_mode,weight_power", [(1, 0.0), (0, 0.0), (1, 1.5)])
def test_residual_matches_lstsq_restatement(cloud5k, outer_mode, weight_power):
    """Point residuals re-assembled with library least squares per split stencil
    (Eq. 14 membership, Eq. 24 derivatives, frames and boundary readings;
    weighted rows when weight_power > 0)."""
    oc = O.OracleCloud.from_cloud(cloud5k, outer_mode=outer_mode, weight_power=weight_power)
    W = Cl.perturbed_state(cloud5k, 0.63, 2.0, amplitude=0.05)
    q = O.prim_to_q(W)
    qx, qy = O.q_derivatives(oc, q, 2)
    R, bad = O.flux_residual(oc, q, qx, qy)
    assert bad == 0
    pts = np.concatenate([np.arange(12), RNG.choice(cloud5k.n, 40, replace=False),
                          np.arange(cloud5k.n - 8, cloud5k.n)])
    for i in pts:
        f = cloud5k.flags[i]
        if f == 2 and outer_mode == 1:
            assert np.all(R[i] == 0.0)  # held at the free stream: not an unknown
            continue
        if f == 0:
            t, nn = np.array([1.0, 0.0]), np.array([0.0, 1.0])
        else:
            nn = cloud5k.normals[i]
            t = np.array([nn[1], -nn[0]])
        nb = cloud5k.neighbours(i)
        d = cloud5k.xy[nb] - cloud5k.xy[i]
        ds, dn = d @ t, d @ nn
        qtj = q[nb] - 0.5 * (d[:, :1] * qx[nb] + d[:, 1:] * qy[nb])
        qt0 = q[i][None, :] - 0.5 * (d[:, :1] * qx[i][None, :] + d[:, 1:] * qy[i][None, :])

        def local(Wg):
            return np.stack([Wg[:, 0], Wg[:, 1:3] @ t, Wg[:, 1:3] @ nn, Wg[:, 3]], 1)

        Lj, L0 = local(O.q_to_prim(qtj)), local(O.q_to_prim(qt0))
        stencils = [(ds < 0, 0, +1, 0), (ds > 0, 0, -1, 0)]
        if f != 1:
            stencils.append((dn < 0, 1, +1, 1))
        if f != 2:
            stencils.append((dn > 0, 1, -1, 1))
        Rl = np.zeros(4)
        for mask, direction, sign, comp in stencils:
            dG = O.split_flux(Lj[mask], direction, sign) - O.split_flux(L0[mask], direction, sign)
            A = np.stack([ds[mask], dn[mask]], 1)
            r = _row_scale(d[mask], weight_power)[:, None]
            sol, *_ = np.linalg.lstsq(r * A, r * dG, rcond=None)
            Rl += sol[comp] * (2.0 if (f == 1 and direction == 1) else 1.0)
        Rg = np.array([Rl[0], Rl[1] * t[0] + Rl[2] * nn[0], Rl[1] * t[1] + Rl[2] * nn[1], Rl[3]])
        assert np.allclose(R[i], Rg, rtol=1e-8, atol=1e-9 * np.abs(Rg).max()), (i, f, R[i], Rg)


# -------------------------------------------------------- time step, RK, wall

def test_timestep_worked_example():
    """dt = CFL min_j d_ij / (|u| + a) on a three-point cloud."""
    xy = np.array([[0.0, 0.0], [3.0, 4.0], [-1.0, 0.0]])
    oc = O.OracleCloud(xy, np.tile([0.0, 1.0], (3, 1)), np.zeros(3, np.int8),
                       np.array([0, 2, 3, 4], np.int32), np.array([1, 2, 0, 0], np.int32))
    W = np.array([[1.4, 0.3, 0.4, 1.0]] * 3)  # |u| = 0.5, a = 1
    dt = O.timestep(oc, W, 0.2)
    assert dt[0] == pytest.approx(0.2 * 1.0 / 1.5, rel=1e-15)
    assert dt[1] == pytest.approx(0.2 * 5.0 / 1.5, rel=1e-15)
    assert dt[2] == pytest.approx(0.2 * 1.0 / 1.5, rel=1e-15)


def test_ssp_rk_stability_polynomial():
    """Four-stage third-order SSP-RK (Section 2, after Eq. 14) applied to
    dU/dt = -lambda U has the amplification factor 1 + z + z^2/2 + z^3/6 + z^4/48."""
    for z in (-0.1, -0.7, -1.9, 0.3):
        lam_dt = -z
        U0 = np.array([1.0, -2.0, 0.5, 3.0])
        U = U0.copy()
        for stage in (1, 2, 3, 4):
            U = O.rk_stage(stage, U0, U, lam_dt * U, 1.0)
        amp = 1 + z + z * z / 2 + z ** 3 / 6 + z ** 4 / 48
        assert np.allclose(U, amp * U0, rtol=1e-14)


def test_wall_projection_removes_normal_momentum():
    ang = 0.37
    nx, ny = math.cos(ang), math.sin(ang)
    U = np.array([1.2, 0.4, -0.9, 2.5])
    P = O.wall_project(U, nx, ny)
    assert P[0] == U[0] and P[3] == U[3]
    assert abs(P[1] * nx + P[2] * ny) < 1e-16
    assert P[1] * ny - P[2] * nx == pytest.approx(U[1] * ny - U[2] * nx, rel=1e-15)


def test_residue_worked_example():
    R = np.array([[3.0, 9, 9, 9], [4.0, 9, 9, 9]])
    assert O.residue(R) == 2.5


def test_forces_closed_form_on_circle():
    """p = p_inf + c y on a circle of radius a: F = -c (0, pi a^2) (divergence
    theorem), so Cl = -c pi a^2 / q_inf at alpha = 0, and rotating alpha
    rotates (Cd, Cl)."""
    m, a, c, mach = 4000, 0.5, 0.3, 0.6
    th = 2 * np.pi * np.arange(m) / m
    xy = np.stack([a * np.cos(th), a * np.sin(th)], 1)
    nrm = np.stack([np.cos(th), np.sin(th)], 1)
    flags = np.ones(m, np.int8)
    off = np.zeros(m + 1, np.int32)
    oc = O.OracleCloud(xy, nrm, flags, off, np.zeros(0, np.int32))
    W = np.zeros((m, 4))
    W[:, 0] = 1.0
    W[:, 3] = 1 / GAMMA + c * xy[:, 1]
    cl, cd = O.forces(oc, W, np.arange(m), mach, 0.0)
    assert cl == pytest.approx(-c * math.pi * a * a / (0.5 * mach * mach), rel=1e-5)
    assert abs(cd) < 1e-12
    cl2, cd2 = O.forces(oc, W, np.arange(m), mach, 30.0)
    r = math.radians(30.0)
    assert cl2 == pytest.approx(cl * math.cos(r), rel=1e-12)
    assert cd2 == pytest.approx(cl * math.sin(r), rel=1e-12)


def test_freestream_definition():
    W = O.freestream(0.63, 2.0)
    assert W[0] == 1.0 and W[3] == pytest.approx(1 / GAMMA)
    assert math.hypot(W[1], W[2]) == pytest.approx(0.63, rel=1e-15)
    assert math.degrees(math.atan2(W[2], W[1])) == pytest.approx(2.0, rel=1e-13)


# --------------------------------------------------------------- whole solver

def test_symmetric_cloud_gives_symmetric_flow():
    """Mirror-symmetric cloud at alpha = 0: rho, p even and v odd about y = 0,
    zero lift, after 100 iterations of Algorithm 1."""
    c = Cl.naca0012_cloud(128, 40, symmetric=True)
    oc = O.OracleCloud.from_cloud(c)
    W0 = np.tile(O.freestream(0.63, 0.0), (c.n, 1))
    W, res, st = O.iterate(oc, W0, 100)
    assert st == 0
    mirror = c.l * c.n_c + (c.n_c - c.k) % c.n_c
    assert np.allclose(W[:, 0], W[mirror, 0], rtol=0, atol=1e-12)
    assert np.allclose(W[:, 3], W[mirror, 3], rtol=0, atol=1e-12)
    assert np.allclose(W[:, 1], W[mirror, 1], rtol=0, atol=1e-12)
    assert np.allclose(W[:, 2], -W[mirror, 2], rtol=0, atol=1e-12)
    cl, cd = O.forces(oc, W, c.wall_loop, 0.63, 0.0)
    assert abs(cl) < 1e-11


def test_residue_decays_on_5k_cloud(cloud5k, oc5k):
    """Pseudo-time iterations from free stream damp the residue (Algorithm 1)."""
    W0 = np.tile(O.freestream(0.63, 2.0), (cloud5k.n, 1))
    W, res, st = O.iterate(oc5k, W0, 600)
    assert st == 0
    assert res[0] == 0.0  # a uniform state has zero residual
    assert res[-1] < 0.35 * res[1:20].max()
    assert np.all(np.isfinite(W)) and np.all(W[:, 0] > 0) and np.all(W[:, 3] > 0)


# ------------------------------------------------------- regression guard

def test_oracle_matches_its_stored_regression_values():
    """The oracle's results on a small seeded case equal the values stored by
    tests/golden/make_oracle_regression.py (a guard against accidental
    changes of its arithmetic; libm may differ by an ulp across machines,
    which the split-flux differences amplify to ~1e-13)."""
    import json
    import os
    import sys
    here = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
    sys.path.insert(0, here)
    import make_oracle_regression as G
    with open(os.path.join(here, "oracle_regression.json")) as f:
        ref = json.load(f)
    now = G.compute()
    R, R_ref = np.array(now["residual_of_perturbed_state"]), np.array(ref["residual_of_perturbed_state"])
    assert np.abs(R - R_ref).max() <= 1e-10 * np.abs(R_ref).max()
    a, b = now["iterate_50_from_freestream"], ref["iterate_50_from_freestream"]
    assert a["status"] == b["status"] == 0
    W, W_ref = np.array(a["state"]), np.array(b["state"])
    assert np.abs(W - W_ref).max() <= 1e-10 * np.abs(W_ref).max()
    assert abs(a["cl"] - b["cl"]) <= 1e-10 and abs(a["cd"] - b["cd"]) <= 1e-10
    assert np.allclose(a["residue"], b["residue"], rtol=1e-9, atol=0)
