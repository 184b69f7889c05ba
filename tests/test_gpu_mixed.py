"""GPU parity of the mixed-precision path (precision = LSKUM_MIXED) against the
FP64 oracle.

The mixed path does the stencil, least-squares and split-flux arithmetic in
FP32, in difference form on q stored as float pairs, and keeps FP64 for the
state accumulation, q-variables, determinants, residue and forces. Its error
is FP32 rounding relative to the residual itself (2^-24 ~ 6e-8 per
operation, a few hundred operations per neighbour through sums of ~14 terms):
the bound used here is 2e-5 norm-wise on one residual evaluation, and the
target 1e-4 on Cl/Cd after 1000 iterations.
"""

import numpy as np
import pytest

from oracle import oracle as O
from paper_2108_07031_gb300 import cloud as Cl

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2108_07031_gb300 import lskum as L  # noqa: E402

TOL_MIXED = 2e-5


def normwise(a, b):
    scale = np.abs(b).max(axis=0)
    scale = np.where(scale > 0, scale, 1.0)
    return float((np.abs(np.asarray(a) - b).max(axis=0) / scale).max())


@pytest.fixture(scope="module")
def c_ragged():
    return Cl.naca0012_cloud(130, 41, shuffle=True, seed=99)


@pytest.fixture(scope="module")
def c5k():
    return Cl.naca0012_cloud(128, 40)


def test_mixed_q_derivatives_and_residual(c_ragged):
    W = Cl.perturbed_state(c_ragged, 0.63, 2.0)
    oc = O.OracleCloud.from_cloud(c_ragged)
    q = O.prim_to_q(W)
    qx_o, qy_o = O.q_derivatives(oc, q, 2)
    R_o, _ = O.flux_residual(oc, q, qx_o, qy_o)
    with L.Solver.from_cloud(c_ragged, precision=L.MIXED) as s:
        s.set_state(W)
        qx, qy = s.eval_q_derivatives()
        R = s.eval_residual()
    e_qx, e_qy, e_r = normwise(qx, qx_o), normwise(qy, qy_o), normwise(R, R_o)
    print(f"mixed vs oracle: qx {e_qx:.2e} qy {e_qy:.2e} R {e_r:.2e}")
    assert e_qx < TOL_MIXED and e_qy < TOL_MIXED and e_r < TOL_MIXED


def test_mixed_uniform_state_zero_residual(c_ragged):
    with L.Solver.from_cloud(c_ragged, precision=L.MIXED) as s:
        s.set_freestream(0.85, 1.0)
        assert np.all(s.eval_residual() == 0.0)


@pytest.mark.parametrize("opts", [dict(order=1, inner_iters=0), dict(outer_mode=0),
                                  dict(block_size=256), dict(inner_iters=3),
                                  dict(weight_power=2.0)])
def test_mixed_option_variants(c_ragged, opts):
    ok = {k: v for k, v in opts.items() if k in ("order", "outer_mode", "weight_power")}
    oc = O.OracleCloud.from_cloud(c_ragged, **ok)
    W = Cl.perturbed_state(c_ragged, 0.85, 1.0)
    R_o, _ = O.residual_of_state(oc, W, inner=opts.get("inner_iters", 2))
    with L.Solver.from_cloud(c_ragged, precision=L.MIXED, **opts) as s:
        s.set_state(W)
        R = s.eval_residual()
    assert normwise(R, R_o) < TOL_MIXED


def test_mixed_1000_iterations_cl_cd(c5k):
    """1000 iterations from the free stream at M 0.63, alpha 2: state, residue
    and Cl/Cd against the FP64 oracle (Cl/Cd within 1e-4)."""
    oc = O.OracleCloud.from_cloud(c5k)
    W0 = np.tile(O.freestream(0.63, 2.0), (c5k.n, 1))
    W_o, res_o, st = O.iterate(oc, W0, 1000)
    assert st == 0
    with L.Solver.from_cloud(c5k, precision=L.MIXED) as s:
        s.set_freestream(0.63, 2.0)
        s.step(1000)
        W = s.get_state()
        r = s.residual_norm()
        cl, cd = s.forces()
    cl_o, cd_o = O.forces(oc, W_o, c5k.wall_loop, 0.63, 2.0)
    e_w = normwise(W, W_o)
    print(f"mixed 1000 it: state {e_w:.2e}, residue {r:.4e} vs {res_o[-1]:.4e}, "
          f"Cl {cl:.6f} vs {cl_o:.6f}, Cd {cd:.6f} vs {cd_o:.6f}")
    assert e_w < 1e-4
    assert abs(cl - cl_o) < 1e-4 and abs(cd - cd_o) < 1e-4
    assert abs(r - res_o[-1]) < 1e-2 * res_o[-1]


def test_mixed_full_size_sampled():
    """10M points (the benchmark's cloud and launch configuration), residual at
    ~2200 sampled points against the oracle."""
    n_c, n_r = Cl.cloud_dims(10_000_000)
    c = Cl.naca0012_cloud(n_c, n_r, shuffle=True)
    W = Cl.perturbed_state(c, 0.63, 2.0)
    with L.Solver.from_cloud(c, precision=L.MIXED) as s:
        s.set_state(W)
        R = s.eval_residual()
    oc = O.OracleCloud.from_cloud(c)
    q = O.prim_to_q(W)
    qx_o, qy_o = O.q_derivatives(oc, q, 2)
    rng = np.random.Generator(np.random.PCG64(5))
    idx = np.concatenate([np.arange(n_c), rng.choice(c.n, 2000, replace=False)])
    R_o, bad = O.flux_residual_subset(oc, q, qx_o, qy_o, idx)
    e = normwise(R[idx], R_o)
    print(f"mixed full-size sampled residual: {e:.2e}")
    assert e < TOL_MIXED
