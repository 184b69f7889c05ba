"""Batched solves: several free streams on one cloud (n_conditions, condition-
innermost layout) and ragged batches of packed clouds, against independent
single-condition solves and the oracle; and the block-size autotuner."""

import numpy as np
import pytest

from oracle import oracle as O
from paper_2108_07031_gb300 import cloud as Cl
from parity_utils import describe, exact_errors, normwise

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2108_07031_gb300 import lskum as L  # noqa: E402


@pytest.fixture(scope="module")
def cloud():
    return Cl.naca0012_cloud(130, 41, shuffle=True, seed=99)


def _check_residual(oc, W, R, inner=2):
    """One condition's FP64 residual: per component, at most twice the FP64
    oracle's own 2-norm distance from the binary128 reference."""
    errs = exact_errors(oc, W, {"R": R}, inner=inner)
    print(describe(errs))
    assert np.all(errs["R"]["gpu_rms"] <= 2.0 * errs["R"]["oracle_rms"])


@pytest.mark.parametrize("precision", [L.FP64, L.MIXED])
def test_conditions_equal_independent_solves(cloud, precision):
    """Each condition of a batch evolves exactly (bitwise) as a solve of its own:
    the per-(point, condition) arithmetic is the same code; only the residue's
    summation order differs."""
    mach, alpha = Cl.conditions(4)
    with L.Solver.from_cloud(cloud, precision=precision, n_conditions=4) as b:
        b.set_conditions(mach, alpha)
        b.step(15)
        Wb = b.get_state()
        rb = b.residual_norm()
        clb, cdb = b.forces()
    for k in range(4):
        with L.Solver.from_cloud(cloud, precision=precision) as s:
            s.set_freestream(mach[k], alpha[k])
            s.step(15)
            assert np.array_equal(Wb[k], s.get_state())
            assert abs(rb[k] - s.residual_norm()) <= 1e-13 * s.residual_norm()
            cl, cd = s.forces()
            assert abs(clb[k] - cl) <= 1e-12 * max(1.0, abs(cl))
            assert abs(cdb[k] - cd) <= 1e-12 * max(1.0, abs(cd))


def test_64_conditions_against_oracle(cloud):
    """64 seeded conditions (M ~ U[0.3, 0.8], alpha ~ U[-4, 6] deg) in FP64:
    two of them checked against the oracle after 5 iterations."""
    mach, alpha = Cl.conditions(64)
    with L.Solver.from_cloud(cloud, n_conditions=64) as b:
        b.set_conditions(mach, alpha)
        b.step(5)
        Wb = b.get_state()
        rb = b.residual_norm()
    oc = O.OracleCloud.from_cloud(cloud)
    for k in (3, 41):
        W0 = np.tile(O.freestream(mach[k], alpha[k]), (cloud.n, 1))
        W5, res, st = O.iterate(oc, W0, 5)
        assert st == 0
        scale = np.abs(W5).max(axis=0)
        assert np.all(np.abs(Wb[k] - W5).max(axis=0) <= 1e-12 * scale)
        assert abs(rb[k] - res[-1]) <= 1e-11 * res[-1]


def test_set_state_and_residual_layout(cloud):
    """Host arrays are condition-major: [condition][point][4]."""
    W = np.stack([Cl.perturbed_state(cloud, 0.5, 1.0, seed=s) for s in (1, 2)])
    with L.Solver.from_cloud(cloud, n_conditions=2) as b:
        b.set_state(W)
        R = b.eval_residual()
    oc = O.OracleCloud.from_cloud(cloud)
    for k in range(2):
        _check_residual(oc, W[k], R[k])


@pytest.mark.parametrize("opts", [dict(weight_power=1.5, inner_iters=3),
                                  dict(order=1, inner_iters=0), dict(outer_mode=0)])
def test_batched_option_variants_against_oracle(cloud, opts):
    """Options apply to every condition of a batch: 4 conditions with
    least-squares weights / first-order LSKUM / the kinetic far field, the
    residual of each developed state against the oracle with the same
    options, then 3 iterations."""
    ok = {k: v for k, v in opts.items() if k in ("order", "outer_mode", "weight_power")}
    inner = opts.get("inner_iters", 2)
    oc = O.OracleCloud.from_cloud(cloud, **ok)
    mach, alpha = Cl.conditions(4, seed=77)
    W = np.stack([Cl.perturbed_state(cloud, mach[k], alpha[k], seed=k + 1) for k in range(4)])
    with L.Solver.from_cloud(cloud, n_conditions=4, **opts) as b:
        b.set_conditions(mach, alpha)
        b.set_state(W)
        R = b.eval_residual()
        b.step(3)
        W3 = b.get_state()
    for k in (0, 3):
        _check_residual(oc, W[k], R[k], inner=inner)
        W3_o, _, st = O.iterate(oc, W[k], 3, inner=inner)
        assert st == 0
        assert normwise(W3[k], W3_o) < 1e-11


def test_set_conditions_checks_count(cloud):
    with L.Solver.from_cloud(cloud, n_conditions=4) as b:
        with pytest.raises(L.LskumError) as e:
            b.set_conditions([0.5, 0.6], [0.0, 1.0])
        assert e.value.code == -1


def test_ragged_packed_clouds_equal_separate_solves():
    """Three clouds of uneven size packed into one: every member evolves
    exactly as it does alone (neighbour order per point is kept)."""
    members = [Cl.naca0012_cloud(48, 14, seed=1), Cl.naca0012_cloud(96, 30, seed=2, shuffle=True),
               Cl.naca0012_cloud(64, 20, seed=3)]
    packed, offs = Cl.pack(members)
    with L.Solver.from_cloud(packed, precision=L.MIXED) as p:
        p.set_freestream(0.7, 1.5)
        p.step(10)
        Wp = p.get_state()
        assert p.info()["n_wall"] == sum(m.n_c for m in members)
    for m, a, b in zip(members, offs[:-1], offs[1:]):
        with L.Solver.from_cloud(m, precision=L.MIXED) as s:
            s.set_freestream(0.7, 1.5)
            s.step(10)
            assert np.array_equal(Wp[a:b], s.get_state())


def test_autotune_keeps_state_and_results(cloud):
    W = Cl.perturbed_state(cloud, 0.63, 2.0)
    with L.Solver.from_cloud(cloud) as a, L.Solver.from_cloud(cloud) as ref:
        a.set_freestream(0.63, 2.0)
        a.set_state(W)
        best = a.autotune(2)
        assert best[0] in (128, 256) and best[1] in (128, 256)
        ref.set_freestream(0.63, 2.0)
        ref.set_state(W)
        assert np.array_equal(a.get_state(), ref.get_state())
        a.step(3)
        ref.step(3)
        assert np.array_equal(a.get_state(), ref.get_state())
