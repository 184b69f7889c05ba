"""lskum_residue_noalloc against the solver's own residue (lskum_residual_norm).

The allocation-free entry point serves callers that may not allocate device
memory (code inside a CUDA-graph capture it does not own, plug-ins whose host
framework owns every allocation). It must give the same residue as the
solver's lskum_step / lskum_residual_norm path for the same stage-1 residual.
The file is named so that pytest collects it last.
"""

import numpy as np
import pytest

from paper_2108_07031_gb300 import cloud as Cl

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2108_07031_gb300 import lskum as L  # noqa: E402

TOL = 1e-12  # the one-step parity tolerance of the FP64 path


def _reference_residue(cloud, W):
    """Stage-1 residual of W and the residue lskum_step reports for it."""
    with L.Solver.from_cloud(cloud) as s:
        s.set_state(W)
        R = s.eval_residual()
        s.step(1)
        return R, s.residual_norm()


def test_noalloc_residue_matches_solver_two_calls_in_a_row():
    # the first call covers more scratch blocks (3) than the second (1), so a
    # stale partial sum from the first call would show up in the second
    big = Cl.naca0012_cloud(256, 80)     # 20480 points
    small = Cl.naca0012_cloud(128, 40)   # 5120 points
    cases = [(big, Cl.perturbed_state(big, 0.63, 2.0)),
             (small, Cl.perturbed_state(small, 0.85, 1.0, seed=3))]
    refs = [_reference_residue(c, W) for c, W in cases]
    stream = torch.cuda.current_stream()
    outs = []
    for (c, _), (R, _) in zip(cases, refs):
        R_dev = torch.from_numpy(R).to("cuda")
        out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
        L.residue_noalloc(R_dev.data_ptr(), c.n, out.data_ptr(), stream.cuda_stream)
        torch.cuda.synchronize()
        outs.append(float(out.item()))
    for got, (_, want) in zip(outs, refs):
        assert want > 0
        assert abs(got - want) <= TOL * want, (got, want)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    R_dev = torch.zeros((4, 4), dtype=torch.float64, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    for n in (0, L.NOALLOC_MAX_POINTS + 1):
        with pytest.raises(L.LskumError) as e:
            L.residue_noalloc(R_dev.data_ptr(), n, out.data_ptr(), 0)
        assert e.value.code == -1
    assert "outside" in L.load().lskum_last_error().decode()
