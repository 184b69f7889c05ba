"""Warm-start surrogate on the GPU: the BF16 tensor-core network against its
FP64 reference (features, forward, gradients), training, and what the
trained network gains over the free-stream start."""

import numpy as np
import pytest

from oracle import mlp_oracle as M
from paper_2108_07031_gb300 import cloud as Cl
from parity_utils import normwise

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2108_07031_gb300 import lskum as L  # noqa: E402
from paper_2108_07031_gb300 import surrogate as S  # noqa: E402


@pytest.fixture(scope="module")
def net():
    m = S.MLP(capacity=4096, seed=1)
    yield m
    m.close()


def test_features_match_reference(net):
    rng = np.random.Generator(np.random.PCG64(1))
    raw = np.stack([rng.uniform(-20, 20, 500), rng.uniform(-20, 20, 500), rng.uniform(0, 20, 500),
                    rng.uniform(0.3, 0.8, 500), rng.uniform(-4, 6, 500)], 1).astype(np.float32)
    f = net.features(torch.from_numpy(raw).cuda()).cpu().numpy()
    ref = M.features(raw, net.proj)
    assert np.abs(f - ref).max() < 2e-5


def _batch(n, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    feat = rng.normal(0, 1, (n, 32)).astype(np.float32)
    feat[:, 21:] = 0.0
    T = rng.normal(0, 0.5, (n, 4)).astype(np.float32)
    return feat, T


@pytest.mark.parametrize("n", [1000, 333, 40])
def test_forward_and_gradients_match_reference(net, n):
    """GPU (BF16 operands, FP32 accumulation) against the FP64 reference with
    the same BF16 rounding points: outputs to 5e-3 and gradients to 2e-2
    norm-wise (activations rounded to BF16 can land on the other side of a
    rounding boundary than in FP64). Batch sizes: ragged against the 128-row
    tiles of the pipelined GEMM (1000, 333) and below its 64-row minimum (40,
    the 64 x 64 kernel)."""
    feat, T = _batch(n, 2)
    p = S.init_params(3)
    p[-4:] = [0.1, -0.2, 0.05, 0.3]  # non-zero output bias
    net.set_params(p)
    fd = torch.from_numpy(feat).cuda()
    Td = torch.from_numpy(T).cuda()
    Y = net.predict(fd).cpu().numpy()
    Y_o, _ = M.forward(p, feat, emulate=True)
    assert normwise(Y, Y_o) < 5e-3
    loss, g = net.gradients(fd, Td)
    loss_o, g_o = M.loss_and_grad(p, feat, T, emulate=True)
    assert abs(loss - loss_o) < 1e-3 * loss_o
    # per layer, weights and biases
    off = 0
    for n, k in M.layer_shapes():
        for size in (n * k, n):
            gl, gol = g[off:off + size], g_o[off:off + size]
            assert np.abs(gl - gol).max() <= 2e-2 * np.abs(gol).max() + 1e-9, (n, k, size)
            off += size


@pytest.mark.parametrize("n", [4096, 1000, 333, 40])
def test_tcgen05_forward_matches_reference(net, n):
    """The forward pass with its 256-wide layers on tcgen05 (tensor-memory
    accumulators, 128-row tiles; ragged batches fill the last tile with zero
    rows): outputs against the FP64 reference with the same BF16 rounding
    points (5e-3 norm-wise) and against the mma.sync path (the two sum the
    same FP32 products in another order: 1e-2 of the output's scale, where a
    hidden activation's BF16 rounding may flip between them); gradients with
    it to the reference's 2e-2 per layer."""
    feat, T = _batch(n, 4)
    p = S.init_params(5)
    p[-4:] = [0.1, -0.2, 0.05, 0.3]
    net.set_params(p)
    fd, Td = torch.from_numpy(feat).cuda(), torch.from_numpy(T).cuda()
    try:
        net.set_gemm(S.GEMM_MMA_SYNC)
        Y_ref = net.predict(fd).cpu().numpy()
        net.set_gemm(S.GEMM_TCGEN05)
        Y = net.predict(fd).cpu().numpy()
        Y2 = net.predict(fd).cpu().numpy()
        loss, g = net.gradients(fd, Td)
    finally:
        net.set_gemm(S.GEMM_MMA_SYNC)
    assert np.array_equal(Y, Y2)  # deterministic
    Y_o, _ = M.forward(p, feat, emulate=True)
    print(f"n {n}: tcgen05 vs reference {normwise(Y, Y_o):.2e}, vs mma.sync {normwise(Y, Y_ref):.2e}")
    assert normwise(Y, Y_o) < 5e-3
    assert normwise(Y, Y_ref) < 1e-2
    loss_o, g_o = M.loss_and_grad(p, feat, T, emulate=True)
    assert abs(loss - loss_o) < 1e-3 * loss_o
    off = 0
    for nn_, k in M.layer_shapes():
        for size in (nn_ * k, nn_):
            gl, gol = g[off:off + size], g_o[off:off + size]
            assert np.abs(gl - gol).max() <= 2e-2 * np.abs(gol).max() + 1e-9, (nn_, k, size)
            off += size


def test_training_reduces_loss(net):
    """Adam on a smooth target of the features: loss falls by 10x in 300 steps."""
    rng = np.random.Generator(np.random.PCG64(5))
    feat = rng.uniform(-1, 1, (4096, 32)).astype(np.float32)
    feat[:, 21:] = 0.0
    T = np.stack([np.sin(2 * feat[:, 0]) * feat[:, 1], feat[:, 2] ** 2 - 0.3,
                  np.tanh(feat[:, 3] + feat[:, 4]), 0.5 * feat[:, 5]], 1).astype(np.float32)
    net.set_params(S.init_params(7))
    fd, Td = torch.from_numpy(feat).cuda(), torch.from_numpy(T).cuda()
    first = None
    for it in range(300):
        loss = net.train_step(fd, Td, 1e-3)
        first = loss if first is None else first
    assert loss < 0.1 * first, (first, loss)


def test_warm_start_gains_iterations():
    """Trained on 32 converged conditions of the 5,120-point cloud, the warm
    start needs fewer iterations to a 6-order residue drop than the
    free-stream start on held-out conditions (mixed precision, CFL 0.8 to keep
    the test short), and both starts converge to the same lift and drag
    (within 1e-4): the prediction keeps the exact free stream at the held
    far-field points, whose state is the problem's boundary data."""
    cloud = Cl.naca0012_cloud(128, 40)
    wd = S.wall_distance(cloud)
    rng = np.random.Generator(np.random.PCG64(11))
    mach_tr, alpha_tr = rng.uniform(0.3, 0.7, 32), rng.uniform(-3.0, 4.0, 32)
    W_tr, _ = S.converged_solutions(cloud, mach_tr, alpha_tr, tol=1e-6, max_iters=30_000)
    raw = np.concatenate(S.raw_inputs(cloud, wd, mach_tr, alpha_tr))
    T = np.concatenate([S.targets(W_tr[k], mach_tr[k], alpha_tr[k]) for k in range(32)])
    net = S.MLP(capacity=16384, seed=2)
    feats = net.features(torch.from_numpy(raw).cuda())
    Td = torch.from_numpy(T).cuda()
    losses = S.train(net, feats, Td, epochs=100, batch=4096, lr=2e-3, lr_final=5e-5)
    assert losses[-1] < 0.05 * losses[0]
    mach_te, alpha_te = np.array([0.42, 0.61]), np.array([-1.3, 2.4])
    gains, dcl = [], []
    for m, a in zip(mach_te, alpha_te):
        res = {}
        for mode in ("cold", "warm"):
            with L.Solver.from_cloud(cloud, precision=L.MIXED, cfl=0.8) as s:
                s.set_freestream(m, a)
                if mode == "warm":
                    W0 = S.predict_state(net, cloud, wd, m, a)
                    assert W0 is not None
                    s.set_state(W0)
                hist = []
                for _ in range(150):
                    s.step(100)
                    hist.append(s.residual_norm())
                res[mode] = (np.array(hist), s.forces())
        cold, warm = res["cold"][0], res["warm"][0]
        with L.Solver.from_cloud(cloud, precision=L.MIXED, cfl=0.8) as s:
            s.set_freestream(m, a)  # reference: first residue of the free-stream start
            s.step(2)
            r_first = s.residual_norm()
        thr = 1e-6 * r_first
        assert cold.min() < thr and warm.min() < thr, (cold.min(), warm.min(), thr)
        it_cold = 100 * (1 + np.argmax(cold < thr))
        it_warm = 100 * (1 + np.argmax(warm < thr))
        gains.append(1 - it_warm / it_cold)
        dcl.append(res["warm"][1][0] - res["cold"][1][0])
        assert abs(res["warm"][1][1] - res["cold"][1][1]) < 1e-4  # Cd
    print("warm-start iteration savings:", [f"{g:.0%}" for g in gains],
          "converged Cl shift:", [f"{d:+.2e}" for d in dcl])
    assert np.mean(gains) > 0.1
    assert np.all(np.abs(dcl) < 1e-4)
    net.close()
