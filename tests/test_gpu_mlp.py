"""Learned warm start on the GPU: tensor-core GEMMs, forward, back-propagation and AdamW against
the FP64 CPU reference (oracle/mlp_ref.py) on the same bf16-rounded weights and inputs, and the
glue between BMPC batches and the network."""
import numpy as np
import pytest

import scenes
from oracle import mlp_ref

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _bf(a):
    return torch.from_numpy(np.asarray(a, np.float32)).to(torch.bfloat16).cuda()


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


@pytest.mark.parametrize("K", [192, 1024])
@pytest.mark.parametrize("ta,tb", [(False, False), (True, False), (False, True), (True, True)])
def test_gemm_variants_match_fp64(ta, tb, K):
    """Every operand major on the tcgen05 path; K = 1024 cycles the 3-stage ring five times."""
    from paper_2506_13624_b300 import mlp
    rng = np.random.default_rng(int(ta) * 2 + int(tb) + K)
    M, N = 256, 384
    A = mlp_ref.bf16(rng.standard_normal((K, M) if ta else (M, K)))
    B = mlp_ref.bf16(rng.standard_normal((N, K) if tb else (K, N)))
    C = mlp.gemm(_bf(A), _bf(B), ta, tb).cpu().numpy()
    mlp.status()
    ref = (A.T if ta else A) @ (B.T if tb else B)
    assert _rel(C, ref) < 1e-5


def _net_and_ref(dims, seed=0):
    from paper_2506_13624_b300 import mlp
    net = mlp.MLP(dims, seed=seed)
    rng = np.random.default_rng(seed)
    for t in net.params:            # non-zero biases to exercise the epilogues
        t["b"].copy_(torch.from_numpy(0.1 * rng.standard_normal(t["b"].shape[0]).astype(np.float32)))
    Ws = [t["w_bf16"].float().cpu().numpy().astype(np.float64) for t in net.params]
    bs = [t["b"].cpu().numpy().astype(np.float64) for t in net.params]
    return net, Ws, bs


def test_forward_matches_reference():
    from paper_2506_13624_b300 import mlp
    dims = [256, 128, 128, 384]
    net, Ws, bs = _net_and_ref(dims)
    x = mlp_ref.bf16(np.random.default_rng(1).standard_normal((128, dims[0])))
    pred = net.forward(_bf(x)).cpu().numpy()
    mlp.status()
    ref, _ = mlp_ref.forward(Ws, bs, x, bf=True)
    assert _rel(pred, ref) < 5e-3


def test_training_step_gradients_and_adamw_match_reference():
    from paper_2506_13624_b300 import mlp
    dims = [256, 128, 128, 384]
    net, Ws, bs = _net_and_ref(dims, seed=3)
    rng = np.random.default_rng(2)
    x = mlp_ref.bf16(rng.standard_normal((128, dims[0])))
    t = mlp_ref.bf16(rng.standard_normal((128, dims[-1])))
    w_before = [p["w"].cpu().numpy().astype(np.float64) for p in net.params]
    loss = float(net.train_step(_bf(x), _bf(t), lr=1e-3, weight_decay=1e-2))
    mlp.status()
    rl, dWs, dbs = mlp_ref.loss_and_grads(Ws, bs, x, t, bf=True)
    assert abs(loss - rl) < 1e-3 * rl
    for l, p in enumerate(net.params):
        assert _rel(p["dw"].cpu().numpy(), dWs[l]) < 2e-2, l
        assert _rel(p["db"].cpu().numpy(), dbs[l]) < 2e-2, l
        g = p["dw"].cpu().numpy().astype(np.float64)
        w_ref, _, _ = mlp_ref.adamw(w_before[l], 0.0, 0.0, g, 1, 1e-3, 1e-2)
        assert _rel(p["w"].cpu().numpy(), w_ref) < 1e-6


def test_split_k_forward_and_gradients_match_reference():
    """Shapes whose GEMMs split along K (long inner dimension, few output tiles): the first layer's
    forward (bias + GELU epilogue) and the back-propagation through the output layer (GELU'
    epilogue) go through partial products and the split-K reduction."""
    from paper_2506_13624_b300 import mlp
    dims = [1664, 128, 128, 1024]
    net, Ws, bs = _net_and_ref(dims, seed=5)
    w_, _, _, _ = net.work(128)
    assert w_.splitk_floats > 0
    rng = np.random.default_rng(4)
    x = mlp_ref.bf16(rng.standard_normal((128, dims[0])))
    t = mlp_ref.bf16(rng.standard_normal((128, dims[-1])))
    pred = net.forward(_bf(x)).cpu().numpy()
    mlp.status()
    ref, _ = mlp_ref.forward(Ws, bs, x, bf=True)
    assert _rel(pred, ref) < 5e-3
    net.train_step(_bf(x), _bf(t), lr=1e-3)
    mlp.status()
    _, dWs, dbs = mlp_ref.loss_and_grads(Ws, bs, x, t, bf=True)
    for l, p in enumerate(net.params):
        assert _rel(p["dw"].cpu().numpy(), dWs[l]) < 2e-2, l
        assert _rel(p["db"].cpu().numpy(), dbs[l]) < 2e-2, l


def test_targets_and_starts_round_trip():
    from paper_2506_13624_b300 import bmpc, mlp, warmstart
    ps = scenes.batch_problems(1, 4, model=scenes.MODEL_KINEMATIC, N=20, splits={1: 3}, n_obs=2, n_cross=1,
                               cross_dist=(30.0, 50.0))
    b = warmstart.solve_batch(ps)
    sol = b.get_solutions()
    D = warmstart.target_dim(ps[0])
    tg = torch.empty((len(ps), D), dtype=torch.float32, device="cuda")
    mlp.targets(b, tg)
    mean = tg.mean(0)
    std = tg.std(0).clamp_min(1e-3)
    pred = ((tg - mean) / std).contiguous()
    st = torch.empty((len(ps), b.start_stride()), dtype=torch.float32, device="cuda")
    mlp.starts(b, pred, mean, std, st)
    st = st.cpu().numpy()
    for k, (p, s) in enumerate(zip(ps, sol)):
        n, nx, nc = p["n"], p["nx"], bmpc.n_con(p)
        # the start rolls the (converged, defect-free) controls out again: it reproduces the solution
        packed = np.concatenate([s["x"].ravel(), s["u"].ravel(), s["lam"].ravel(), s["y"].ravel()])
        np.testing.assert_allclose(st[k, :packed.size], packed, atol=2e-3 * max(1.0, np.abs(packed).max()))
    f = torch.zeros((len(ps), warmstart.feature_dim(ps[0])), dtype=torch.float32, device="cuda")
    mlp.features(b, f, warmstart.N_SCEN, warmstart.N_OBS)
    f = f.cpu().numpy()
    p = ps[0]
    assert abs(f[0, 0] - p["x0"][1]) < 1e-6
    leaf = int(np.where(p["stage"] == p["stage"].max())[0][0])
    assert abs(f[0, 3 + 2] - (p["obs"][leaf, 0, 0] - p["x0"][0])) < 1e-4
    b.close()


def test_bounded_wait_gives_up_and_the_context_stays_usable():
    """A wait for an mbarrier phase that nothing completes gives up after its limit (about 1 ms here),
    bmpc_mlp_status reports the timeout once and clears it, and a GEMM afterwards is exact: the
    failure path of the tensor-core kernels, exercised without any fault."""
    from paper_2506_13624_b300 import mlp
    assert mlp.status_code() == 0
    mlp.selftest_wait(2_000_000)
    assert mlp.status_code() == -4
    assert mlp.status_code() == 0
    g = torch.Generator().manual_seed(3)
    A = torch.randn(128, 64, generator=g).to(torch.bfloat16)
    B = torch.randn(64, 128, generator=g).to(torch.bfloat16)
    Cg = mlp.gemm(A.cuda(), B.cuda()).cpu().double()
    ref = A.double() @ B.double()
    assert torch.allclose(Cg, ref, rtol=1e-5, atol=1e-4)
    assert mlp.status_code() == 0

