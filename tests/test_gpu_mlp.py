"""Learned warm start on the GPU: tensor-core GEMMs, forward, back-propagation and AdamW against
the FP64 CPU reference (oracle/mlp_ref.py) on the same bf16-rounded weights and inputs, and the
glue between BMPC batches and the network.

Element-wise bars.  A GEMM sums K products in FP32: against the FP64 sum of the same bf16 operands
its error is at most about K u (|A| |B|)_ij with u = 2^-24 (the bound of recursive summation; the
tensor core's order is another order of the same sums), so every entry is checked against
ACC * K u (|A| |B|)_ij.  A bf16 result (pre-activation, activation, back-propagated gradient) is
bf16(v) of an FP32 value v that is within that bound of the FP64 one: it equals the reference's
bf16 rounding except where v lies that close to a rounding boundary, and then differs by one bf16
ulp.  Those checks compare layer by layer, each layer fed the GPU's own inputs (its bf16
activations and gradients), so that a rounding flip in one layer does not blur the next layer's
bar.  The end-to-end forward pass is also compared against the reference run from the input alone,
by relative Frobenius norm (flips do propagate there)."""
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


U32 = 2.0 ** -24          # FP32 unit roundoff
ACC = 4.0                 # slack factor on the K u accumulation bound


def _acc_bound(A, B, K):
    """ACC K u (|A| |B|): the FP32 accumulation bound of every entry of A @ B."""
    return ACC * K * U32 * (np.abs(A) @ np.abs(B))


def _f64(t):
    return t.float().cpu().numpy().astype(np.float64)


def _bf_ulp(v):
    """One bf16 ulp at |v| (8 significant bits)."""
    e = np.floor(np.log2(np.maximum(np.abs(v), 2.0 ** -126)))
    return 2.0 ** (e - 7)


def _assert_bf16_matches(got, ref_exact, name, max_flip_frac=2e-3):
    """got = bf16 of an FP32 value close to ref_exact: equal to bf16(ref_exact) except for one-ulp
    rounding flips, which must be rare."""
    want = mlp_ref.bf16(ref_exact)
    diff = np.abs(got - want)
    assert (diff <= _bf_ulp(ref_exact) * 1.0001 + 1e-30).all(), (name, float(diff.max()))
    flips = np.count_nonzero(diff)
    assert flips <= max(2, max_flip_frac * got.size), (name, flips, got.size)


@pytest.mark.parametrize("N", [384, 512])
@pytest.mark.parametrize("K", [192, 1024])
@pytest.mark.parametrize("ta,tb", [(False, False), (True, False), (False, True), (True, True)])
def test_gemm_variants_match_fp64(ta, tb, K, N):
    """Every operand major on the tcgen05 path, with 128 x 128 output tiles (N = 384) and 128 x 256
    ones (N = 512); K = 1024 cycles the 4-stage ring four times."""
    from paper_2506_13624_b300 import mlp
    rng = np.random.default_rng(int(ta) * 2 + int(tb) + K + N)
    M = 256
    A = mlp_ref.bf16(rng.standard_normal((K, M) if ta else (M, K)))
    B = mlp_ref.bf16(rng.standard_normal((N, K) if tb else (K, N)))
    C = mlp.gemm(_bf(A), _bf(B), ta, tb).cpu().numpy()
    mlp.status()
    opA, opB = (A.T if ta else A), (B.T if tb else B)
    ref = opA @ opB
    assert (np.abs(C - ref) <= _acc_bound(opA, opB, K)).all()
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


def _layerwise_forward(net, Ws, bs, x, pred):
    """Every layer of the GPU forward pass element by element, fed the GPU's own inputs."""
    w, keep, _, _ = net.work(x.shape[0])
    hidden = len(Ws) - 1
    h = x
    for l in range(len(Ws)):
        z = h @ Ws[l] + bs[l]
        bound = _acc_bound(h, Ws[l], h.shape[1]) + 4 * U32 * np.abs(bs[l])
        if l < hidden:
            pre, act = _f64(keep[2 * l]), _f64(keep[2 * l + 1])
            _assert_bf16_matches(pre, z, f"pre{l}")
            assert (np.abs(pre - z) <= _bf_ulp(z) + bound).all()
            _assert_bf16_matches(act, mlp_ref.gelu(pre), f"act{l}")
            h = act
        else:
            assert (np.abs(pred - z) <= bound).all(), float(np.max(np.abs(pred - z) - bound))


def test_forward_matches_reference():
    from paper_2506_13624_b300 import mlp
    dims = [256, 128, 128, 384]
    net, Ws, bs = _net_and_ref(dims)
    x = mlp_ref.bf16(np.random.default_rng(1).standard_normal((128, dims[0])))
    pred = net.forward(_bf(x)).cpu().numpy().astype(np.float64)
    mlp.status()
    _layerwise_forward(net, Ws, bs, x, pred)
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
    _layerwise_backward(net, Ws, x, t)
    for l, p in enumerate(net.params):
        assert _rel(p["dw"].cpu().numpy(), dWs[l]) < 2e-2, l
        assert _rel(p["db"].cpu().numpy(), dbs[l]) < 2e-2, l
        g = p["dw"].cpu().numpy().astype(np.float64)
        w_ref, _, _ = mlp_ref.adamw(w_before[l], 0.0, 0.0, g, 1, 1e-3, 1e-2)
        np.testing.assert_allclose(p["w"].cpu().numpy(), w_ref, rtol=1e-6, atol=1e-7)


def _layerwise_backward(net, Ws, x, t):
    """The back-propagation of a training step element by element, three layers (the work buffers
    then hold g_1 and g_0, the gradients at the two hidden layers): the output gradient from the
    GPU's own prediction, each hidden gradient from the GPU's own upper gradient and
    pre-activation, and every dW, db from the GPU's own activations and gradients."""
    assert len(Ws) == 3
    B = x.shape[0]
    w, keep, pred, _ = net.work(B)
    pre = [_f64(keep[0]), _f64(keep[2])]
    act = [_f64(keep[1]), _f64(keep[3])]
    # dy0, dy1 hold contiguous [B][width] gradients: g_0 in dy0, g_1 in dy1 after the step
    h0, h1 = Ws[0].shape[1], Ws[1].shape[1]
    # only the first B * width entries are written: the rest of the buffer is never read
    g0 = _f64(keep[-5].reshape(-1)[:B * h0]).reshape(B, h0)
    g1 = _f64(keep[-4].reshape(-1)[:B * h1]).reshape(B, h1)
    P = _f64(pred)
    e = P - t
    g2_exact = 2.0 * e / e.size
    g2 = mlp_ref.bf16(g2_exact)
    # hidden gradients: bf16((g W^T) * gelu'(pre)) from the GPU's own g and pre
    up1 = g2 @ Ws[2].T
    _assert_bf16_matches(g1, up1 * mlp_ref.gelu_grad(pre[1]), "g1")
    up0 = g1 @ Ws[1].T
    _assert_bf16_matches(g0, up0 * mlp_ref.gelu_grad(pre[0]), "g0")
    ins = [x, act[0], act[1]]
    gs = [g0, g1, g2]
    for l, p in enumerate(net.params):
        dw, db = _f64(p["dw"]), _f64(p["db"])
        want = ins[l].T @ gs[l]
        bound = _acc_bound(ins[l].T, gs[l], B)
        if l == 2:
            # the output gradient is recomputed here: allow a rare bf16 flip in it
            bound = bound + np.abs(ins[l].T) @ _bf_ulp(g2_exact) * (np.abs(g2 - mlp_ref.bf16(g2_exact)) > 0)
            flip = np.abs(dw - want) > bound
            assert np.count_nonzero(flip) <= max(2, 1e-3 * dw.size), (l, np.count_nonzero(flip))
            assert (np.abs(dw - want) <= bound + np.abs(ins[l].T) @ _bf_ulp(g2_exact)).all()
        else:
            assert (np.abs(dw - want) <= bound).all(), (l, float(np.max(np.abs(dw - want) - bound)))
        assert (np.abs(db - gs[l].sum(axis=0)) <= ACC * B * U32 * np.abs(gs[l]).sum(axis=0) + 1e-30).all(), l


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
    pred = net.forward(_bf(x)).cpu().numpy().astype(np.float64)
    mlp.status()
    _layerwise_forward(net, Ws, bs, x, pred)
    ref, _ = mlp_ref.forward(Ws, bs, x, bf=True)
    assert _rel(pred, ref) < 5e-3
    net.train_step(_bf(x), _bf(t), lr=1e-3)
    mlp.status()
    _layerwise_backward(net, Ws, x, t)
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
    for y_sqrt in (0, 1):
        mlp.targets(b, tg, y_sqrt)
        mean = tg.mean(0)
        std = tg.std(0).clamp_min(1e-3)
        pred = ((tg - mean) / std).contiguous()
        st = torch.empty((len(ps), b.start_stride()), dtype=torch.float32, device="cuda")
        mlp.starts(b, pred, mean, std, st, y_sqrt)
        st = st.cpu().numpy()
        tgh = tg.cpu().numpy()
        for k, (p, s) in enumerate(zip(ps, sol)):
            n, nx, nc = p["n"], p["nx"], bmpc.n_con(p)
            # the start rolls the (converged, defect-free) controls out again: it reproduces the solution
            packed = np.concatenate([s["x"].ravel(), s["u"].ravel(), s["lam"].ravel(), s["y"].ravel()])
            np.testing.assert_allclose(st[k, :packed.size], packed, atol=2e-3 * max(1.0, np.abs(packed).max()))
            # the multiplier targets in the requested form
            yt = tgh[k, packed.size - s["y"].size:packed.size]
            np.testing.assert_allclose(yt, np.sqrt(s["y"].ravel()) if y_sqrt else s["y"].ravel(), rtol=1e-6,
                                       atol=1e-30)
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

