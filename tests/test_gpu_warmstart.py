"""What the trained warm-start network gains: a network trained by the library's own kernels on
solutions of the library's own solver, on a smaller scene family than the full experiment
(kinematic bicycle, N = 30, binary splits at stages 1, 5 and 10, three obstacles), against the
cold start of Sec. V-B and against the same network untrained."""
import numpy as np
import pytest

import scenes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SPLITS = {1: 2, 5: 2, 10: 2}


def _family(seed, count):
    ps = scenes.batch_problems(seed, count, model=scenes.MODEL_KINEMATIC, N=30, splits=SPLITS, n_obs=3,
                               n_cross=1)
    for p in ps:
        p["obs"] = p["obs"].astype(np.float32)
    return ps


def _unpack(p, s, nc):
    n, nx = p["n"], p["nx"]
    o = [0, n * nx, n * nx + 2 * n, 2 * n * nx + 2 * n, 2 * n * nx + 2 * n + n * nc]
    return (s[o[0]:o[1]].reshape(n, nx), s[o[1]:o[2]].reshape(n, 2), s[o[2]:o[3]].reshape(n, nx),
            s[o[3]:o[4]].reshape(n, nc))


def _packed_starts(net, b, stats):
    from paper_2506_13624_b300 import mlp, warmstart
    rows = (b.n + 127) // 128 * 128
    fx = torch.zeros((rows, net.dims[0]), dtype=torch.float32, device="cuda")
    mlp.features(b, fx, warmstart.N_SCEN, warmstart.N_OBS)
    xb = torch.empty((rows, net.dims[0]), dtype=torch.bfloat16, device="cuda")
    mlp.standardize(fx, stats["fm"], stats["fs"], xb)
    st = torch.empty((b.n, b.start_stride()), dtype=torch.float32, device="cuda")
    mlp.starts(b, net.forward(xb), stats["tm"], stats["ts"], st)
    return st


def _dist(ps, starts, sols, nc):
    """Mean over problems of the RMS distance of the start's states and controls to the solution."""
    d = []
    for p, s, r in zip(ps, starts, sols):
        x, u = _unpack(p, s, nc)[:2]
        d.append(np.sqrt(np.mean((x - r["x"]) ** 2) + np.mean((u - r["u"]) ** 2)))
    return float(np.mean(d))


def _summary(res):
    it = np.array([r["inner_iters"] for r in res])
    return float(it.mean()), float(np.mean([r["status"] == 0 for r in res]))


def test_trained_network_gains_over_cold_start_and_untrained_network():
    import oracle
    from paper_2506_13624_b300 import bmpc, mlp, warmstart
    opts = bmpc.default_opts()
    X, Y, info = warmstart.build_dataset(lambda c, cnt: _family(1000 + c, cnt), 8192, 4096, opts, log=None)
    assert info["kept"] > 0.9 * info["total"]
    Xb, Yb, stats = warmstart.standardise(X, Y)
    dims = [Xb.shape[1], 256, 256, 256, Yb.shape[1]]
    untrained = mlp.MLP(dims, seed=1)
    net = mlp.MLP(dims, seed=1)
    hist, _ = warmstart.train(net, Xb, Yb, 30, batch=256, lr=1e-3, log=None)
    assert hist[-1] < 0.5 * hist[0]

    ps = _family(999, 512)                 # held-out scenes
    nc = bmpc.n_con(ps[0])
    b = bmpc.Batch(ps)
    b.set_problems()
    b.solve(opts)
    sol = b.get_solutions()
    it_cold, conv_cold = _summary(sol)
    ok = [k for k, r in enumerate(sol) if r["status"] == 0]

    # the trained start is much closer to the converged solutions than the cold start or the untrained network
    st = _packed_starts(net, b, stats)
    st_h = st.cpu().numpy()
    st_u = _packed_starts(untrained, b, stats).cpu().numpy()
    cold = []
    for p in ps:
        x, u, lam, y = oracle.cold_start(p)
        cold.append(np.concatenate([x.ravel(), u.ravel(), lam.ravel(), y.ravel()]).astype(np.float32))
    sub = lambda a: [a[k] for k in ok]
    d_net, d_cold, d_untr = (_dist(sub(ps), sub(a), sub(sol), nc) for a in (st_h, cold, st_u))
    assert d_net < 0.5 * d_cold and d_net < 0.5 * d_untr, (d_net, d_cold, d_untr)

    # merit selection with the cold start as fallback: the start used has the lower merit
    sel = bmpc.default_opts(warm_select=1)
    b.set_problems()
    b.set_warm_device(st, slot=0)
    b.solve(sel)
    res = b.get_solutions()
    checked = 0
    for k in range(0, len(ps), 16):
        x, u, lam, y = _unpack(ps[k], st_h[k], nc)
        m_net = oracle.merit(ps[k], x, u, lam, y, sel.select_rho, sel.select_mu)
        m_cold = oracle.merit(ps[k], *oracle.cold_start(ps[k]), sel.select_rho, sel.select_mu)
        if abs(m_net - m_cold) > 1e-3 * max(abs(m_net), abs(m_cold)):
            assert res[k]["start_used"] == (1 if m_net < m_cold else 0), (k, m_net, m_cold)
            checked += 1
    assert checked >= 16
    it_sel, conv_sel = _summary(res)

    # a solve from the learned start ends where the oracle's solve from the same start ends: the
    # FP64 KKT conditions hold at the GPU's point, the controls agree, and so do the iteration counts
    compared = 0
    for k in range(0, len(ps), 16):
        g = res[k]
        if g["start_used"] != 1:
            continue
        warm = tuple(np.asarray(a, np.float64) for a in _unpack(ps[k], st_h[k], nc))
        r = oracle.solve(ps[k], warm=warm, **oracle.PRODUCT_RULE)
        if r["status"] != oracle.OK:
            continue
        assert g["status"] == oracle.OK, (k, g["status"], g["r_kkt"])
        assert oracle.kkt(ps[k], g["x"], g["u"], g["lam"], g["y"])[:4].max() <= 1e-5, k
        du = np.abs(g["u"] - r["u"]).max()
        assert du <= 1e-4 * max(1.0, np.abs(r["u"]).max()), (k, du)
        assert abs(g["inner_iters"] - r["inner_iters"]) <= 1, (k, g["inner_iters"], r["inner_iters"])
        compared += 1
    assert compared >= 8, compared

    # and the solves: fewer iterations on average and no fewer converged problems than the cold start
    print(f"\ncold: {it_cold:.2f} iterations, {conv_cold:.3f} converged; learned with cold fallback: "
          f"{it_sel:.2f} iterations, {conv_sel:.3f} converged, network start used for "
          f"{np.mean([r['start_used'] == 1 for r in res]):.3f}; start distance {d_net:.3g} vs cold {d_cold:.3g}")
    assert it_sel < it_cold
    assert conv_sel >= conv_cold - 1.0 / len(ps)
    b.close()
