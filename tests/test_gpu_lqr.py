"""The general-size tree LQR (include/bmpc_lqr.h) against the FP64 oracle's tree Riccati recursion
with per-edge matrices (orc_tree_lqr, pinned on the CPU against dense KKT solves) and against dense
KKT solves written here.

Bar: every returned block (K, k, P, p, x, u, lam) element by element, relative to the block's
magnitude max(1, |block|_inf).  The recursion is FP32 dot products of length n_x + n_u per entry,
carried through the tree's depth; on these well-conditioned problems (the mass-spring chains of
Sec. V-A, random edges close to the identity) the worst element was a few 1e-6 of its block in
the measurements, and the bar is 1e-4.
"""
import numpy as np
import pytest

import oracle
import scenes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-4


def _tree(rng, n_max):
    """Level-ordered ragged tree: fan-out 0..3 (at least 1 at the root), leaves at any depth."""
    parent, frontier = [-1], [0]
    while frontier and len(parent) < n_max:
        nxt = []
        for q in frontier:
            for _ in range(int(rng.integers(1 if q == 0 else 0, 4))):
                if len(parent) < n_max:
                    parent.append(q)
                    nxt.append(len(parent) - 1)
        frontier = nxt
    return np.array(parent, np.int32)


def _random_data(rng, parent, nx, nu, batch):
    n = len(parent)
    leaf = np.ones(n, bool)
    leaf[parent[1:]] = False
    Q, M, R = np.zeros((batch, n, nx, nx)), np.zeros((batch, n, nu, nx)), np.zeros((batch, n, nu, nu))
    for t in range(batch):
        for i in range(n):
            F = rng.standard_normal((nx + nu, nx + nu)) / np.sqrt(nx + nu)
            W = F @ F.T + 0.5 * np.eye(nx + nu)
            Q[t, i] = W[:nx, :nx]
            if not leaf[i]:
                M[t, i], R[t, i] = W[nx:, :nx], W[nx:, nx:]
    q = rng.standard_normal((batch, n, nx))
    r = rng.standard_normal((batch, n, nu)) * (~leaf)[None, :, None]
    A = np.eye(nx) + (0.3 / np.sqrt(nx)) * rng.standard_normal((batch, n, nx, nx))
    B = rng.standard_normal((batch, n, nx, nu)) / np.sqrt(nx)
    c = rng.standard_normal((batch, n, nx))
    c[:, 0] = 0.0
    return leaf, Q, M, R, q, r, A, B, c


def _dev(a):
    return torch.tensor(np.ascontiguousarray(a, np.float32), device="cuda")


def _solve(parent, nx, nu, Q, R, q, r, A, B, c, x0, M=None, schedule=0):
    from paper_2506_13624_b300 import lqr
    h = lqr.TreeLQR(parent, nx, nu, batch=Q.shape[0], schedule=schedule)
    out = h.solve(_dev(Q), _dev(R), _dev(q), _dev(r), _dev(A), _dev(B), _dev(c), _dev(x0),
                  M=None if M is None else _dev(M))
    res = {k: v.cpu().numpy().astype(np.float64) for k, v in out.items()}
    h.close()
    return res


def _close(got, want, what):
    scale = max(1.0, float(np.abs(want).max()))
    d = float(np.abs(got - want).max()) / scale
    assert d <= TOL, (what, d)
    return d


@pytest.mark.parametrize("schedule", [1, 2])
@pytest.mark.parametrize("nx,nu", [(4, 2), (7, 3), (10, 4), (16, 8), (30, 14), (32, 16)])
def test_matches_the_oracle_tree_recursion(nx, nu, schedule):
    """Random ragged trees, per-edge A_m, B_m, c_m, cross terms M, a batch of three problems: every
    block equal to the oracle's (dx_0 = 0 there, so x0 = 0 here), with a launch per stage and with
    one block per problem."""
    rng = np.random.default_rng(500 + nx)
    parent = _tree(rng, 40)
    batch = 3
    leaf, Q, M, R, q, r, A, B, c = _random_data(rng, parent, nx, nu, batch)
    got = _solve(parent, nx, nu, Q, R, q, r, A, B, c, np.zeros((batch, nx)), M=M, schedule=schedule)
    worst = 0.0
    for t in range(batch):
        K, k, P, pv, dx, du, lam = oracle.tree_lqr(parent, Q[t], M[t], R[t], q[t], r[t], A[t], B[t], c[t], edge=True)
        ref = dict(K=K, k=k, P=P, p=pv, x=dx, u=du, lam=lam)
        for key, want in ref.items():
            g = got[key][t]
            if key in ("K", "k", "u"):
                g, want = g[~leaf], want[~leaf]
            worst = max(worst, _close(g, want, (nx, nu, t, key)))
        assert np.all(got["u"][t][leaf] == 0) and np.all(got["K"][t][leaf] == 0)
    print(f"nx={nx} nu={nu} n={len(parent)} worst {worst:.2e}")


def _dense_kkt_x0(parent, leaf, Q, M, R, q, r, A, B, c, x0):
    """The tree LQR as one equality-constrained QP with x_0 = x0: returns x, u."""
    n, nx, nu = len(parent), Q.shape[1], R.shape[1]
    uidx, off = {}, n * nx
    for i in range(n):
        if not leaf[i]:
            uidx[i] = off
            off += nu
    H, h = np.zeros((off, off)), np.zeros(off)
    for i in range(n):
        xi = slice(i * nx, (i + 1) * nx)
        H[xi, xi] += Q[i]
        h[xi] += q[i]
        if i in uidx:
            ui = slice(uidx[i], uidx[i] + nu)
            H[ui, ui] += R[i]
            H[ui, xi] += M[i]
            H[xi, ui] += M[i].T
            h[ui] += r[i]
    E, e = np.zeros((n * nx, off)), np.zeros(n * nx)
    E[:nx, :nx] = np.eye(nx)
    e[:nx] = x0
    for m in range(1, n):
        p_ = parent[m]
        rows = slice(m * nx, (m + 1) * nx)
        E[rows, m * nx:(m + 1) * nx] = np.eye(nx)
        E[rows, p_ * nx:(p_ + 1) * nx] -= A[m]
        E[rows, uidx[p_]:uidx[p_] + nu] -= B[m]
        e[rows] = c[m]
    KKT = np.block([[H, E.T], [E, np.zeros((n * nx, n * nx))]])
    z = np.linalg.solve(KKT, np.concatenate([-h, e]))[:off]
    x = z[:n * nx].reshape(n, nx)
    u = np.zeros((n, nu))
    for i, o in uidx.items():
        u[i] = z[o:o + nu]
    return x, u


@pytest.mark.parametrize("nx,nu", [(6, 2), (30, 14)])
def test_initial_state_against_the_dense_kkt_solution(nx, nu):
    """x_0 = x0 (not zero) on a small tree: x and u equal the dense KKT solution; the costates are
    the gradients of the returned value functions, P x + p."""
    rng = np.random.default_rng(600 + nx)
    parent = _tree(rng, 12)
    leaf, Q, M, R, q, r, A, B, c = _random_data(rng, parent, nx, nu, 2)
    x0 = rng.standard_normal((2, nx))
    got = _solve(parent, nx, nu, Q, R, q, r, A, B, c, x0, M=M)
    for t in range(2):
        x, u = _dense_kkt_x0(parent, leaf, Q[t], M[t], R[t], q[t], r[t], A[t], B[t], c[t], x0[t])
        _close(got["x"][t], x, "x")
        _close(got["u"][t], u, "u")
        lam = np.einsum("nij,nj->ni", got["P"][t], got["x"][t]) + got["p"][t]
        _close(got["lam"][t], lam, "lam")
        assert np.allclose(got["x"][t][0], x0[t].astype(np.float32), atol=1e-6)


@pytest.mark.parametrize("Nr", [1, 3, 5])
def test_mass_spring_chain_of_the_paper(Nr):
    """Sec. V-A's trees at the paper's size: 15 masses (n_x = 30, n_u = 14), n_d = 2 spring constants
    per stage up to N_r, horizon 20, a batch of two.  Against the oracle through the deviation from
    the open-loop rollout x^ (x = x^ + dx, dx_0 = 0, q' = Q x^, r' = 0, c' = 0): x, u, K, P and the
    costates agree directly."""
    d = scenes.mass_spring_chain(Nr, M=15, N=20, Nr=Nr, batch=2)
    parent, nx, nu = d["parent"], d["nx"], d["nu"]
    got = _solve(parent, nx, nu, d["Q"], d["R"], d["q"], d["r"], d["A"], d["B"], d["c"], d["x0"])
    n = len(parent)
    leaf = np.ones(n, bool)
    leaf[parent[1:]] = False
    for t in range(2):
        xh = np.zeros((n, nx))
        xh[0] = d["x0"][t]
        for m in range(1, n):
            xh[m] = d["A"][t, m] @ xh[parent[m]]
        qd = np.einsum("nij,nj->ni", d["Q"][t], xh) + d["q"][t]
        K, k, P, pv, dx, du, lam = oracle.tree_lqr(parent, d["Q"][t], np.zeros((n, nu, nx)), d["R"][t], qd,
                                                   d["r"][t], d["A"][t], d["B"][t], np.zeros((n, nx)), edge=True)
        _close(got["x"][t], xh + dx, "x")
        _close(got["u"][t][~leaf], du[~leaf], "u")
        _close(got["K"][t][~leaf], K[~leaf], "K")
        _close(got["P"][t], P, "P")
        _close(got["lam"][t], lam, "lam")


def test_non_positive_definite_h_is_reported_and_cleared():
    """A node whose R makes H indefinite: the solve completes, bmpc_lqr_status reports
    BMPC_ERR_NUMERIC once, and a good solve on the same handle afterwards is clean."""
    from paper_2506_13624_b300 import bmpc, lqr
    rng = np.random.default_rng(7)
    parent = _tree(rng, 10)
    leaf, Q, M, R, q, r, A, B, c = _random_data(rng, parent, 4, 2, 1)
    h = lqr.TreeLQR(parent, 4, 2, batch=1)
    bad = R.copy()
    bad[0, 0] = -50.0 * np.eye(2)
    args = [_dev(a) for a in (Q, bad, q, r, A, B, c, np.zeros((1, 4)))]
    h.solve(*args, check=False)
    assert int(lqr._lib().bmpc_lqr_status(h.handle)) == bmpc.ERR_NUMERIC
    args[1] = _dev(R)
    h.solve(*args, check=False)
    assert int(lqr._lib().bmpc_lqr_status(h.handle)) == bmpc.OK
    h.close()


@pytest.mark.parametrize("nx,nu", [(10, 4), (30, 14)])
def test_schedules_agree_bitwise(nx, nu):
    """The two launch schedules run the same node steps: identical bits."""
    rng = np.random.default_rng(700 + nx)
    parent = _tree(rng, 30)
    leaf, Q, M, R, q, r, A, B, c = _random_data(rng, parent, nx, nu, 2)
    x0 = rng.standard_normal((2, nx))
    a = _solve(parent, nx, nu, Q, R, q, r, A, B, c, x0, M=M, schedule=1)
    b = _solve(parent, nx, nu, Q, R, q, r, A, B, c, x0, M=M, schedule=2)
    for key in a:
        assert np.array_equal(a[key], b[key]), key


def test_wide_stages_agree_bitwise_and_match_the_oracle():
    """Sec. V-A's chain with 32 scenario paths and a batch of six: the last stages hold 192 node steps,
    more than the GPU has SMs, so the launch-per-stage schedule runs them with the two-blocks-per-SM
    instance (whose Cholesky is lane-parallel), and the one-block-per-problem schedule runs every
    node in post-order with the register Cholesky.  Both factorisations do the same operations in the
    same order, so the two schedules agree bit for bit; problem 5 is checked against the oracle."""
    d = scenes.mass_spring_chain(11, M=15, N=10, Nr=5, batch=6)
    parent, nx, nu = d["parent"], d["nx"], d["nu"]
    args = (d["Q"], d["R"], d["q"], d["r"], d["A"], d["B"], d["c"], d["x0"])
    a = _solve(parent, nx, nu, *args, schedule=1)
    b = _solve(parent, nx, nu, *args, schedule=2)
    for key in a:
        assert np.array_equal(a[key], b[key]), key
    n, t = len(parent), 5
    leaf = np.ones(n, bool)
    leaf[parent[1:]] = False
    xh = np.zeros((n, nx))
    xh[0] = d["x0"][t]
    for m in range(1, n):
        xh[m] = d["A"][t, m] @ xh[parent[m]]
    qd = np.einsum("nij,nj->ni", d["Q"][t], xh) + d["q"][t]
    K, k, P, pv, dx, du, lam = oracle.tree_lqr(parent, d["Q"][t], np.zeros((n, nu, nx)), d["R"][t], qd, d["r"][t],
                                               d["A"][t], d["B"][t], np.zeros((n, nx)), edge=True)
    _close(a["x"][t], xh + dx, "x")
    _close(a["u"][t][~leaf], du[~leaf], "u")
    _close(a["K"][t][~leaf], K[~leaf], "K")
    _close(a["P"][t], P, "P")
    _close(a["lam"][t], lam, "lam")
