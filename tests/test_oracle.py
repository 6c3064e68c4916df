"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: closed-form
motion, a textbook steady-state gain, central finite differences, a dense KKT
solve of the tree LQR QP (exactness of the recursion in Sec. III-A), the
discrete algebraic Riccati equation (scipy), the one-step convergence of the
Gauss-Newton/LQR step on a linear-quadratic problem, nonanticipativity and the
value-function summation at branch points, and the KKT conditions of Eq. (bmpc)
at the returned point.
"""
import math

import numpy as np
import pytest
import scipy.linalg

import oracle
import scenes


# ------------------------------------------------------------------ dynamics
def test_kinematic_straight_line_closed_form():
    """delta = 0, constant a: position is quadratic in time, RK4 is exact."""
    p = scenes.config1(0)
    x = np.array([1.0, -2.0, 0.3, 4.0])
    a, dt = 1.5, p["dt"]
    xn, _, _ = oracle.dynamics(p, x, np.array([a, 0.0]))
    s = x[3] * dt + 0.5 * a * dt * dt
    ref = np.array([x[0] + s * math.cos(x[2]), x[1] + s * math.sin(x[2]), x[2], x[3] + a * dt])
    np.testing.assert_allclose(xn, ref, rtol=0, atol=1e-14)


def test_kinematic_circle_closed_form():
    """a = 0, constant steering: circular arc of radius L / tan(delta)."""
    p = scenes.config1(0)
    L, dt = p["params"][0], p["dt"]
    x = np.array([0.0, 0.0, 0.2, 6.0])
    d = 0.3
    xn, _, _ = oracle.dynamics(p, x, np.array([0.0, d]))
    w = x[3] * math.tan(d) / L
    Rc = L / math.tan(d)
    psi1 = x[2] + w * dt
    ref = np.array([x[0] + Rc * (math.sin(psi1) - math.sin(x[2])),
                    x[1] - Rc * (math.cos(psi1) - math.cos(x[2])), psi1, x[3]])
    # classical RK4 local error is O((w dt)^5) * Rc
    np.testing.assert_allclose(xn, ref, rtol=0, atol=1e-8)


def test_dynamic_straight_line_closed_form():
    p = scenes.config3(0)
    x = np.array([3.0, 1.0, -0.4, 7.0, 0.0, 0.0])
    a, dt = -2.0, p["dt"]
    xn, _, _ = oracle.dynamics(p, x, np.array([a, 0.0]))
    s = x[3] * dt + 0.5 * a * dt * dt
    ref = np.array([x[0] + s * math.cos(x[2]), x[1] + s * math.sin(x[2]), x[2], x[3] + a * dt, 0.0, 0.0])
    np.testing.assert_allclose(xn, ref, rtol=0, atol=1e-13)


def test_dynamic_bicycle_steady_state_yaw_gain():
    """Linear single-track model: r_ss = u delta / (L + K u^2), K = m (lr Cr - lf Cf) / (L Cf Cr)."""
    p = scenes.config3(0)
    L_, m, Iz, lf, lr, Cf, Cr = p["params"][:7]
    u0, d = 8.0, 0.004
    x = np.array([0.0, 0.0, 0.0, u0, 0.0, 0.0])
    for _ in range(60):
        x, _, _ = oracle.dynamics(p, x, np.array([0.0, d]))
    L = lf + lr
    K = m * (lr * Cr - lf * Cf) / (L * Cf * Cr)
    r_ss = x[3] * d / (L + K * x[3] ** 2)
    assert abs(x[5] - r_ss) < 2e-3 * abs(r_ss)


def test_unicycle_straight_line_closed_form():
    """omega = 0, constant a: the unicycle moves on a straight line, quadratic in time (RK4 exact)."""
    p = scenes.unicycle(0)
    x = np.array([1.0, -2.0, 0.3, 1.5])
    a, dt = 1.2, p["dt"]
    xn, _, _ = oracle.dynamics(p, x, np.array([a, 0.0]))
    s = x[3] * dt + 0.5 * a * dt * dt
    ref = np.array([x[0] + s * math.cos(x[2]), x[1] + s * math.sin(x[2]), x[2], x[3] + a * dt])
    np.testing.assert_allclose(xn, ref, rtol=0, atol=1e-14)


def test_unicycle_circle_closed_form():
    """a = 0, constant omega: a circular arc of radius v / omega, heading advancing by omega dt."""
    p = scenes.unicycle(0)
    dt = p["dt"]
    x = np.array([0.5, 0.0, -0.4, 2.0])
    w = 1.1
    xn, _, _ = oracle.dynamics(p, x, np.array([0.0, w]))
    Rc = x[3] / w
    th1 = x[2] + w * dt
    ref = np.array([x[0] + Rc * (math.sin(th1) - math.sin(x[2])),
                    x[1] - Rc * (math.cos(th1) - math.cos(x[2])), th1, x[3]])
    np.testing.assert_allclose(xn, ref, rtol=0, atol=1e-8)


@pytest.mark.parametrize("cfg", [1, 3, "unicycle"])
def test_jacobians_central_differences(cfg):
    p = scenes.unicycle(1) if cfg == "unicycle" else scenes.instances(cfg, 1)[0]
    rng = np.random.default_rng(7 if cfg == "unicycle" else cfg)
    nx = p["nx"]
    for _ in range(5):
        x = p["x0"] + 0.5 * rng.standard_normal(nx)
        u = 0.3 * rng.standard_normal(2)
        _, A, B = oracle.dynamics(p, x, u)
        h = 1e-6
        Afd = np.stack([(oracle.dynamics(p, x + h * e, u)[0] - oracle.dynamics(p, x - h * e, u)[0]) / (2 * h)
                        for e in np.eye(nx)], 1)
        Bfd = np.stack([(oracle.dynamics(p, x, u + h * e)[0] - oracle.dynamics(p, x, u - h * e)[0]) / (2 * h)
                        for e in np.eye(2)], 1)
        np.testing.assert_allclose(A, Afd, rtol=0, atol=1e-6 * max(1.0, np.abs(A).max()))
        np.testing.assert_allclose(B, Bfd, rtol=0, atol=1e-6 * max(1.0, np.abs(B).max()))


# ------------------------------------------------------------------ constraints
def test_ellipse_constraint_boundary_and_jacobian():
    p = scenes.config2(0)
    i = 5
    cx, cy, hd, a, b = p["obs"][i, 0]
    rows = 4
    for t in np.linspace(0, 2 * math.pi, 7):
        X = cx + a * math.cos(t) * math.cos(hd) - b * math.sin(t) * math.sin(hd)
        Y = cy + a * math.cos(t) * math.sin(hd) + b * math.sin(t) * math.cos(hd)
        g, Jx, Ju, ex = oracle.constraints(p, i, False, np.array([X, Y, 0, 0]), np.zeros(2))
        assert abs(g[rows]) < 1e-6          # on the ellipse: normalised distance 1
        x = np.array([X + 0.3, Y - 0.2, 0.0, 0.0])
        g0, Jx0, _, _ = oracle.constraints(p, i, False, x, np.zeros(2))
        h = 1e-6
        fd = [(oracle.constraints(p, i, False, x + h * e, np.zeros(2))[0][rows]
               - oracle.constraints(p, i, False, x - h * e, np.zeros(2))[0][rows]) / (2 * h) for e in np.eye(4)]
        np.testing.assert_allclose(Jx0[rows], fd, atol=1e-7)
    g, _, _, ex = oracle.constraints(p, i, False, np.array([cx, cy, 0, 0]), np.zeros(2))
    assert abs(g[rows] - 1.0) < 2e-3 and ex[rows]
    g, _, _, ex = oracle.constraints(p, 0, False, np.array([cx, cy, 0, 0]), np.array([5.0, 0.0]))
    assert not ex[rows] and ex[0] and abs(g[0] - 2.0) < 1e-12      # root: no state rows, box exists
    g, _, _, ex = oracle.constraints(p, p["n"] - 1, True, np.array([cx, cy, 0, 0]), np.zeros(2))
    assert not ex[:4].any() and ex[rows]                              # leaf: no input rows


# ------------------------------------------------------------------ tree LQR
def _random_tree(rng, n_max=30):
    """Level-ordered tree with random fan-out 0..3 and leaves at ragged depths."""
    parent = [-1]
    frontier = [0]
    while frontier and len(parent) < n_max:
        nxt = []
        for q in frontier:
            for _ in range(int(rng.integers(1 if q == 0 else 0, 4))):
                if len(parent) >= n_max:
                    break
                parent.append(q)
                nxt.append(len(parent) - 1)
        frontier = nxt
    return np.array(parent, np.int32)


def _random_lqr(rng, parent, nx, nu):
    n = len(parent)
    leaf = np.ones(n, bool)
    leaf[parent[1:]] = False
    Q, M, R = np.zeros((n, nx, nx)), np.zeros((n, nu, nx)), np.zeros((n, nu, nu))
    for i in range(n):
        F = rng.standard_normal((nx + nu, nx + nu))
        W = F @ F.T + 0.2 * np.eye(nx + nu)
        Q[i] = W[:nx, :nx]
        if not leaf[i]:
            M[i], R[i] = W[nx:, :nx], W[nx:, nx:]
    q, r = rng.standard_normal((n, nx)), rng.standard_normal((n, nu)) * (~leaf)[:, None]
    A = np.eye(nx) + 0.3 * rng.standard_normal((n, nx, nx))
    B = rng.standard_normal((n, nx, nu))
    c = rng.standard_normal((n, nx))
    c[0] = 0
    return leaf, Q, M, R, q, r, A, B, c


def _dense_kkt(parent, leaf, Q, M, R, q, r, A, B, c, edge=False):
    """Dense KKT system of Eq. (lqr_tree_approx) with dx_0 = 0: returns dx, du, lam.  A, B per parent,
    or per edge (row m: the edge into m) with edge=True."""
    n, nx, nu = len(parent), Q.shape[1], R.shape[1]
    uidx = {}
    off = n * nx
    for i in range(n):
        if not leaf[i]:
            uidx[i] = off
            off += nu
    nz = off
    H = np.zeros((nz, nz))
    h = np.zeros(nz)
    for i in range(n):
        xi = slice(i * nx, (i + 1) * nx)
        H[xi, xi] += Q[i]
        h[xi] += q[i]
        if not leaf[i]:
            ui = slice(uidx[i], uidx[i] + nu)
            H[ui, ui] += R[i]
            H[ui, xi] += M[i]
            H[xi, ui] += M[i].T
            h[ui] += r[i]
    ncon = n * nx
    E = np.zeros((ncon, nz))
    e = np.zeros(ncon)
    E[0:nx, 0:nx] = np.eye(nx)                      # dx_0 = 0
    for m in range(1, n):
        pnt = parent[m]
        rows = slice(m * nx, (m + 1) * nx)
        E[rows, m * nx:(m + 1) * nx] = np.eye(nx)
        E[rows, pnt * nx:(pnt + 1) * nx] -= A[m] if edge else A[pnt]
        E[rows, uidx[pnt]:uidx[pnt] + nu] -= B[m] if edge else B[pnt]
        e[rows] = c[m]
    K = np.block([[H, E.T], [E, np.zeros((ncon, ncon))]])
    sol = np.linalg.solve(K, np.concatenate([-h, e]))
    z, nu_ = sol[:nz], sol[nz:]
    dx = z[:n * nx].reshape(n, nx)
    du = np.zeros((n, nu))
    for i, o in uidx.items():
        du[i] = z[o:o + nu]
    lam = -nu_.reshape(n, nx)        # lambda multiplies (A dx + B du + c - dx_m)
    return dx, du, lam


@pytest.mark.parametrize("seed", range(8))
def test_tree_lqr_equals_dense_kkt(seed):
    rng = np.random.default_rng(100 + seed)
    nx, nu = (4, 2) if seed % 2 == 0 else (3, 1)
    parent = _random_tree(rng)
    leaf, Q, M, R, q, r, A, B, c = _random_lqr(rng, parent, nx, nu)
    K, k, P, pv, dx, du, lam = oracle.tree_lqr(parent, Q, M, R, q, r, A, B, c)
    dx2, du2, lam2 = _dense_kkt(parent, leaf, Q, M, R, q, r, A, B, c)
    scale = max(1.0, np.abs(dx2).max(), np.abs(lam2).max())
    np.testing.assert_allclose(dx, dx2, atol=1e-10 * scale)
    np.testing.assert_allclose(du, du2, atol=1e-10 * scale)
    np.testing.assert_allclose(lam[1:], lam2[1:], atol=1e-10 * scale)


@pytest.mark.parametrize("seed", range(8))
def test_per_edge_tree_lqr_equals_dense_kkt(seed):
    """Per-branch dynamics (Sec. V-A's trees: every edge its own A_m, B_m): the tree Riccati recursion
    and the scan form both equal the dense KKT solution of the tree LQR with per-edge matrices."""
    rng = np.random.default_rng(200 + seed)
    nx, nu = (4, 2) if seed % 2 == 0 else (3, 1)
    parent = _random_tree(rng) if seed < 4 else _scan_case_tree(seed)[1]
    leaf, Q, M, R, q, r, A, B, c = _random_lqr(rng, parent, nx, nu)
    n = len(parent)
    Ae = np.eye(nx) + 0.3 * rng.standard_normal((n, nx, nx))     # a different matrix on every edge
    Be = rng.standard_normal((n, nx, nu))
    dx2, du2, lam2 = _dense_kkt(parent, leaf, Q, M, R, q, r, Ae, Be, c, edge=True)
    scale = max(1.0, np.abs(dx2).max(), np.abs(lam2).max())
    for fn in (oracle.tree_lqr, oracle.tree_lqr_scan):
        K, k, P, pv, dx, du, lam = fn(parent, Q, M, R, q, r, Ae, Be, c, edge=True)
        np.testing.assert_allclose(dx, dx2, atol=1e-9 * scale)
        np.testing.assert_allclose(du, du2, atol=1e-9 * scale)
        np.testing.assert_allclose(lam[1:], lam2[1:], atol=1e-9 * scale)
    # with the parent's matrices copied to every edge the per-edge path is the per-parent one
    Ap = np.array([A[parent[m]] if m else A[0] for m in range(n)])
    Bp = np.array([B[parent[m]] if m else B[0] for m in range(n)])
    got = oracle.tree_lqr(parent, Q, M, R, q, r, Ap, Bp, c, edge=True)
    ref = oracle.tree_lqr(parent, Q, M, R, q, r, A, B, c)
    for a, b in zip(got, ref):
        np.testing.assert_allclose(a, b, atol=1e-12 * max(1.0, np.abs(b).max()))


@pytest.mark.parametrize("nx,nu", [(10, 4), (30, 14), (32, 16)])
def test_per_edge_tree_lqr_at_the_mass_spring_sizes(nx, nu):
    """The tree Riccati recursion with per-edge matrices at the state and input dimensions of Sec.
    V-A's mass-spring chains (n_x = 2M, n_u = M - 1) and the largest supported: equal to the dense
    KKT solution."""
    rng = np.random.default_rng(300 + nx)
    parent = _random_tree(rng, n_max=14)
    leaf, Q, M, R, q, r, A, B, c = _random_lqr(rng, parent, nx, nu)
    n = len(parent)
    Ae = np.eye(nx) + (0.3 / np.sqrt(nx)) * rng.standard_normal((n, nx, nx))
    Be = rng.standard_normal((n, nx, nu)) / np.sqrt(nx)
    dx2, du2, lam2 = _dense_kkt(parent, leaf, Q, M, R, q, r, Ae, Be, c, edge=True)
    K, k, P, pv, dx, du, lam = oracle.tree_lqr(parent, Q, M, R, q, r, Ae, Be, c, edge=True)
    scale = max(1.0, np.abs(dx2).max(), np.abs(lam2).max())
    np.testing.assert_allclose(dx, dx2, atol=1e-9 * scale)
    np.testing.assert_allclose(du, du2, atol=1e-9 * scale)
    np.testing.assert_allclose(lam[1:], lam2[1:], atol=1e-9 * scale)


def _dense_lq_solution(p):
    """The whole LQ problem of a per-edge linear tree (no constraints) as one equality-constrained QP:
    min sum_i w_i [1/2 (x_i - xref_i)' Q (x_i - xref_i) + 1/2 u_i' R u_i] s.t. x_0 = x-bar,
    x_m = A_m x_p(m) + B_m u_p(m); returns x, u."""
    n, nx, nu, par = p["n"], p["nx"], p["nu"], p["parent"]
    leaf = np.ones(n, bool)
    leaf[par[1:]] = False
    nz = n * (nx + nu)
    H, h = np.zeros((nz, nz)), np.zeros(nz)
    xs = lambda i: slice(i * nx, (i + 1) * nx)
    us = lambda i: slice(n * nx + i * nu, n * nx + (i + 1) * nu)
    for i in range(n):
        Qd = np.diag(p["QNw"] if leaf[i] else p["Qw"]) * p["weight"][i]
        H[xs(i), xs(i)] = Qd
        h[xs(i)] = -Qd @ p["xref"][i]
        H[us(i), us(i)] = np.diag(p["Rw"]) * p["weight"][i] if not leaf[i] else np.eye(nu)
    rows = []
    rhs = []
    E0 = np.zeros((nx, nz))
    E0[:, xs(0)] = np.eye(nx)
    rows.append(E0)
    rhs.append(p["x0"])
    for m in range(1, n):
        Em = np.zeros((nx, nz))
        Em[:, xs(m)] = np.eye(nx)
        Em[:, xs(par[m])] -= p["Aedge"][m]
        Em[:, us(par[m])] -= p["Bedge"][m]
        rows.append(Em)
        rhs.append(np.zeros(nx))
    for i in np.where(leaf)[0]:          # leaves have no input: pin it to zero
        El = np.zeros((nu, nz))
        El[:, us(i)] = np.eye(nu)
        rows.append(El)
        rhs.append(np.zeros(nu))
    E, e = np.vstack(rows), np.concatenate(rhs)
    Kk = np.block([[H, E.T], [E, np.zeros((E.shape[0], E.shape[0]))]])
    z = np.linalg.solve(Kk, np.concatenate([-h, e]))[:nz]
    return z[:n * nx].reshape(n, nx), z[n * nx:].reshape(n, nu)


@pytest.mark.parametrize("seed,N,Nr", [(0, 20, 2), (1, 12, 3), (2, 30, 5)])
def test_per_edge_lq_solve_is_the_qp_solution(seed, N, Nr):
    """The mass-spring tree with a spring constant per branch (Sec. V-A): one iteration of the method
    reaches the solution of the whole QP, solved here as one dense equality-constrained system."""
    p = scenes.mass_spring(seed, N=N, Nr=Nr)
    r = oracle.solve(p)
    assert r["status"] == oracle.OK and r["inner_iters"] == 1
    x, u = _dense_lq_solution(p)
    leaf = np.ones(p["n"], bool)
    leaf[p["parent"][1:]] = False
    np.testing.assert_allclose(r["x"], x, atol=1e-9 * max(1.0, np.abs(x).max()))
    np.testing.assert_allclose(r["u"][~leaf], u[~leaf], atol=1e-9 * max(1.0, np.abs(u).max()))


def test_per_edge_model_changes_the_plan_only_after_the_split():
    """Two trees that differ only in one branch's spring constant plan the same root input up to the
    hedging the tree imposes, and the branches' states differ only below the split."""
    p = scenes.mass_spring(4, N=15, Nr=1)
    q = dict(p)
    q["Aedge"] = p["Aedge"].copy()
    first_child = int(np.where(p["parent"] == 0)[0][0])
    chain = [first_child]
    while True:
        nxt = np.where(p["parent"] == chain[-1])[0]
        if len(nxt) == 0:
            break
        chain.append(int(nxt[0]))
    Kc = np.array([[-2.0 * 3.0, 3.0], [3.0, -2.0 * 3.0]])
    Ac = np.block([[np.zeros((2, 2)), np.eye(2)], [Kc, np.zeros((2, 2))]])
    A3, _ = scenes.generator._rk4_linear(Ac, np.vstack([np.zeros((2, 2)), np.eye(2)]), 0.1)
    for m in chain:
        q["Aedge"][m] = scenes.f32(A3)
    rp, rq = oracle.solve(p), oracle.solve(q)
    assert rp["status"] == rq["status"] == oracle.OK
    assert np.abs(rp["u"][0] - rq["u"][0]).max() > 1e-6          # the root hedges over both models
    assert np.abs(rp["x"][chain[0]] - rq["x"][chain[0]]).max() > 1e-6


def test_single_path_riccati_reaches_dare():
    rng = np.random.default_rng(7)
    nx, nu, N = 4, 2, 400
    A1 = np.eye(nx) + 0.1 * rng.standard_normal((nx, nx))
    B1 = rng.standard_normal((nx, nu))
    F = rng.standard_normal((nx, nx))
    Q1 = F @ F.T + np.eye(nx)
    R1 = np.diag([0.5, 2.0])
    parent = np.arange(-1, N, dtype=np.int32)
    n = N + 1
    Q = np.repeat(Q1[None], n, 0)
    R = np.repeat(R1[None], n, 0)
    R[-1] = 0
    M = np.zeros((n, nu, nx))
    A = np.repeat(A1[None], n, 0)
    B = np.repeat(B1[None], n, 0)
    K, k, P, pv, dx, du, lam = oracle.tree_lqr(parent, Q, M, R, np.zeros((n, nx)), np.zeros((n, nu)),
                                               A, B, np.zeros((n, nx)))
    Pd = scipy.linalg.solve_discrete_are(A1, B1, Q1, R1)
    np.testing.assert_allclose(P[0], Pd, rtol=1e-9, atol=1e-9 * np.abs(Pd).max())
    Kd = -np.linalg.solve(R1 + B1.T @ Pd @ B1, B1.T @ Pd @ A1)
    np.testing.assert_allclose(K[0], Kd, rtol=1e-8, atol=1e-9)


# ------------------------------------------------------------------ iLQR step, merit
def test_lq_problem_converges_in_one_iteration():
    p = scenes.linear_problem(3, N=12, splits={2: 2, 6: 3})
    r = oracle.solve(p)
    assert r["status"] == oracle.OK
    assert r["inner_iters"] == 1
    k = oracle.kkt(p, r["x"], r["u"], r["lam"], r["y"])
    assert k.max() < 1e-11


def test_lq_full_step_merit_identity():
    """For linear dynamics and quadratic cost phi(1) - phi(0) = phi'(0)/2 exactly."""
    p = scenes.linear_problem(4, N=8, splits={3: 2})
    x, u, lam, y = oracle.cold_start(p)
    x[0] = p["x0"]
    lam = 0.1 * np.random.default_rng(0).standard_normal(lam.shape)
    lam[0] = 0
    dx, du, dl, info = oracle.direction(p, x, u, lam, y, 10.0, 3.0)
    phi1 = oracle.merit(p, x + dx, u + du, lam + dl, y, 10.0, 3.0)
    assert abs((phi1 - info[0]) - 0.5 * info[1]) < 1e-9 * max(1.0, abs(info[1]))
    # and the closed form phi'(0; 0) = -dz'W dz + 2 dlam'd of the exact QP step
    nx = p["nx"]
    d = np.zeros_like(x)
    for m in range(1, p["n"]):
        pn = p["parent"][m]
        d[m] = oracle.dynamics(p, x[pn], u[pn])[0] - x[m]
    assert abs(info[4] - (-info[2] + 2 * np.sum(dl[1:] * d[1:]))) < 1e-9 * max(1.0, abs(info[4]))
    assert nx == 4


@pytest.mark.parametrize("cfg", [1, 2])
def test_merit_directional_derivative_matches_central_difference(cfg):
    p = scenes.instances(cfg, 1, seed0=5)[0]
    x, u, lam, y = oracle.cold_start(p)
    x[0] = p["x0"]
    rng = np.random.default_rng(1)
    lam = 0.05 * rng.standard_normal(lam.shape)
    lam[0] = 0
    y = np.abs(0.1 * rng.standard_normal(y.shape))
    rho, mu = 10.0, 2.0
    dx, du, dl, info = oracle.direction(p, x, u, lam, y, rho, mu)
    h = 1e-6
    fp = oracle.merit(p, x + h * dx, u + h * du, lam + h * dl, y, rho, mu)
    fm = oracle.merit(p, x - h * dx, u - h * du, lam - h * dl, y, rho, mu)
    fd = (fp - fm) / (2 * h)
    assert abs(fd - info[1]) < 1e-6 * max(1.0, abs(info[1]))
    assert info[0] == pytest.approx(oracle.merit(p, x, u, lam, y, rho, mu), rel=1e-14)


# ------------------------------------------------------------------ tree structure
def test_identical_branches_are_bitwise_equal():
    """Nonanticipativity is exact: with stage-only data, all scenarios coincide bit for bit."""
    p = scenes.linear_problem(5, N=10, splits={2: 3, 5: 2})
    st = p["stage"]
    xr = np.zeros((st.max() + 1, p["nx"]))
    for i in range(p["n"]):
        xr[st[i]] = p["xref"][i]
    p["xref"] = xr[st]
    r = oracle.solve(p)
    for k in range(st.max() + 1):
        rows = r["x"][st == k]
        assert (rows == rows[0]).all()


def test_branch_value_functions_sum():
    """b identical children of weight w/b give the same plan as one child of weight w."""
    base = scenes.linear_problem(6, N=9, splits={})
    tree = scenes.linear_problem(6, N=9, splits={4: 3})
    for q in (base, tree):
        st = q["stage"]
        q["xref"] = base["xref"][st]
        q["weight"] = scenes.branch_weights(q["parent"])
    rb, rt = oracle.solve(base), oracle.solve(tree)
    st = tree["stage"]
    first = {}
    for i in range(tree["n"]):
        first.setdefault(st[i], i)
    for k, i in first.items():
        np.testing.assert_allclose(rt["x"][i], rb["x"][k], atol=1e-10)
        if k < st.max():
            np.testing.assert_allclose(rt["u"][i], rb["u"][k], atol=1e-10)


# ------------------------------------------------------------------ AL method, KKT
@pytest.mark.parametrize("cfg,seed", [(1, 0), (1, 1), (1, 2), (2, 0), (2, 3)])
def test_al_reaches_kkt_of_original_problem(cfg, seed):
    p = scenes.instances(cfg, 1, seed0=seed)[0]
    r = oracle.solve(p)
    assert r["status"] == oracle.OK
    k = oracle.kkt(p, r["x"], r["u"], r["lam"], r["y"])
    assert k[:4].max() < 1e-5                  # stationarity, defects, feasibility, complementarity
    assert (r["y"] >= 0).all() and k[4] == 0.0


def _objective(p, x, u):
    return oracle.aug_lagrangian(p, x, u, np.zeros((p["n"], oracle.n_con(p))), 1e-300)


def test_stationarity_by_finite_differences():
    """grad of sum(l) + y'g + lam'd vanishes at the returned point (FD, independent of the KKT code)."""
    p = scenes.config1(3)
    r = oracle.solve(p)
    assert r["status"] == oracle.OK
    x, u, lam, y = r["x"], r["u"], r["lam"], r["y"]
    n, nx, nu = p["n"], p["nx"], p["nu"]
    ch = [[] for _ in range(n)]
    for i in range(1, n):
        ch[p["parent"][i]].append(i)

    def lagr(xx, uu):
        v = _objective(p, xx, uu)
        for i in range(n):
            g, _, _, ex = oracle.constraints(p, i, not ch[i], xx[i], uu[i])
            v += float(np.sum(y[i][ex] * g[ex]))
            if ch[i]:
                f = oracle.dynamics(p, xx[i], uu[i])[0]
                for m in ch[i]:
                    v += float(lam[m] @ (f - xx[m]))
        return v

    h = 1e-5
    worst = 0.0
    rng = np.random.default_rng(0)
    for i in rng.choice(np.arange(1, n), 12, replace=False):
        for j in range(nx):
            xp, xm = x.copy(), x.copy()
            xp[i, j] += h
            xm[i, j] -= h
            worst = max(worst, abs((lagr(xp, u) - lagr(xm, u)) / (2 * h)))
        if ch[i]:
            for j in range(nu):
                up, um = u.copy(), u.copy()
                up[i, j] += h
                um[i, j] -= h
                worst = max(worst, abs((lagr(x, up) - lagr(x, um)) / (2 * h)))
    assert worst < 2e-5


def test_inactive_constraints_give_zero_multipliers():
    """Obstacles moved far away: same plan as without them and y = 0 on their rows."""
    p = scenes.config1(4)
    far = dict(p)
    far["obs"] = p["obs"].copy()
    far["obs"][:, :, 1] += 1000.0
    none = dict(p)
    none["obs"] = p["obs"][:, :0, :]
    none["n_obs"] = 0
    rf, rn = oracle.solve(far), oracle.solve(none)
    assert rf["status"] == oracle.OK and rn["status"] == oracle.OK
    np.testing.assert_allclose(rf["u"], rn["u"], atol=1e-7)
    assert (rf["y"][:, 4] == 0).all()


def test_invalid_tree_rejected():
    p = scenes.config1(0)
    bad = dict(p)
    par = p["parent"].copy()
    par[5] = 7                       # parent after child: not level ordered
    bad["parent"] = par
    r = oracle.solve(bad)
    assert r["status"] == -1


# ------------------------------------------------------------------ learned warm-start network (reference)
def test_mlp_reference_gradients_match_central_differences():
    from oracle import mlp_ref
    rng = np.random.default_rng(0)
    dims = [7, 9, 6, 5]
    Ws = [0.5 * rng.standard_normal((a, b)) for a, b in zip(dims[:-1], dims[1:])]
    bs = [0.1 * rng.standard_normal(b) for b in dims[1:]]
    x = rng.standard_normal((4, dims[0]))
    t = rng.standard_normal((4, dims[-1]))
    loss, dWs, dbs = mlp_ref.loss_and_grads(Ws, bs, x, t, bf=False)
    h = 1e-6
    for l in range(len(Ws)):
        for (i, j) in [(0, 0), (dims[l] - 1, dims[l + 1] - 1), (2, 1)]:
            Wp = [W.copy() for W in Ws]
            Wm = [W.copy() for W in Ws]
            Wp[l][i, j] += h
            Wm[l][i, j] -= h
            fd = (mlp_ref.loss_and_grads(Wp, bs, x, t, bf=False)[0] - mlp_ref.loss_and_grads(Wm, bs, x, t, bf=False)[0]) / (2 * h)
            assert abs(fd - dWs[l][i, j]) < 1e-6 * max(1.0, abs(fd))
        bp = [b.copy() for b in bs]
        bm = [b.copy() for b in bs]
        bp[l][1] += h
        bm[l][1] -= h
        fd = (mlp_ref.loss_and_grads(Ws, bp, x, t, bf=False)[0] - mlp_ref.loss_and_grads(Ws, bm, x, t, bf=False)[0]) / (2 * h)
        assert abs(fd - dbs[l][1]) < 1e-6 * max(1.0, abs(fd))


def test_gelu_and_bf16_rounding():
    from oracle import mlp_ref
    x = np.linspace(-4, 4, 41)
    h = 1e-6
    fd = (mlp_ref.gelu(x + h) - mlp_ref.gelu(x - h)) / (2 * h)
    np.testing.assert_allclose(mlp_ref.gelu_grad(x), fd, atol=1e-8)
    assert mlp_ref.gelu(np.array([0.0]))[0] == 0.0 and abs(mlp_ref.gelu(np.array([10.0]))[0] - 10.0) < 1e-12
    # bfloat16: 8 significant bits, ties to even
    assert mlp_ref.bf16(1.0 + 2.0 ** -8) == 1.0                 # tie -> even (1.0)
    assert mlp_ref.bf16(1.0 + 3 * 2.0 ** -8) == 1.0 + 2.0 ** -6  # tie -> even (1 + 2^-6)
    assert mlp_ref.bf16(1.0 + 2.0 ** -7) == 1.0 + 2.0 ** -7      # exactly representable
    assert mlp_ref.bf16(-3.0) == -3.0


def test_adamw_first_step_closed_form():
    """AdamW's bias-corrected first step moves every weight by lr (g / (|g| + eps) + wd w)."""
    from oracle import mlp_ref
    rng = np.random.default_rng(7)
    w, g = rng.standard_normal(50), rng.standard_normal(50)
    lr, wd, eps = 1e-3, 0.1, 1e-8
    w1, m1, v1 = mlp_ref.adamw(w, np.zeros(50), np.zeros(50), g, 1, lr, wd, eps=eps)
    np.testing.assert_allclose(w1, w - lr * (g / (np.abs(g) + eps) + wd * w), rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(m1, 0.1 * g, rtol=1e-12)
    np.testing.assert_allclose(v1, 0.001 * g * g, rtol=1e-12)


# ------------------------------------------------------------------ tree LQR by scans (Sec. III-B)
def _scan_case_tree(seed):
    """Ragged random trees (short segments), single paths (one long segment: several scan levels)
    and branch-point trees shaped like the driving scenes (long segments after the splits)."""
    rng = np.random.default_rng(300 + seed)
    kind = seed % 4
    if kind == 0:
        return rng, _random_tree(rng)
    if kind == 1:
        return rng, np.arange(-1, 20 + 13 * (seed // 4), dtype=np.int32)
    from scenes.generator import tree_parents
    splits = {1: 3} if kind == 2 else {1: 2, 4: 2, 9: 2}
    parent, _ = tree_parents(12 + seed, splits)
    return rng, np.asarray(parent, np.int32)


@pytest.mark.parametrize("seed", range(12))
def test_scan_tree_lqr_equals_riccati_and_dense_kkt(seed):
    """The segment-wise CVF scans with tree Riccati steps at branch nodes and the path-wise forward
    scans reproduce the sequential tree Riccati recursion (value functions, laws, rollout) and the
    dense KKT solution; the scans combine the elements in a different association than the
    sequential recursion, so this also checks the associativity of the combination rule."""
    rng, parent = _scan_case_tree(seed)
    nx, nu = (4, 2) if seed % 2 == 0 else (3, 1)
    leaf, Q, M, R, q, r, A, B, c = _random_lqr(rng, parent, nx, nu)
    ref = oracle.tree_lqr(parent, Q, M, R, q, r, A, B, c)
    got = oracle.tree_lqr_scan(parent, Q, M, R, q, r, A, B, c)
    for name, a, b in zip(("K", "k", "P", "p", "dx", "du", "lam"), got, ref):
        scale = max(1.0, np.abs(b).max())
        np.testing.assert_allclose(a, b, atol=1e-9 * scale, err_msg=name)
    if len(parent) <= 60:
        dx2, du2, lam2 = _dense_kkt(parent, leaf, Q, M, R, q, r, A, B, c)
        scale = max(1.0, np.abs(dx2).max(), np.abs(lam2).max())
        np.testing.assert_allclose(got[4], dx2, atol=1e-9 * scale)
        np.testing.assert_allclose(got[5], du2, atol=1e-9 * scale)
        np.testing.assert_allclose(got[6][1:], lam2[1:], atol=1e-9 * scale)


@pytest.mark.parametrize("cfg,seed", [(1, 0), (1, 5), (2, 3), (0, 4)])
def test_full_solve_with_scan_lqr_equals_riccati(cfg, seed):
    """The whole AL-iLQR solve with its search direction from the scans of Sec. III-B takes the same
    iterations to the same point as with the sequential tree Riccati recursion: the scan form
    replaces the recursion inside the method, not only on random LQ data."""
    p = scenes.linear_problem(seed, N=14, splits={3: 2, 7: 3}, constrained=True) if cfg == 0 else \
        scenes.instances(cfg, 1, seed0=seed)[0]
    a = oracle.solve(p)
    b = oracle.solve(p, lqr_scan=1)
    assert a["status"] == b["status"]
    assert (a["inner_iters"], a["outer_iters"]) == (b["inner_iters"], b["outer_iters"])
    for key in ("x", "u", "lam", "y"):
        scale = max(1.0, np.abs(a[key]).max())
        np.testing.assert_allclose(b[key], a[key], atol=1e-8 * scale, err_msg=key)


# ------------------------------------------------------------------ exact Hessian option (Sec. IV-A)
@pytest.mark.parametrize("cfg", [1, 3, "unicycle"])
def test_dynamics_second_derivatives_match_differences_of_the_jacobian(cfg):
    """sum_i mu_i d^2 f_i / dz dz of the RK4 map by hyper-dual numbers against central differences of
    the analytic Jacobian (itself pinned by central differences of f)."""
    p = scenes.unicycle(1) if cfg == "unicycle" else scenes.instances(cfg, 1)[0]
    rng = np.random.default_rng(11)
    nx, nu = p["nx"], p["nu"]
    for _ in range(3):
        x = p["x0"] + 0.5 * rng.standard_normal(nx)
        u = 0.3 * rng.standard_normal(nu)
        mu = rng.standard_normal(nx)
        H = oracle.dyn_hessian(p, x, u, mu)
        assert np.allclose(H, H.T)
        h = 1e-5
        cols = []
        for j in range(nx + nu):
            e = np.zeros(nx + nu)
            e[j] = h
            _, Ap, Bp = oracle.dynamics(p, x + e[:nx], u + e[nx:])
            _, Am, Bm = oracle.dynamics(p, x - e[:nx], u - e[nx:])
            Jp, Jm = np.hstack([Ap, Bp]), np.hstack([Am, Bm])
            cols.append(mu @ (Jp - Jm) / (2 * h))
        Hfd = np.array(cols).T
        np.testing.assert_allclose(H, Hfd, rtol=0, atol=1e-6 * max(1.0, np.abs(H).max()))
        assert np.abs(H[:2]).max() == 0.0 or p["model"] == 2   # positions do not enter the vehicle dynamics


def test_keep_out_curvature_matches_differences_of_the_gradient():
    p = scenes.config1(0)
    ob = p["obs"][5, 0]
    for X, Y in ((ob[0] + 2.0, ob[1] + 0.7), (ob[0] - 1.0, ob[1] - 1.6), (ob[0] + 3.5, ob[1])):
        hxy = oracle.obs_hessian(ob, X, Y)
        h = 1e-5
        x = np.array([X, Y, 0.0, 1.0])
        grads = []
        for e in (np.array([h, 0, 0, 0]), np.array([0, h, 0, 0])):
            q = dict(p)
            _, Jp, _, _ = oracle.constraints(q, 5, False, x + e, np.zeros(2))
            _, Jm, _, _ = oracle.constraints(q, 5, False, x - e, np.zeros(2))
            grads.append((Jp[4, :2] - Jm[4, :2]) / (2 * h))
        fd = np.array(grads)
        np.testing.assert_allclose([hxy[0], hxy[1], hxy[2]], [fd[0, 0], fd[0, 1], fd[1, 1]], atol=1e-6)


@pytest.mark.parametrize("n", [3, 6, 8])
def test_jacobi_eigen_decomposition_and_modification(n):
    """The cyclic Jacobi eigen-decomposition against numpy's symmetric eigensolver, and the eigenvalue
    modification: positive definite afterwards, eigenvectors kept, eigenvalues above the floor kept."""
    rng = np.random.default_rng(n)
    F = rng.standard_normal((n, n))
    S = F + F.T
    ev, V = oracle.jacobi_eig(S)
    np.testing.assert_allclose(np.sort(ev), np.linalg.eigvalsh(S), atol=1e-12 * np.abs(ev).max())
    np.testing.assert_allclose(V @ np.diag(ev) @ V.T, S, atol=1e-12 * np.abs(S).max())
    np.testing.assert_allclose(V.T @ V, np.eye(n), atol=1e-12)
    Sm = oracle.eig_modify(S)
    em = np.linalg.eigvalsh(Sm)
    floor = 1e-6 * max(1.0, np.abs(ev).max())
    assert em.min() >= floor * (1 - 1e-9)
    keep = np.sort(ev[ev > floor])
    np.testing.assert_allclose(em[-len(keep):], keep, atol=1e-10 * np.abs(ev).max())
    Spd = F @ F.T + np.eye(n)
    np.testing.assert_allclose(oracle.eig_modify(Spd), Spd, atol=1e-10 * np.abs(Spd).max())


@pytest.mark.parametrize("cfg,seed", [(1, 0), (1, 3), (2, 1), ("unicycle", 2)])
def test_exact_hessian_solves_reach_the_kkt_point(cfg, seed):
    """With the exact Hessian (eigenvalue-modified) the method reaches a KKT point of Eq. (bmpc), the
    same one as with Gauss-Newton."""
    p = scenes.unicycle(seed) if cfg == "unicycle" else scenes.instances(cfg, 1, seed0=seed)[0]
    a, b = oracle.solve(p), oracle.solve(p, hessian=1)
    assert a["status"] == b["status"] == oracle.OK
    k = oracle.kkt(p, b["x"], b["u"], b["lam"], b["y"])
    assert k[:4].max() < 1e-5
    inner = np.ones(p["n"], bool)
    inner[[i for i in range(p["n"]) if i not in set(p["parent"][1:].tolist())]] = False
    assert np.abs(a["u"][inner] - b["u"][inner]).max() <= 1e-4 * max(1.0, np.abs(a["u"]).max())


def test_exact_hessian_equals_gauss_newton_on_linear_quadratic_trees():
    """No curvature in the dynamics or the constraints: the two options take the same single step."""
    p = scenes.linear_problem(3, N=12, splits={2: 2, 6: 3})
    a, b = oracle.solve(p), oracle.solve(p, hessian=1)
    assert a["inner_iters"] == b["inner_iters"] == 1
    np.testing.assert_allclose(a["u"], b["u"], atol=1e-10)
