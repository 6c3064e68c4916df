"""Seeded synthetic driving scenes for branch MPC (scenario-tree) problems.

This module only *generates inputs*: scenario trees, initial states, reference
trajectories, per-node obstacle predictions and model constants.  It contains
none of the solver's arithmetic (no dynamics integration of the ego vehicle,
no costs, no constraints) and is the one module shared by the FP64 oracle and
the CUDA path.

Every floating-point value is rounded to the nearest float32, so the FP64
oracle and the FP32 GPU path receive bit-identical problem data.

Problem layout (all arrays are numpy):
  parent  int32  [n]            parent[0] = -1, parent[i] < i, level order
                                (nodes sorted by stage, children of a node
                                contiguous and in parent order)
  stage   int32  [n]            stage of each node (root stage 0)
  x0      f64    [nx]           measured state x-bar (the root state is fixed)
  xref    f64    [n, nx]        tracking reference per node
  weight  f64    [n]            node cost weight (branch probability)
  Qw, QNw f64    [nx]           diagonal stage / final state weights
  Rw      f64    [nu]           diagonal input weights
  u_lo, u_hi f64 [nu]           input box
  box_on, lane_on int           which constraint families exist
  lane_lo, lane_hi float        lateral lane bounds on the Y coordinate
  obs     f64    [n, n_obs, 5]  obstacle ellipse per node: cx, cy, heading, a, b
  params  f64    [10]           model constants (see MODEL_PARAMS_*)
  Alin, Blin                    discrete dynamics for the linear model (model 2)

The tree sizes follow the convention "a branch at stage s with factor b gives
every stage-(s-1) node b children at stage s"; leaves are at stage N.  Scene
recipes stand in for the intersection / overtaking planning problems of the
paper's Sec. II-B (Fig. 1a) and Sec. V-B; no dataset is used.
"""
from __future__ import annotations

import math
import numpy as np

MODEL_KINEMATIC = 0
MODEL_DYNAMIC = 1
MODEL_LINEAR = 2
MODEL_UNICYCLE = 3

# params layout: [L, m, Iz, lf, lr, Cf, Cr, vmin, veps, n_sub]
MODEL_PARAMS_KINEMATIC = (2.7, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 1.0)
MODEL_PARAMS_DYNAMIC = (2.7, 1500.0, 2250.0, 1.2, 1.5, 8.0e4, 8.0e4, 2.0, 0.1, 4.0)
MODEL_PARAMS_LINEAR = (0.0,) * 9 + (1.0,)
MODEL_PARAMS_UNICYCLE = (0.0,) * 9 + (1.0,)   # one RK4 step per dt

V_REF = 8.0          # lane cruising speed [m/s]
REF_ACCEL = 1.0      # speed ramp of the reference profile [m/s^2]
ELLIPSE_A = 3.0      # keep-out semi-axis along the obstacle heading [m]
ELLIPSE_B = 1.5      # keep-out semi-axis across the obstacle heading [m]
LANE = (-5.25, 5.25)


def f32(a):
    """Round to the nearest float32 and return float64 (exactly representable)."""
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def tree_parents(N: int, splits: dict[int, int]):
    """Level-ordered scenario tree: root at stage 0, leaves at stage N.

    ``splits`` maps a stage s to the factor b: every stage-(s-1) node gets b
    children at stage s; every other stage has fan-out 1.
    """
    parent = [-1]
    stage = [0]
    frontier = [0]
    for k in range(1, N + 1):
        b = int(splits.get(k, 1))
        nxt = []
        for p in frontier:
            for _ in range(b):
                parent.append(p)
                stage.append(k)
                nxt.append(len(parent) - 1)
        frontier = nxt
    return np.asarray(parent, np.int32), np.asarray(stage, np.int32)


def branch_weights(parent: np.ndarray) -> np.ndarray:
    """Uniform branch probabilities: a child of a b-way split gets 1/b of its parent."""
    n = parent.shape[0]
    nch = np.zeros(n, np.int64)
    for i in range(1, n):
        nch[parent[i]] += 1
    w = np.ones(n)
    for i in range(1, n):
        w[i] = w[parent[i]] / nch[parent[i]]
    return w


def _reference(x0, stage, nx, dt, y_line=0.0):
    """Straight reference line Y = y_line, heading 0, speed ramping to V_REF."""
    N = int(stage.max())
    v0 = float(x0[3])
    v = np.array([v0 + np.clip(V_REF - v0, -REF_ACCEL * k * dt, REF_ACCEL * k * dt)
                  for k in range(N + 1)])
    X = np.empty(N + 1)
    X[0] = x0[0]
    for k in range(N):
        X[k + 1] = X[k] + 0.5 * (v[k] + v[k + 1]) * dt
    ref_stage = np.zeros((N + 1, nx))
    ref_stage[:, 0] = X
    ref_stage[:, 1] = y_line
    ref_stage[:, 3] = v
    return ref_stage[stage]


# ---------------------------------------------------------------- obstacles
def _sample_mode(rng, family, side):
    """Behaviour of one obstacle on one branch segment: (speed or None, yaw_rate, decel)."""
    if family == "line":            # straight-line car, speed per branch U[0, 10]
        return (rng.uniform(0.0, 10.0), 0.0, 0.0)
    r = rng.uniform()
    if family == "adjacent":        # car in a neighbouring lane: keep, brake, or drift in
        if r < 0.4:
            return (None, 0.0, 0.0)
        if r < 0.7:
            return (None, 0.0, 2.0)
        return (None, -side * 0.05, 0.0)
    if r < 0.4:                     # crossing car: go (constant velocity)
        return (None, 0.0, 0.0)
    if r < 0.75:                    # yield: decelerate to a stop at 2 m/s^2
        return (None, 0.0, 2.0)
    return (None, rng.choice([-0.2, 0.2]), 0.0)   # turning branch


def _obstacle_tree(rng, parent, stage, dt, init_states, families):
    """Propagate each obstacle along the tree; branches resample the behaviour."""
    if isinstance(families, str):
        families = [families] * len(init_states)
    n = parent.shape[0]
    n_obs = len(init_states)
    nch = np.zeros(n, np.int64)
    for i in range(1, n):
        nch[parent[i]] += 1
    # state per node per obstacle: cx, cy, heading, speed, yaw_rate, decel
    st = np.zeros((n, n_obs, 6))
    for j, s0 in enumerate(init_states):
        st[0, j] = s0
    for i in range(1, n):
        p = parent[i]
        for j in range(n_obs):
            cx, cy, hd, sp, yr, dc = st[p, j]
            if nch[p] > 1:
                m_sp, m_yr, m_dc = _sample_mode(rng, families[j], np.sign(st[0, j, 1]) or 1.0)
                if m_sp is not None:
                    sp = m_sp
                yr, dc = m_yr, m_dc
            sp_new = max(0.0, sp - dc * dt)
            hd_new = hd + yr * dt
            vmean = 0.5 * (sp + sp_new)
            cx += vmean * math.cos(hd_new) * dt
            cy += vmean * math.sin(hd_new) * dt
            st[i, j] = (cx, cy, hd_new, sp_new, yr, dc)
    obs = np.zeros((n, n_obs, 5))
    obs[:, :, 0:3] = st[:, :, 0:3]
    obs[:, :, 3] = ELLIPSE_A
    obs[:, :, 4] = ELLIPSE_B
    return obs, st


def _inside_any(obs_root, X, Y):
    for cx, cy, hd, a, b in obs_root:
        dx, dy = X - cx, Y - cy
        dpar = math.cos(hd) * dx + math.sin(hd) * dy
        dper = -math.sin(hd) * dx + math.cos(hd) * dy
        if (dpar / a) ** 2 + (dper / b) ** 2 < 1.5:
            return True
    return False


# ---------------------------------------------------------------- problems
def _base(model, N, splits, dt=0.1):
    parent, stage = tree_parents(N, splits)
    if model == MODEL_KINEMATIC:
        nx, params = 4, MODEL_PARAMS_KINEMATIC
        Qw, Rw = [1.0, 1.0, 0.1, 0.5], [0.1, 1.0]
    elif model == MODEL_DYNAMIC:
        nx, params = 6, MODEL_PARAMS_DYNAMIC
        Qw, Rw = [1.0, 1.0, 0.1, 0.5, 0.1, 0.1], [0.1, 1.0]
    else:
        raise ValueError(model)
    return dict(model=model, nx=nx, nu=2, dt=dt, parent=parent, stage=stage,
                params=np.array(params, np.float64), Qw=np.array(Qw), QNw=np.array(Qw),
                Rw=np.array(Rw), u_lo=np.array([-3.0, -0.5]), u_hi=np.array([3.0, 0.5]),
                box_on=1, weight=branch_weights(parent))


def _finish(p):
    """Round every float array to float32 and fill derived entries."""
    for k in ("x0", "xref", "weight", "Qw", "QNw", "Rw", "u_lo", "u_hi", "obs", "params"):
        p[k] = f32(p[k])
    p["lane_lo"] = float(np.float32(p.get("lane_lo", LANE[0])))
    p["lane_hi"] = float(np.float32(p.get("lane_hi", LANE[1])))
    p["dt"] = float(np.float32(p["dt"]))
    p["n"] = int(p["parent"].shape[0])
    p["n_obs"] = int(p["obs"].shape[1])
    p.setdefault("Alin", np.zeros((p["nx"], p["nx"])))
    p.setdefault("Blin", np.zeros((p["nx"], p["nu"])))
    return p


def _x0(rng, model, box_y, heading, vrange):
    X = rng.uniform(-10.0, 10.0)
    Y = rng.uniform(-box_y, box_y)
    psi = rng.uniform(-heading, heading)
    v = rng.uniform(*vrange)
    return np.array([X, Y, psi, v] + ([0.0, 0.0] if model == MODEL_DYNAMIC else []))


def _crossing_obstacle(rng, X0, dist=(30.0, 50.0)):
    """Car approaching an intersection dist[0]-dist[1] m ahead from either side."""
    side = rng.choice([-1.0, 1.0])
    return (X0 + rng.uniform(*dist), side * rng.uniform(10.0, 18.0),
            -side * math.pi / 2, rng.uniform(3.0, 8.0), 0.0, 0.0)


def _adjacent_obstacle(rng, X0):
    """Car in a neighbouring lane (centre +-3.5 m), 5-30 m ahead."""
    side = rng.choice([-1.0, 1.0])
    return (X0 + rng.uniform(5.0, 30.0), side * 3.5, 0.0, rng.uniform(4.0, 9.0), 0.0, 0.0)


def config1(seed: int):
    """Kinematic bicycle, N = 20, root splits into 3; one obstacle car driving ahead on the
    ego's line (offset by up to 1 m), with a different speed U[0, 10] on each branch."""
    rng = np.random.default_rng([1, seed])
    p = _base(MODEL_KINEMATIC, 20, {1: 3})
    x0 = _x0(rng, MODEL_KINEMATIC, 10.0, math.pi / 6, (0.0, 10.0))
    p["x0"] = f32(x0)
    p["xref"] = _reference(p["x0"], p["stage"], p["nx"], p["dt"], y_line=float(p["x0"][1]))
    init = [(x0[0] + rng.uniform(15.0, 30.0), x0[1] + rng.uniform(-1.0, 1.0), 0.0, 0.0, 0.0, 0.0)]
    p["obs"], p["obs_state"] = _obstacle_tree(rng, p["parent"], p["stage"], p["dt"], init, "line")
    p["obs_family"] = ["line"]
    p["y_line"] = float(p["x0"][1])
    p["lane_on"] = 0
    return _finish(p)


def _multi_obstacle(rng, p, n_obs, n_cross, cross_dist=(30.0, 50.0)):
    x0 = p["x0"]
    init, fam = [], []
    for j in range(n_obs):
        if j < n_cross:
            init.append(_crossing_obstacle(rng, x0[0], cross_dist))
            fam.append("crossing")
        else:
            init.append(_adjacent_obstacle(rng, x0[0]))
            fam.append("adjacent")
    p["obs"], p["obs_state"] = _obstacle_tree(rng, p["parent"], p["stage"], p["dt"], init, fam)
    p["obs_family"] = fam
    p["y_line"] = 0.0
    p["lane_on"] = 1
    return p


def config2(seed: int):
    """Kinematic bicycle, N = 40, binary splits at 1, 5, 10, 15, 20; 3 crossing cars."""
    rng = np.random.default_rng([2, seed])
    p = _base(MODEL_KINEMATIC, 40, {1: 2, 5: 2, 10: 2, 15: 2, 20: 2})
    p["x0"] = f32(_x0(rng, MODEL_KINEMATIC, 1.5, math.pi / 12, (0.0, 10.0)))
    p["xref"] = _reference(p["x0"], p["stage"], p["nx"], p["dt"])
    return _finish(_multi_obstacle(rng, p, 3, 3))


def config3(seed: int):
    """Dynamic bicycle, N = 60, factor 4 at 1, 10, 20; 5 obstacles."""
    rng = np.random.default_rng([3, seed])
    p = _base(MODEL_DYNAMIC, 60, {1: 4, 10: 4, 20: 4})
    p["x0"] = f32(_x0(rng, MODEL_DYNAMIC, 1.5, math.pi / 12, (2.0, 10.0)))
    p["xref"] = _reference(p["x0"], p["stage"], p["nx"], p["dt"])
    return _finish(_multi_obstacle(rng, p, 5, 2, cross_dist=(45.0, 70.0)))


def config4_problem(seed: int, index: int):
    """One problem of the mixed batch: S in {2..64}, N in [20, 60], 1-5 obstacles."""
    rng = np.random.default_rng([4, seed, index])
    S = int(rng.choice([2, 4, 8, 16, 32, 64]))
    N = int(rng.integers(20, 61))
    n_obs = int(rng.integers(1, 6))
    model = MODEL_KINEMATIC if rng.uniform() < 0.5 else MODEL_DYNAMIC
    levels = int(round(math.log2(S)))
    gap = max(1, N // (2 * levels))
    splits = {1 + j * gap: 2 for j in range(levels)}
    p = _base(model, N, splits)
    vr = (0.0, 10.0) if model == MODEL_KINEMATIC else (2.0, 10.0)
    p["x0"] = f32(_x0(rng, model, 1.5, math.pi / 12, vr))
    p["xref"] = _reference(p["x0"], p["stage"], p["nx"], p["dt"])
    return _finish(_multi_obstacle(rng, p, n_obs, min(n_obs, 2)))


def config4(seed: int = 4, count: int = 4096):
    return [config4_problem(seed, i) for i in range(count)]


def chain_problem(seed: int, model: int, N: int, n_obs: int = 3):
    """A single-path tree (one scenario, N + 1 nodes) of the mixed-batch family: the given model,
    horizon and obstacle count.  Its iterations run the sweeps' dependent chain with no branching,
    which measures the per-stage latency of the sweeps.  The unicycle's chain is its benchmark
    scene with horizon N."""
    if model == MODEL_UNICYCLE:
        return unicycle(seed, N=N)
    if model == MODEL_LINEAR:
        return mass_spring(seed, N=N, Nr=1, nd=1, constrained=True)
    rng = np.random.default_rng([8, seed, model, N])
    p = _base(model, N, {})
    vr = (0.0, 10.0) if model == MODEL_KINEMATIC else (2.0, 10.0)
    p["x0"] = f32(_x0(rng, model, 1.5, math.pi / 12, vr))
    p["xref"] = _reference(p["x0"], p["stage"], p["nx"], p["dt"])
    return _finish(_multi_obstacle(rng, p, n_obs, min(n_obs, 2)))


def linear_problem(seed: int, N: int = 10, splits=None, nx: int = 4, nu: int = 2,
                   constrained: bool = False):
    """Linear dynamics x+ = A x + B u with quadratic cost (the LQ special case)."""
    rng = np.random.default_rng([7, seed])
    parent, stage = tree_parents(N, splits or {})
    n = parent.shape[0]
    A = np.eye(nx) + 0.1 * rng.standard_normal((nx, nx))
    B = 0.1 * rng.standard_normal((nx, nu)) + 0.1 * np.eye(nx, nu)
    p = dict(model=MODEL_LINEAR, nx=nx, nu=nu, dt=0.1, parent=parent, stage=stage,
             params=np.array(MODEL_PARAMS_LINEAR), Qw=rng.uniform(0.5, 2.0, nx),
             QNw=rng.uniform(0.5, 2.0, nx), Rw=rng.uniform(0.1, 1.0, nu),
             u_lo=-np.ones(nu) * (0.5 if constrained else 1e3),
             u_hi=np.ones(nu) * (0.5 if constrained else 1e3),
             box_on=1 if constrained else 0, lane_on=0, weight=branch_weights(parent),
             x0=rng.standard_normal(nx), xref=0.3 * rng.standard_normal((n, nx)),
             obs=np.zeros((n, 0, 5)), Alin=f32(A), Blin=f32(B))
    return _finish(p)


UNICYCLE_TARGET = (10.0, 0.0, 0.0, 0.0)
UNICYCLE_OBSTACLES = ((3.5, 0.25, 1.0), (6.5, -0.35, 0.8))   # circle centres and radii [m]


def unicycle(seed: int, N: int = 50, splits=None):
    """The constraint benchmark of Sec. V-B with the unicycle (nx = 4: X, Y, theta, v; nu = 2:
    a, omega), dt = 0.1 s, N = 50: the initial state is sampled around the nominal (0, 0, 0, 0)
    (X, Y ~ U[-1, 1] m, theta ~ U[-0.3, 0.3], v ~ U[0, 1] m/s), the target state is fixed at
    (10, 0, 0, 0), two circular obstacles lie near the straight line to it (a distance constraint:
    the keep-out ellipse with equal semi-axes), and the inputs are bounded (|a| <= 2, |omega| <= 1.5).
    The reference is the target at every node; the start is the linear interpolation to it (the cold
    start).  The paper does not print its obstacle layout or weights: these are this recipe's.
    With ``splits`` the same problem on a scenario tree whose branches see the obstacles shifted
    laterally by up to 0.3 m."""
    rng = np.random.default_rng([10, seed])
    parent, stage = tree_parents(N, splits or {})
    n = parent.shape[0]
    x0 = np.array([rng.uniform(-1.0, 1.0), rng.uniform(-1.0, 1.0), rng.uniform(-0.3, 0.3), rng.uniform(0.0, 1.0)])
    xref = np.tile(np.asarray(UNICYCLE_TARGET), (n, 1))
    obs = np.zeros((n, len(UNICYCLE_OBSTACLES), 5))
    shift = np.zeros(n)
    for i in range(1, n):
        nch = np.count_nonzero(parent == parent[i])
        shift[i] = shift[parent[i]] + (rng.uniform(-0.3, 0.3) if nch > 1 else 0.0)
    for j, (cx, cy, r) in enumerate(UNICYCLE_OBSTACLES):
        obs[:, j] = np.stack([np.full(n, cx), cy + shift, np.zeros(n), np.full(n, r), np.full(n, r)], axis=1)
    p = dict(model=MODEL_UNICYCLE, nx=4, nu=2, dt=0.1, parent=parent, stage=stage,
             params=np.array(MODEL_PARAMS_UNICYCLE), Qw=np.array([0.01, 0.01, 0.01, 0.01]),
             QNw=np.array([10.0, 10.0, 1.0, 1.0]), Rw=np.array([0.1, 0.1]),
             u_lo=np.array([-2.0, -1.5]), u_hi=np.array([2.0, 1.5]), box_on=1, lane_on=0,
             weight=branch_weights(parent), x0=x0, xref=xref, obs=obs)
    return _finish(p)


def _rk4_linear(Ac, Bc, h):
    """Discrete matrices of one classical RK4 step of x' = Ac x + Bc u with u held: the RK4 map of a
    linear system is x+ = (I + hA + (hA)^2/2 + (hA)^3/6 + (hA)^4/24) x + h (I + hA/2 + (hA)^2/6 +
    (hA)^3/24) B u.  Problem data for the per-edge linear model (it is the plant, not the solver)."""
    n = Ac.shape[0]
    hA = h * Ac
    I = np.eye(n)
    A = I + hA + hA @ hA / 2 + hA @ hA @ hA / 6 + hA @ hA @ hA @ hA / 24
    B = h * (I + hA / 2 + hA @ hA / 6 + hA @ hA @ hA / 24) @ Bc
    return A, B


def mass_spring(seed: int, N: int = 20, Nr: int = 2, nd: int = 2, constrained: bool = False):
    """The tree setting of Sec. V-A: a chain of masses and springs between two walls whose spring
    constant is uncertain, sampled n_d ways at every stage up to the robust horizon N_r (Z = n_d^N_r
    scenario paths); each edge of the tree carries the dynamics of its branch's spring constant.
    Two unit masses (n_x = 4: positions, then velocities) with a force on each (n_u = 2), springs
    k ~ U[0.5, 1.5] per branch, dt = 0.1 s by RK4, tracking the origin with Q = I, R = 0.1 I,
    x-bar random; with ``constrained`` the forces are bounded by 0.5."""
    rng = np.random.default_rng([11, seed])
    parent, stage = tree_parents(N, {s: nd for s in range(1, Nr + 1)})
    n = parent.shape[0]
    dt = 0.1
    Ae, Be = np.zeros((n, 4, 4)), np.zeros((n, 4, 2))
    for m in range(1, n):
        k = rng.uniform(0.5, 1.5) if stage[m] <= Nr else None
        if k is None:   # past the robust horizon the branch keeps its parent edge's model
            Ae[m], Be[m] = Ae[parent[m]], Be[parent[m]]
            continue
        Kc = np.array([[-2.0 * k, k], [k, -2.0 * k]])
        Ac = np.block([[np.zeros((2, 2)), np.eye(2)], [Kc, np.zeros((2, 2))]])
        Bc = np.vstack([np.zeros((2, 2)), np.eye(2)])
        Ae[m], Be[m] = _rk4_linear(Ac, Bc, dt)
    p = dict(model=MODEL_LINEAR, nx=4, nu=2, dt=dt, parent=parent, stage=stage,
             params=np.array(MODEL_PARAMS_LINEAR), Qw=np.ones(4), QNw=np.ones(4), Rw=np.full(2, 0.1),
             u_lo=-np.ones(2) * (0.5 if constrained else 1e3), u_hi=np.ones(2) * (0.5 if constrained else 1e3),
             box_on=1 if constrained else 0, lane_on=0, weight=branch_weights(parent),
             x0=np.concatenate([rng.uniform(-1.0, 1.0, 2), np.zeros(2)]), xref=np.zeros((n, 4)),
             obs=np.zeros((n, 0, 5)), Aedge=f32(Ae), Bedge=f32(Be))
    return _finish(p)


def mass_spring_chain(seed: int, M: int = 15, N: int = 40, Nr: int = 3, nd: int = 2, batch: int = 1,
                      dt: float = 0.1):
    """Tree LQR data of Sec. V-A at the paper's sizes: a chain of M unit masses joined by springs,
    with walls at both ends (n_x = 2M: positions, then velocities) and M - 1 actuators, actuator a
    pushing masses a and a + 1 apart (n_u = M - 1).  The spring constant is uncertain: n_d values
    k ~ U[0.5, 1.5] at every stage up to the robust horizon N_r (Z = n_d^N_r scenario paths), each
    edge carrying the RK4 discretisation (step dt) of its branch's spring constant; past N_r a branch
    keeps its parent edge's model.  Cost: Q = I at every node, R = 0.1 I, no linear terms; the batch
    of `batch` problems shares the tree and differs in the spring samples and the initial positions
    x0 ~ U[-1, 1] (velocities 0).  Returns float64 arrays in the layout of the general tree LQR
    ([batch][n][...]), with parent and stage."""
    rng = np.random.default_rng([12, seed, M, N, Nr, nd])
    nx, nu = 2 * M, M - 1
    parent, stage = tree_parents(N, {s: nd for s in range(1, Nr + 1)})
    n = parent.shape[0]
    E = np.zeros((M, nu))
    for a in range(nu):
        E[a, a], E[a + 1, a] = 1.0, -1.0
    A = np.zeros((batch, n, nx, nx))
    B = np.zeros((batch, n, nx, nu))
    for t in range(batch):
        for m in range(1, n):
            if stage[m] > Nr:
                A[t, m], B[t, m] = A[t, parent[m]], B[t, parent[m]]
                continue
            k = rng.uniform(0.5, 1.5)
            Kc = k * (np.diag(np.full(M, -2.0)) + np.diag(np.ones(M - 1), 1) + np.diag(np.ones(M - 1), -1))
            Ac = np.block([[np.zeros((M, M)), np.eye(M)], [Kc, np.zeros((M, M))]])
            Bc = np.vstack([np.zeros((M, nu)), E])
            A[t, m], B[t, m] = _rk4_linear(Ac, Bc, dt)
    Q = np.broadcast_to(np.eye(nx), (batch, n, nx, nx)).copy()
    R = np.broadcast_to(0.1 * np.eye(nu), (batch, n, nu, nu)).copy()
    x0 = np.concatenate([rng.uniform(-1.0, 1.0, (batch, M)), np.zeros((batch, M))], axis=1)
    return dict(parent=parent, stage=stage, nx=nx, nu=nu, Q=Q, R=R, q=np.zeros((batch, n, nx)),
                r=np.zeros((batch, n, nu)), A=A, B=B, c=np.zeros((batch, n, nx)), x0=x0)


def instances(config: int, count: int, seed0: int = 0):
    """Seeded instances of a configuration (1-3), seeds seed0 .. seed0+count-1."""
    gen = {1: config1, 2: config2, 3: config3}[config]
    return [gen(seed0 + s) for s in range(count)]


def advance(p, x0_next, seed: int):
    """The next receding-horizon problem of scene p: the same tree and costs, measured state
    x0_next, the reference restarted from it, and every obstacle continuing from its state at the
    first scenario's stage-1 node with behaviours resampled for the new branches."""
    rng = np.random.default_rng([9, seed])
    q = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in p.items()}
    q["x0"] = f32(np.asarray(x0_next, dtype=np.float64))
    q["xref"] = _reference(q["x0"], p["stage"], p["nx"], p["dt"], y_line=p.get("y_line", 0.0))
    init = [tuple(v) for v in p["obs_state"][1]]
    q["obs"], q["obs_state"] = _obstacle_tree(rng, p["parent"], p["stage"], p["dt"], init, p["obs_family"])
    return _finish(q)


# ---------------------------------------------------------------- vectorised batches (one tree)
def _modes_batch(rng, fam, side, shape):
    """Vectorised _sample_mode for obstacles of one family: (speed or nan, yaw_rate, decel)."""
    r = rng.uniform(size=shape)
    sp = np.full(shape, np.nan)
    yr = np.zeros(shape)
    dc = np.zeros(shape)
    if fam == "line":
        sp = rng.uniform(0.0, 10.0, size=shape)
        return sp, yr, dc
    if fam == "adjacent":
        dc = np.where((r >= 0.4) & (r < 0.7), 2.0, 0.0)
        yr = np.where(r >= 0.7, -side * 0.05, 0.0)
        return sp, yr, dc
    turn = rng.choice([-0.2, 0.2], size=shape)
    dc = np.where((r >= 0.4) & (r < 0.75), 2.0, 0.0)
    yr = np.where(r >= 0.75, turn, 0.0)
    return sp, yr, dc


def _obstacle_tree_batch(rng, parent, stage, dt, init, families):
    """Obstacle propagation along one tree for P scenes at once; init [P, n_obs, 6].  Returns the
    per-node ellipses [P, n, n_obs, 5] (float32 values) and the obstacle states at node 1."""
    P, n_obs = init.shape[0], init.shape[1]
    n = parent.shape[0]
    nch = np.bincount(parent[1:], minlength=n)
    obs = np.zeros((P, n, n_obs, 5), np.float32)
    obs[:, :, :, 3] = ELLIPSE_A
    obs[:, :, :, 4] = ELLIPSE_B
    obs[:, 0, :, 0:3] = init[:, :, 0:3]
    side = np.sign(init[:, :, 1])
    side[side == 0] = 1.0
    prev_nodes, prev_state = np.array([0]), init[:, None].copy()      # [P, m, n_obs, 6]
    st1 = None
    for k in range(1, int(stage.max()) + 1):
        nodes = np.where(stage == k)[0]
        par = parent[nodes]
        loc = np.searchsorted(prev_nodes, par)
        prev = prev_state[:, loc]
        sp, yr, dc = prev[..., 3].copy(), prev[..., 4].copy(), prev[..., 5].copy()
        branch = nch[par] > 1
        if branch.any():
            bi = np.where(branch)[0]
            for j, fam in enumerate(families):
                m_sp, m_yr, m_dc = _modes_batch(rng, fam, side[:, None, j], (P, bi.size))
                cur = sp[:, bi, j]
                sp[:, bi, j] = np.where(np.isnan(m_sp), cur, m_sp)
                yr[:, bi, j] = m_yr
                dc[:, bi, j] = m_dc
        sp_new = np.maximum(0.0, sp - dc * dt)
        hd_new = prev[..., 2] + yr * dt
        vmean = 0.5 * (sp + sp_new)
        cur = np.empty_like(prev)
        cur[..., 0] = prev[..., 0] + vmean * np.cos(hd_new) * dt
        cur[..., 1] = prev[..., 1] + vmean * np.sin(hd_new) * dt
        cur[..., 2] = hd_new
        cur[..., 3] = sp_new
        cur[..., 4] = yr
        cur[..., 5] = dc
        obs[:, nodes, :, 0:3] = cur[..., 0:3]
        if k == 1:
            st1 = cur[:, 0].copy()
        prev_nodes, prev_state = nodes, cur
    return obs, st1


def _reference_batch(x0, stage, nx, dt, y_line):
    """Vectorised _reference for P initial states x0 [P, nx]."""
    N = int(stage.max())
    k = np.arange(N + 1)
    v0 = x0[:, 3:4]
    v = v0 + np.clip(V_REF - v0, -REF_ACCEL * k * dt, REF_ACCEL * k * dt)
    X = np.concatenate([x0[:, 0:1], x0[:, 0:1] + np.cumsum(0.5 * (v[:, :-1] + v[:, 1:]) * dt, axis=1)], axis=1)
    ref = np.zeros((x0.shape[0], N + 1, nx))
    ref[:, :, 0] = X
    ref[:, :, 1] = np.asarray(y_line)[:, None] if np.ndim(y_line) else y_line
    ref[:, :, 3] = v
    return ref[:, stage]


def batch_problems(seed: int, count: int, model=MODEL_DYNAMIC, N=60, splits=None, n_obs=5, n_cross=2,
                   cross_dist=(45.0, 70.0)):
    """`count` scenes on one tree (default: the config-3 recipe), generated vectorised from one
    seed: initial states, references and per-node obstacle predictions as in config3()."""
    splits = {1: 4, 10: 4, 20: 4} if splits is None else splits
    rng = np.random.default_rng([11, seed])
    base = _base(model, N, splits)
    parent, stage, nx = base["parent"], base["stage"], base["nx"]
    vr = (2.0, 10.0) if model == MODEL_DYNAMIC else (0.0, 10.0)
    x0 = np.zeros((count, nx))
    x0[:, 0] = rng.uniform(-10.0, 10.0, count)
    x0[:, 1] = rng.uniform(-1.5, 1.5, count)
    x0[:, 2] = rng.uniform(-math.pi / 12, math.pi / 12, count)
    x0[:, 3] = rng.uniform(*vr, count)
    x0 = f32(x0)
    xref = _reference_batch(x0, stage, nx, base["dt"], 0.0)
    init = np.zeros((count, n_obs, 6))
    fam = []
    for j in range(n_obs):
        if j < n_cross:
            side = rng.choice([-1.0, 1.0], count)
            init[:, j] = np.stack([x0[:, 0] + rng.uniform(*cross_dist, count), side * rng.uniform(10.0, 18.0, count),
                                   -side * math.pi / 2, rng.uniform(3.0, 8.0, count), np.zeros(count),
                                   np.zeros(count)], 1)
            fam.append("crossing")
        else:
            side = rng.choice([-1.0, 1.0], count)
            init[:, j] = np.stack([x0[:, 0] + rng.uniform(5.0, 30.0, count), side * 3.5, np.zeros(count),
                                   rng.uniform(4.0, 9.0, count), np.zeros(count), np.zeros(count)], 1)
            fam.append("adjacent")
    obs, st1 = _obstacle_tree_batch(rng, parent, stage, base["dt"], init, fam)
    obs, xref = obs.astype(np.float64), f32(xref)
    shared = _finish(dict(base, x0=x0[0], xref=xref[0], obs=obs[0], lane_on=1))
    out = []
    for i in range(count):
        p = dict(shared)
        p["x0"] = x0[i]
        p["xref"] = xref[i]
        p["obs"] = obs[i]
        p["obs_state"] = np.zeros((2,) + st1.shape[1:])
        p["obs_state"][1] = st1[i]
        p["obs_family"] = fam
        p["y_line"] = 0.0
        out.append(p)
    return out
