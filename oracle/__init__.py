"""FP64 CPU oracle for the branch-MPC AL-iLQR method (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It wraps ``bmpc_oracle.c`` (plain C,
double precision) through ctypes and shares no code with the CUDA path.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bmpc_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

OK, MAX_ITER, LS_FAIL = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/liboracle.so`` (plain IEEE double, no fast-math)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-ffp-contract=off",
                               "-o", _LIB, _SRC, "-lm"])
    return _LIB


_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int)


class Problem(C.Structure):
    _fields_ = [("n", C.c_int), ("nx", C.c_int), ("nu", C.c_int), ("model", C.c_int),
                ("n_obs", C.c_int), ("box_on", C.c_int), ("lane_on", C.c_int),
                ("parent", _ip), ("dt", C.c_double), ("params", _dp), ("x0", _dp),
                ("xref", _dp), ("weight", _dp), ("Qw", _dp), ("QNw", _dp), ("Rw", _dp),
                ("u_lo", _dp), ("u_hi", _dp), ("lane_lo", C.c_double), ("lane_hi", C.c_double),
                ("obs", _dp), ("Alin", _dp), ("Blin", _dp), ("Aedge", _dp), ("Bedge", _dp)]


class Opts(C.Structure):
    _fields_ = [("max_iters", C.c_int), ("max_outer", C.c_int), ("n_alpha", C.c_int),
                ("eps_tol", C.c_double), ("tau", C.c_double), ("omega0", C.c_double),
                ("eta0", C.c_double), ("a_omega", C.c_double), ("b_omega", C.c_double),
                ("a_eta", C.c_double), ("b_eta", C.c_double), ("rho0", C.c_double),
                ("rho_max", C.c_double), ("mu0", C.c_double), ("beta", C.c_double),
                ("ls_rel_eps", C.c_double), ("lqr_scan", C.c_int), ("hessian", C.c_int), ("cap_rule", C.c_int),
                ("trace", C.c_void_p), ("trace_user", C.c_void_p)]


# The FP32 library's default constants, which the oracle takes as options to run the same algorithm:
# Algorithm 1 as the oracle's own default, with the library's convergence tests at 0.8 eps_tol (its
# kkt_margin), so that points it returns as converged meet eps_tol = 1e-5 when evaluated exactly.
PRODUCT_RULE = dict(eps_tol=8e-6)
# The library's alternative rule at a failed outer step (cap_rule = 1 with a low cap): the penalty
# is capped at rho_max = 100, and a failure at the cap applies the multiplier step
# y <- max(0, y + rho g) instead of keeping y.
CAP_RULE = dict(cap_rule=1, rho_max=100.0, eps_tol=8e-6)

TRACE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_int, C.POINTER(C.c_double), *([C.POINTER(C.c_double)] * 7))


class Stats(C.Structure):
    _fields_ = [("status", C.c_int), ("inner_iters", C.c_int), ("outer_iters", C.c_int),
                ("ls_fail_total", C.c_int), ("r_kkt", C.c_double), ("c", C.c_double),
                ("rho", C.c_double), ("mu", C.c_double), ("omega", C.c_double), ("eta", C.c_double)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        _lib.orc_merit.restype = C.c_double
        _lib.orc_kkt_relaxed.restype = C.c_double
        _lib.orc_aug_lagrangian.restype = C.c_double
    return _lib


def _d(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a):
    return a.ctypes.data_as(_dp)


def n_con(p) -> int:
    return 2 * p["nu"] * p["box_on"] + p["n_obs"] + 2 * p["lane_on"]


class _Marshal:
    """Holds contiguous float64 copies alive while the C structure points at them."""

    def __init__(self, p):
        self.keep = {k: _d(p[k]) for k in ("params", "x0", "xref", "weight", "Qw", "QNw", "Rw",
                                           "u_lo", "u_hi", "obs", "Alin", "Blin")}
        edge = p.get("Aedge") is not None
        if edge:
            self.keep["Aedge"], self.keep["Bedge"] = _d(p["Aedge"]), _d(p["Bedge"])
        self.parent = np.ascontiguousarray(p["parent"], dtype=np.int32)
        k = self.keep
        self.s = Problem(p["n"], p["nx"], p["nu"], p["model"], p["n_obs"], p["box_on"],
                         p["lane_on"], self.parent.ctypes.data_as(_ip), p["dt"], _ptr(k["params"]),
                         _ptr(k["x0"]), _ptr(k["xref"]), _ptr(k["weight"]), _ptr(k["Qw"]),
                         _ptr(k["QNw"]), _ptr(k["Rw"]), _ptr(k["u_lo"]), _ptr(k["u_hi"]),
                         p["lane_lo"], p["lane_hi"], _ptr(k["obs"]), _ptr(k["Alin"]), _ptr(k["Blin"]),
                         _ptr(k["Aedge"]) if edge else None, _ptr(k["Bedge"]) if edge else None)


def default_opts(**kw) -> Opts:
    o = Opts()
    lib().orc_default_opts(C.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def solve(p, opts: Opts | None = None, warm=None, trace: list | None = None, **kw):
    """Run the AL method (Algorithm 1) to convergence; returns x, u, lam, y and stats.

    With ``trace`` (a list) every inner iteration appends ("inner", info, x, u, lam, y, dx, du, dlam)
    and every outer update ("outer", info, x, u, lam, y_before, y_after), as copies; the info fields
    are listed at ``orc_trace_fn`` in bmpc_oracle.c."""
    m = _Marshal(p)
    n, nx, nu, nc = p["n"], p["nx"], p["nu"], n_con(p)
    x, u, lam, y = (np.zeros((n, nx)), np.zeros((n, nu)), np.zeros((n, nx)), np.zeros((n, max(nc, 1))))
    st = Stats()
    o = opts if opts is not None else default_opts(**kw)
    if trace is not None:
        shapes = [(n, nx), (n, nu), (n, nx), (n, max(nc, 1)), (n, nx), (n, nu), (n, nx)]

        def _cb(_user, kind, info, *arrs):
            k = 16 if kind == 0 else 10
            rec = ["inner" if kind == 0 else "outer", np.ctypeslib.as_array(info, (k,)).copy()]
            shp = shapes if kind == 0 else shapes[:4] + [shapes[3]]
            for a, sh in zip(arrs, shp):
                rec.append(np.ctypeslib.as_array(a, sh).copy()[:, :nc] if sh == shapes[3]
                           else np.ctypeslib.as_array(a, sh).copy())
            trace.append(tuple(rec))

        cb = TRACE_FN(_cb)
        o.trace = C.cast(cb, C.c_void_p)
    if warm is not None:
        w = [_d(a) for a in warm]
        if nc == 0:
            w[3] = np.zeros((n, 1))
        wp = [_ptr(a) for a in w]
    else:
        w, wp = None, [None] * 4
    rc = lib().orc_solve(C.byref(m.s), C.byref(o), *wp, _ptr(x), _ptr(u), _ptr(lam), _ptr(y), C.byref(st))
    return dict(x=x, u=u, lam=lam, y=y[:, :nc], status=rc, inner_iters=st.inner_iters,
                outer_iters=st.outer_iters, r_kkt=st.r_kkt, c=st.c, rho=st.rho, mu=st.mu,
                ls_fail_total=st.ls_fail_total)


def cold_start(p):
    m = _Marshal(p)
    n, nx, nu, nc = p["n"], p["nx"], p["nu"], n_con(p)
    x, u, lam, y = (np.zeros((n, nx)), np.zeros((n, nu)), np.zeros((n, nx)), np.zeros((n, max(nc, 1))))
    lib().orc_cold_start(C.byref(m.s), _ptr(x), _ptr(u), _ptr(lam), _ptr(y))
    return x, u, lam, y[:, :nc]


def dynamics(p, x, u):
    """x+ = f(x, u) with A = df/dx, B = df/du."""
    m = _Marshal(p)
    nx, nu = p["nx"], p["nu"]
    xn, A, B = np.zeros(nx), np.zeros((nx, nx)), np.zeros((nx, nu))
    lib().orc_dynamics(C.byref(m.s), _ptr(_d(x)), _ptr(_d(u)), _ptr(xn), _ptr(A), _ptr(B))
    return xn, A, B


def constraints(p, node, is_leaf, x, u):
    m = _Marshal(p)
    nc, nx, nu = n_con(p), p["nx"], p["nu"]
    g, Jx, Ju = np.zeros(max(nc, 1)), np.zeros((max(nc, 1), nx)), np.zeros((max(nc, 1), nu))
    ex = np.zeros(max(nc, 1), np.int32)
    lib().orc_constraints(C.byref(m.s), int(node), int(is_leaf), _ptr(_d(x)), _ptr(_d(u)), _ptr(g),
                          _ptr(Jx), _ptr(Ju), ex.ctypes.data_as(_ip))
    return g[:nc], Jx[:nc], Ju[:nc], ex[:nc].astype(bool)


def tree_lqr(parent, Q, M, R, q, r, A, B, c, edge=False):
    """Tree LQR of Eq. (lqr_tree_approx): returns K, k, P, p, dx, du, lam.  A, B per parent (row i: the
    Jacobians of node i's dynamics, shared by its children) or, with edge=True, per edge (row m: the
    edge into node m)."""
    parent = np.ascontiguousarray(parent, dtype=np.int32)
    n = parent.shape[0]
    nx, nu = np.shape(B)[1], np.shape(B)[2]
    K, k = np.zeros((n, nu, nx)), np.zeros((n, nu))
    P, pv = np.zeros((n, nx, nx)), np.zeros((n, nx))
    dx, du, lam = np.zeros((n, nx)), np.zeros((n, nu)), np.zeros((n, nx))
    args = [_d(a) for a in (Q, M, R, q, r, A, B, c)]
    rc = lib().orc_tree_lqr(n, parent.ctypes.data_as(_ip), nx, nu, *[_ptr(a) for a in args],
                            _ptr(K), _ptr(k), _ptr(P), _ptr(pv), _ptr(dx), _ptr(du), _ptr(lam), int(edge))
    if rc != 0:
        raise RuntimeError(f"orc_tree_lqr failed: {rc}")
    return K, k, P, pv, dx, du, lam


def tree_lqr_scan(parent, Q, M, R, q, r, A, B, c, edge=False):
    """Tree LQR by scans (Sec. III-B: CVF suffix scans along the non-branching segments, tree Riccati
    steps at branch nodes, prefix scans of the closed-loop maps along every path); outputs as
    tree_lqr."""
    parent = np.ascontiguousarray(parent, dtype=np.int32)
    n = parent.shape[0]
    nx, nu = np.shape(B)[1], np.shape(B)[2]
    K, k = np.zeros((n, nu, nx)), np.zeros((n, nu))
    P, pv = np.zeros((n, nx, nx)), np.zeros((n, nx))
    dx, du, lam = np.zeros((n, nx)), np.zeros((n, nu)), np.zeros((n, nx))
    args = [_d(a) for a in (Q, M, R, q, r, A, B, c)]
    rc = lib().orc_tree_lqr_scan(n, parent.ctypes.data_as(_ip), nx, nu, *[_ptr(a) for a in args],
                                 _ptr(K), _ptr(k), _ptr(P), _ptr(pv), _ptr(dx), _ptr(du), _ptr(lam), int(edge))
    if rc != 0:
        raise RuntimeError(f"orc_tree_lqr_scan failed: {rc}")
    return K, k, P, pv, dx, du, lam


def kkt(p, x, u, lam, y):
    """Original-problem KKT measures: [stationarity, defect, infeasibility, complementarity, y<0]."""
    m = _Marshal(p)
    nc = n_con(p)
    yy = _d(y) if nc else np.zeros((p["n"], 1))
    out = np.zeros(5)
    lib().orc_kkt(C.byref(m.s), _ptr(_d(x)), _ptr(_d(u)), _ptr(_d(lam)), _ptr(yy), _ptr(out))
    return out


def merit(p, x, u, lam, y, rho, mu):
    m = _Marshal(p)
    yy = _d(y) if n_con(p) else np.zeros((p["n"], 1))
    return lib().orc_merit(C.byref(m.s), _ptr(_d(x)), _ptr(_d(u)), _ptr(_d(lam)), _ptr(yy),
                           C.c_double(rho), C.c_double(mu))


def direction(p, x, u, lam, y, rho, mu):
    """Search direction and merit data: dx, du, dlam, info[phi0, dphi, dzWdz, |d|^2, dphi(mu=0), L_a]."""
    m = _Marshal(p)
    n, nx, nu = p["n"], p["nx"], p["nu"]
    yy = _d(y) if n_con(p) else np.zeros((n, 1))
    dx, du, dl, info = np.zeros((n, nx)), np.zeros((n, nu)), np.zeros((n, nx)), np.zeros(6)
    rc = lib().orc_direction(C.byref(m.s), _ptr(_d(x)), _ptr(_d(u)), _ptr(_d(lam)), _ptr(yy),
                             C.c_double(rho), C.c_double(mu), _ptr(dx), _ptr(du), _ptr(dl), _ptr(info))
    if rc != 0:
        raise RuntimeError(f"orc_direction failed: {rc}")
    return dx, du, dl, info


def kkt_relaxed(p, x, u, lam, y, rho):
    m = _Marshal(p)
    yy = _d(y) if n_con(p) else np.zeros((p["n"], 1))
    return lib().orc_kkt_relaxed(C.byref(m.s), _ptr(_d(x)), _ptr(_d(u)), _ptr(_d(lam)), _ptr(yy),
                                 C.c_double(rho))


def aug_lagrangian(p, x, u, y, rho):
    m = _Marshal(p)
    yy = _d(y) if n_con(p) else np.zeros((p["n"], 1))
    return lib().orc_aug_lagrangian(C.byref(m.s), _ptr(_d(x)), _ptr(_d(u)), _ptr(yy), C.c_double(rho))


def dyn_hessian(p, x, u, mu):
    """sum_i mu_i d^2 f_i / dz dz of the discrete dynamics at (x, u), z = (x, u) (exact, hyper-dual)."""
    m = _Marshal(p)
    nz = p["nx"] + p["nu"]
    H = np.zeros((nz, nz))
    rc = lib().orc_dyn_hessian(C.byref(m.s), _ptr(_d(x)), _ptr(_d(u)), _ptr(_d(mu)), _ptr(H))
    if rc != 0:
        raise RuntimeError(f"orc_dyn_hessian failed: {rc}")
    return H


def obs_hessian(ob, X, Y):
    out = np.zeros(3)
    lib().orc_obs_hessian(_ptr(_d(ob)), C.c_double(X), C.c_double(Y), _ptr(out))
    return out


def jacobi_eig(S):
    S = _d(S)
    n = S.shape[0]
    ev, V = np.zeros(n), np.zeros((n, n))
    lib().orc_jacobi_eig(n, _ptr(S), _ptr(ev), _ptr(V))
    return ev, V


def eig_modify(S):
    S = _d(S).copy()
    lib().orc_eig_modify(S.shape[0], _ptr(S))
    return S
