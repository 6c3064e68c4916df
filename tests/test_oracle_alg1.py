"""Pins of the oracle's Algorithm 1 decisions, recomputed from outside the oracle.

The oracle reports every inner iteration and every outer update through its trace
callback.  These tests recompute what each decision must satisfy, from the
paper's definitions and with the oracle's pinned pieces only (the merit
function, itself pinned by finite differences, and the constraint rows and
Jacobians, pinned by finite differences and closed forms):

  * the merit penalty rule (Gill et al. 1992, cited in Algorithm 1): after the
    update phi'(0; mu) <= -1/2 dz'W dz, with phi'(0; mu) taken by central
    differences of the merit and dz'W dz rebuilt here from the cost weights and
    the constraint Jacobians; mu never decreases within a solve;
  * the line search (Eq. sufficient_decrease): the accepted alpha meets the
    Armijo inequality on a recomputed merit, and every larger alpha_i = 2^-i
    fails it (the largest accepted step is taken);
  * the outer update (Sec. IV-B, Algorithm 1): the branch taken follows from
    c = |max(g, -y/rho)|_inf against eta, the multiplier update is
    y <- max(0, y + rho g) with g recomputed here, a failure keeps y and raises
    rho to min(tau rho, rho_max) (the paper's branch), and the product's cap
    rule applies the multiplier step at rho_max instead;
  * the tolerance schedules of Algorithm 1 (read as in Conn et al.'s BCL);
  * the cold start of Sec. V-B by its properties (root at x-bar, each leaf at
    its final reference, states affine in the stage along every path, zero
    controls and multipliers).
"""
import numpy as np
import pytest

import oracle
import scenes

BETA = 1e-4
LS_REL_EPS = 1e-6


def _leaf_mask(p):
    leaf = np.ones(p["n"], bool)
    leaf[np.unique(p["parent"][1:])] = False
    return leaf


def _rows(p, x, u):
    """Constraint values, Jacobians and existence flags of every node (oracle.constraints)."""
    leaf = _leaf_mask(p)
    G, JX, JU, EX = [], [], [], []
    for i in range(p["n"]):
        g, jx, ju, ex = oracle.constraints(p, i, leaf[i], x[i], u[i])
        G.append(g)
        JX.append(jx)
        JU.append(ju)
        EX.append(ex)
    return np.array(G), np.array(JX), np.array(JU), np.array(EX)


def _wq(p, x, u, y, rho, dx, du):
    """dz'W dz of the Gauss-Newton Hessian of L_a (Eq. AL): the weighted tracking and input
    weights plus rho (J_g dz)^2 on the rows where y + rho g > 0."""
    leaf = _leaf_mask(p)
    w = p["weight"]
    Qd = np.where(leaf[:, None], p["QNw"][None, :], p["Qw"][None, :])
    val = np.sum(w[:, None] * Qd * dx ** 2)
    val += np.sum((w * ~leaf)[:, None] * p["Rw"][None, :] * du ** 2)
    if oracle.n_con(p):
        G, JX, JU, EX = _rows(p, x, u)
        act = EX & (y + rho * G > 0)
        jdz = np.einsum("nck,nk->nc", JX, dx) + np.einsum("nck,nk->nc", JU, du)
        val += rho * np.sum(np.where(act, jdz ** 2, 0.0))
    return val


def _traced(p, **kw):
    tr = []
    r = oracle.solve(p, trace=tr, **kw)
    return r, [t for t in tr if t[0] == "inner"], [t for t in tr if t[0] == "outer"]


CASES = [(1, 0), (1, 3), (2, 1), (2, 4)]
RULES = {"paper": {}, "cap": oracle.CAP_RULE}


def _problem(cfg, seed):
    if cfg == 4:
        return scenes.config4_problem(4, seed)
    return scenes.instances(cfg, 1, seed0=seed)[0]


LS_CASES = CASES + [(4, 19), (4, 10)]   # two mixed-batch scenes whose line search backtracks


@pytest.mark.parametrize("rule", sorted(RULES))
@pytest.mark.parametrize("cfg,seed", CASES)
def test_merit_penalty_rule(cfg, seed, rule):
    p = _problem(cfg, seed)
    r, inner, _ = _traced(p, **RULES[rule])
    assert inner
    mus = [t[1][4] for t in inner]
    assert all(b >= a for a, b in zip(mus, mus[1:])), "mu decreased within the solve"
    for _, info, x, u, lam, y, dx, du, dl in inner:
        rho, mu_prev, mu, phi0, dphi, wq_o = info[2], info[3], info[4], info[5], info[6], info[8]
        assert mu >= mu_prev
        # phi(0) is the merit at the iterate (Eq. merit with J = L_a)
        assert phi0 == pytest.approx(oracle.merit(p, x, u, lam, y, rho, mu), rel=1e-12, abs=1e-12)
        # phi'(0; mu) by central differences of the merit along (dx, du, dlam)
        h = 1e-6
        fp = oracle.merit(p, x + h * dx, u + h * du, lam + h * dl, y, rho, mu)
        fm = oracle.merit(p, x - h * dx, u - h * du, lam - h * dl, y, rho, mu)
        dfd = (fp - fm) / (2 * h)
        scale = max(1.0, abs(phi0))
        assert abs(dfd - dphi) <= 1e-6 * scale, (dfd, dphi)
        # dz'W dz rebuilt from the weights and the constraint Jacobians
        wq = _wq(p, x, u, y, rho, dx, du)
        assert wq == pytest.approx(wq_o, rel=1e-9, abs=1e-12)
        # the descent requirement that the penalty rule enforces
        assert dfd <= -0.5 * wq + 1e-6 * scale, (dfd, wq)
        if mu > mu_prev:   # raised exactly to the smallest value meeting the requirement
            need = 2.0 * (info[7] + 0.5 * wq) / info[9]
            assert mu == pytest.approx(need, rel=1e-9)


@pytest.mark.parametrize("beta", [BETA, 0.3])
@pytest.mark.parametrize("rule", sorted(RULES))
@pytest.mark.parametrize("cfg,seed", LS_CASES)
def test_armijo_acceptance_on_recomputed_merits(cfg, seed, rule, beta):
    """beta = 1e-4 is the solver's constant; beta = 0.3 makes the inequality bind on many steps, so
    that a wrong sign or factor in it changes which step is taken."""
    p = _problem(cfg, seed)
    r, inner, _ = _traced(p, beta=beta, **RULES[rule])
    slack_decided = 0
    backtracked = 0
    for _, info, x, u, lam, y, dx, du, dl in inner:
        rho, mu, phi0, dphi, alpha, accepted = info[2], info[4], info[5], info[6], info[10], bool(info[11])
        backtracked += alpha < 1.0
        bound = lambda al: phi0 + beta * al * dphi
        phi = lambda al: oracle.merit(p, x + al * dx, u + al * du, lam + al * dl, y, rho, mu)
        k_star = int(round(-np.log2(alpha)))
        assert alpha == 2.0 ** -k_star
        for k in range(k_star):                        # every larger step fails Eq. (sufficient_decrease)
            assert phi(2.0 ** -k) > bound(2.0 ** -k) + LS_REL_EPS * abs(phi0)
        if accepted:
            pa = phi(alpha)
            assert pa == pytest.approx(info[12], rel=1e-12, abs=1e-12)
            assert pa <= bound(alpha) + LS_REL_EPS * abs(phi0)
            slack_decided += pa > bound(alpha)
            assert bool(info[13]) == (pa > bound(alpha))
    # the absolute slack of the finite-precision reading decides few acceptances
    assert slack_decided <= max(1, len(inner) // 5), (slack_decided, len(inner))
    _BACKTRACKED[beta] = _BACKTRACKED.get(beta, 0) + backtracked


_BACKTRACKED = {}


def test_binding_beta_backtracks_somewhere():
    """With beta = 0.3 the Armijo inequality rejects the full step on some of the cases above (so the
    sign and factor of the inequality are exercised)."""
    total = 0
    for cfg, seed in LS_CASES:
        _, inner, _ = _traced(_problem(cfg, seed), beta=0.3, **oracle.CAP_RULE)
        total += sum(t[1][10] < 1.0 for t in inner)
    assert total >= 3, total


def _check_outer_sequence(p, outer, rule):
    o = oracle.default_opts(**rule)
    omega, eta = o.omega0, o.eta0
    for _, info, x, u, lam, yb, ya in outer:
        branch, c, eta_b, rho_b, rho_a = int(info[1]), info[2], info[3], info[4], info[5]
        omega_a, eta_a, r_kkt, conv = info[6], info[7], info[8], bool(info[9])
        assert eta_b == pytest.approx(eta, rel=1e-12)
        G, _, _, EX = _rows(p, x, u)
        # c = |max(g, -y/rho)|_inf over the rows that exist (Sec. IV-B)
        c_here = np.max(np.abs(np.where(EX, np.maximum(G, -yb / rho_b), 0.0))) if G.size else 0.0
        assert c == pytest.approx(c_here, rel=1e-12, abs=1e-15)
        y_step = np.where(EX, np.maximum(0.0, yb + rho_b * G), yb)
        if branch == 0:
            assert c <= eta_b and rho_a == rho_b
            np.testing.assert_allclose(ya, y_step, rtol=1e-13, atol=1e-15)
            if conv:
                assert max(r_kkt, c) < o.eps_tol
            else:
                omega = max(omega * rho_b ** -o.b_omega, o.eps_tol)
                eta = max(eta * rho_b ** -o.b_eta, o.eps_tol)
        else:
            assert c > eta_b
            if branch == 1:
                assert rho_b < o.rho_max and rho_a == min(o.tau * rho_b, o.rho_max)
                assert np.array_equal(ya, yb)
            elif branch == 2:
                assert rule.get("cap_rule") == 1 and rho_a == rho_b == o.rho_max
                np.testing.assert_allclose(ya, y_step, rtol=1e-13, atol=1e-15)
            else:
                assert branch == 3 and rho_a == rho_b == o.rho_max and rule.get("cap_rule", 0) == 0
                assert np.array_equal(ya, yb)
            omega = max(o.omega0 * rho_a ** -o.a_omega, o.eps_tol)
            eta = max(o.eta0 * rho_a ** -o.a_eta, o.eps_tol)
        if not conv:
            assert omega_a == pytest.approx(omega, rel=1e-12) and eta_a == pytest.approx(eta, rel=1e-12)
    return [int(t[1][1]) for t in outer]


@pytest.mark.parametrize("cfg,seed", CASES + [(3, 0)])
def test_outer_updates_follow_algorithm_1(cfg, seed):
    """The paper's branch (the oracle's default): success updates y, failure keeps y and raises rho."""
    p = _problem(cfg, seed)
    r, _, outer = _traced(p)
    branches = _check_outer_sequence(p, outer, {})
    assert r["status"] != oracle.OK or branches[-1] == 0


def test_failure_branch_keeps_y_and_raises_rho():
    """A scene whose first outer step fails: y is kept bit for bit and rho rises by tau."""
    for seed in range(10):
        p = _problem(2, seed)
        r, _, outer = _traced(p)
        branches = _check_outer_sequence(p, outer, {})
        if 1 in branches:
            return
    pytest.fail("no failed outer step on ten config-2 scenes")


def test_cap_rule_multiplier_step_at_the_cap():
    """The product's rule (rho_max = 100): a failed outer step at the cap applies y <- max(0, y + rho g)
    with rho unchanged, checked on a scene that reaches the cap."""
    for seed in range(40):
        p = scenes.config4_problem(4, seed)
        if p["n"] > 900:
            continue
        r, _, outer = _traced(p, **oracle.CAP_RULE)
        branches = _check_outer_sequence(p, outer, oracle.CAP_RULE)
        if 2 in branches:
            return
    pytest.fail("no outer step at the cap on forty config-4 scenes")


def test_paper_branch_holds_rho_at_its_cap():
    """Algorithm 1 with a low cap (rho_max = 100, cap_rule 0): a failure at the cap keeps y and rho."""
    rule = dict(rho_max=100.0)
    for seed in range(40):
        p = scenes.config4_problem(4, seed)
        if p["n"] > 900:
            continue
        r, _, outer = _traced(p, **rule)
        branches = _check_outer_sequence(p, outer, rule)
        if 3 in branches:
            return
    pytest.fail("no outer step held at the cap on forty config-4 scenes")


@pytest.mark.parametrize("case", ["config1", "config2", "config3", "ragged"])
def test_cold_start_properties(case):
    """Sec. V-B's initialisation, pinned by what it must satisfy rather than by its formula: the root
    holds x-bar, every leaf of a node's first-leaf path holds that leaf's final reference, states are
    affine in the stage along every first-leaf path, and u, lambda, y are zero."""
    if case == "ragged":
        p = scenes.linear_problem(9, N=6, splits={2: 3})
    else:
        p = getattr(scenes, case)(1)
    x, u, lam, y = oracle.cold_start(p)
    par, st, n = p["parent"], p["stage"], p["n"]
    leaf = _leaf_mask(p)
    np.testing.assert_array_equal(x[0], p["x0"])
    assert not u.any() and not lam.any() and not y.any()
    first_child = {}
    for i in range(1, n):
        first_child.setdefault(int(par[i]), i)
    for i in np.where(leaf)[0]:
        np.testing.assert_allclose(x[i], p["xref"][i], rtol=0, atol=1e-12)
    # the nodes sharing a first leaf form a chain of consecutive stages; along it the states are
    # affine in the stage, and the affine function extrapolated to stage 0 passes through x-bar
    chains = {}
    for i in range(n):
        j = i
        while j in first_child:
            j = first_child[j]
        chains.setdefault(j, []).append(i)
    assert sorted(sum(chains.values(), [])) == list(range(n))
    for j, nodes in chains.items():
        nodes = sorted(nodes, key=lambda i: st[i])
        ks = st[nodes].astype(float)
        assert np.array_equal(np.diff(ks), np.ones(len(ks) - 1))
        xs = x[nodes]
        tol = 1e-9 * max(1.0, np.abs(xs).max())
        if len(nodes) >= 3:
            assert np.abs(xs[2:] - 2 * xs[1:-1] + xs[:-2]).max() <= tol
        if len(nodes) >= 2:
            slope = xs[-1] - xs[-2]
            np.testing.assert_allclose(xs[0] - ks[0] * slope, p["x0"], rtol=0, atol=tol * max(1.0, st.max()))
