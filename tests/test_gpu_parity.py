"""GPU (FP32, CUDA through the C ABI) versus the FP64 oracle on identical seeded inputs.

Both sides run Algorithm 1 with the same constants (oracle.PRODUCT_RULE: the library's
convergence tests at 0.8 eps_tol); the cap rule (cap_rule = 1, rho capped at 100) is compared
too, on both sides, and so is the plain FP32 iterate (compensated = 0) with that rule.

Parity bar (per converged problem):
  * controls: |u_gpu - u_oracle|_inf <= 1e-4 * max(|u_oracle|_inf, 1);
  * the oracle's FP64 KKT conditions of Eq. (bmpc) evaluated at the GPU's returned
    (x, u, lambda, y) are below 1e-5 (stationarity, defects, feasibility, complementarity);
  * inner-iteration counts: see ITER_ABS and ITER_MEAN.
The method is an iteration on a nonconvex problem, so FP32 and FP64 may stop at two
different KKT points; such a pair counts as "distinct local minimum" only if the oracle,
warm-started from the GPU solution, confirms it as a KKT point of its own within two
iterations, and such pairs must stay a small minority.

One iteration (test_one_iteration_from_an_identical_iterate): from an identical FP32 iterate, both sides take
exactly one inner iteration (max_iters = 1); the new (x, u, lambda, y) are compared element by
element.  That checks the search direction, the step size and the multiplier updates directly,
which a whole solve cannot (a slightly wrong direction still converges to the same point).
"""
import numpy as np
import pytest

import oracle
import scenes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

U_REL = 1e-4
KKT_TOL = 1e-5
RULE = oracle.PRODUCT_RULE

# Inner-iteration counts of a matched pair: FP32 rounding can move a borderline decision (an
# inner-loop exit at r_kkt <= omega, an Armijo test, the c <= eta test) by one iteration.  Measured on
# B300 over 83 matched pairs of configs 1-4: 82 equal, one differing by 1.  The rule: |delta| <= 1
# for every matched pair and at most a quarter of a test's matched pairs differing at all.
ITER_ABS = 1
ITER_MEAN = 0.25


def _orc(p, **kw):
    return oracle.solve(p, **RULE, **kw)


def _gpu(problems, **kw):
    from paper_2506_13624_b300 import bmpc
    opts = bmpc.default_opts(**kw)
    b = bmpc.Batch(problems)
    b.set_problems()
    b.solve(opts)
    res = b.get_solutions()
    b.close()
    return res


def _check_pair(p, g, r, orc_kw=None):
    """Returns 'match', 'distinct' or raises AssertionError with a reason."""
    assert g["status"] == oracle.OK, f"GPU status {g['status']} (oracle {r['status']}), r_kkt={g['r_kkt']:.2e}"
    nl = np.ones(p["n"], bool)
    nl[np.unique(p["parent"][1:])] = False
    inner = ~nl
    k = oracle.kkt(p, g["x"], g["u"], g["lam"], g["y"])
    assert k[:4].max() <= KKT_TOL, f"FP64 KKT at the GPU point: {k}"
    assert (g["y"] >= 0).all()
    du = np.abs(g["u"][inner] - r["u"][inner]).max()
    if du <= U_REL * max(np.abs(r["u"][inner]).max(), 1.0):
        return "match"
    w = _orc(p, warm=(g["x"], g["u"], g["lam"], g["y"]), **(orc_kw or {}))
    assert w["status"] == oracle.OK and w["inner_iters"] <= 2, "GPU point not confirmed by the oracle"
    assert np.abs(w["u"][inner] - g["u"][inner]).max() <= U_REL * max(np.abs(g["u"][inner]).max(), 1.0)
    return "distinct"


def _run_config(problems, min_match=0.8, orc_kw=None, **kw):
    gres = _gpu(problems, **kw)
    counts = {"match": 0, "distinct": 0, "oracle_fail": 0}
    dits = []
    for p, g in zip(problems, gres):
        r = _orc(p, **(orc_kw or {}))
        if r["status"] != oracle.OK:
            counts["oracle_fail"] += 1
            assert g["status"] in (oracle.OK, oracle.MAX_ITER, oracle.LS_FAIL)
            continue
        kind = _check_pair(p, g, r, orc_kw)
        counts[kind] += 1
        if kind == "match":
            dits.append(g["inner_iters"] - r["inner_iters"])
    solved = counts["match"] + counts["distinct"]
    assert solved >= 1
    assert counts["match"] >= min_match * solved, counts
    _iter_rule(dits)
    counts["iter_delta"] = dits
    return counts


def _iter_rule(dits):
    if not dits:
        return
    d = np.abs(np.asarray(dits))
    assert d.max() <= ITER_ABS and np.mean(d > 0) <= ITER_MEAN, dits


def test_config1_parity():
    print(_run_config(scenes.instances(1, 12)))


def test_config2_parity():
    print(_run_config(scenes.instances(2, 6)))


def test_config3_parity():
    print(_run_config(scenes.instances(3, 8, seed0=1), min_match=0.75))


@pytest.mark.parametrize("cfg", [2, 3])
def test_512_thread_instance_parity(cfg):
    """The one-block-per-SM instance (512 threads per problem, the single-solve choice of the
    autotuner) against the oracle, both sweep forms."""
    ps = scenes.instances(cfg, 3, seed0=40)
    mm = 0.8 if cfg == 2 else 0.5
    _run_config(ps, min_match=mm, block_threads=512)
    _run_config(ps, min_match=mm, block_threads=512, variant=1)


def test_mixed_batch_parity():
    print(_run_config(scenes.config4(4, 24)))


def test_mixed_batch_with_per_model_block_sizes():
    """A mixed batch whose kinematic launch uses 128 threads per problem and its dynamic launch 512:
    the same parity as with one block size."""
    print(_run_config(scenes.config4(4, 16), block_threads=256, block_threads_model=[128, 512, 0]))


def test_linear_quadratic_one_iteration():
    ps = [scenes.linear_problem(s, N=12, splits={2: 2, 6: 3}) for s in range(3)]
    gres = _gpu(ps)
    for p, g in zip(ps, gres):
        r = _orc(p)
        assert g["status"] == oracle.OK and g["inner_iters"] == 1
        np.testing.assert_allclose(g["u"], r["u"], atol=1e-4 * max(1.0, np.abs(r["u"]).max()))
        np.testing.assert_allclose(g["x"], r["x"], atol=1e-4 * max(1.0, np.abs(r["x"]).max()))


def test_constrained_linear_problem_parity():
    ps = [scenes.linear_problem(s, N=15, splits={3: 2, 8: 2}, constrained=True) for s in range(3)]
    print(_run_config(ps, min_match=1.0))


def test_nonanticipativity_bitwise():
    p = scenes.linear_problem(5, N=10, splits={2: 3, 5: 2})
    st = p["stage"]
    xr = np.zeros((st.max() + 1, p["nx"]))
    for i in range(p["n"]):
        xr[st[i]] = p["xref"][i]
    p["xref"] = xr[st]
    g = _gpu([p])[0]
    for k in range(st.max() + 1):
        rows = g["x"][st == k]
        assert (rows == rows[0]).all()


def test_edge_trees():
    """Smallest tree, ragged leaves, more nodes per stage than threads, 8 obstacles, no constraints."""
    base = scenes.linear_problem(1, N=1, splits={})
    assert base["n"] == 2
    wide = scenes.linear_problem(2, N=4, splits={1: 8, 2: 8, 3: 6})      # 384 nodes per stage
    many = scenes.config2(1)
    obs8 = dict(many)
    extra = np.repeat(many["obs"][:, :1, :], 5, axis=1)
    extra[:, :, 1] += 1000.0
    obs8["obs"] = np.concatenate([many["obs"], extra], axis=1)
    obs8["n_obs"] = 8
    ps = [base, wide, obs8]
    gres = _gpu(ps, block_threads=128)
    for p, g in zip(ps, gres):
        r = _orc(p)
        assert r["status"] == oracle.OK
        _check_pair(p, g, r)


def test_ragged_tree_parity():
    """Leaves at different depths (a hand-built level-ordered tree)."""
    p = scenes.linear_problem(9, N=6, splits={2: 3})
    # cut two of the three branches short: keep nodes of branch 0 to the end, others to stage 4
    st, par = p["stage"], p["parent"]
    keep = np.ones(p["n"], bool)
    branch = np.zeros(p["n"], int)
    for i in range(1, p["n"]):
        branch[i] = branch[par[i]] if st[i] > 2 else (i % 3 if st[i] == 2 else 0)
    keep[(branch != 0) & (st > 4)] = False
    idx = np.where(keep)[0]
    remap = -np.ones(p["n"], int)
    remap[idx] = np.arange(len(idx))
    q = dict(p)
    q["parent"] = np.array([-1] + [remap[par[i]] for i in idx[1:]], np.int32)
    q["stage"] = st[idx]
    q["n"] = len(idx)
    for key in ("xref", "weight", "obs"):
        q[key] = p[key][idx]
    r = _orc(q)
    g = _gpu([q])[0]
    assert r["status"] == oracle.OK
    assert _check_pair(q, g, r) == "match"


def test_graph_replay_and_determinism():
    from paper_2506_13624_b300 import bmpc
    ps = scenes.config4(4, 8)
    b = bmpc.Batch(ps)
    b.set_problems()
    b.solve()
    r1 = b.get_solutions()
    b.solve(graph=True)
    r2 = b.get_solutions()
    b.solve(graph=True)
    r3 = b.get_solutions()
    b.close()
    for a, c, d in zip(r1, r2, r3):
        for key in ("x", "u", "lam", "y"):
            assert np.array_equal(a[key], c[key]) and np.array_equal(c[key], d[key])
        assert a["inner_iters"] == c["inner_iters"]


def test_queue_order_changes_nothing_but_the_schedule():
    """Longest-predicted-first (sorted on the device from the previous solve's iterations) and
    largest-tree-first queues give bit-identical solutions; the sorted order is a permutation."""
    from paper_2506_13624_b300 import bmpc
    ps = scenes.config4(5, 40)
    b = bmpc.Batch(ps)
    res = []
    for qo in (0, 1, 1):
        b.set_problems()
        b.solve(bmpc.default_opts(queue_order=qo), graph=qo == 1)
        res.append(b.get_solutions())
    order = b.device_order()
    b.close()
    assert sorted(order.tolist()) == list(range(len(ps)))
    for a, c, d in zip(*res):
        for key in ("x", "u", "lam", "y"):
            assert np.array_equal(a[key], c[key]) and np.array_equal(a[key], d[key])
        assert a["inner_iters"] == c["inner_iters"] == d["inner_iters"]
    # within a model, the last solve visited the problems by decreasing nodes x (iterations + 1)
    cost = {k: int(ps[k]["n"]) * (r["inner_iters"] + 1) for k, r in enumerate(res[-1])}
    models = [int(ps[k]["model"]) for k in order]
    for m in set(models):
        seq = [cost[k] for k, mm in zip(order, models) if mm == m]
        assert seq == sorted(seq, reverse=True)


def test_flat_transfers_equal_the_packed_path():
    """Node-major flat uploads and downloads (device transposition) give the packed host path's
    solutions bit for bit, and the packed download after a flat upload still has absolute states."""
    from paper_2506_13624_b300 import bmpc
    ps = scenes.config4(6, 24)
    b = bmpc.Batch(ps)
    b.set_problems()
    b.solve()
    ref = b.get_solutions()
    b.set_problems_flat(*b.flat_inputs())
    b.solve()
    x, u, lam, y, st = b.get_solutions_flat(b.flat_outputs())
    again = b.get_solutions()
    b.close()
    cat = lambda key: np.concatenate([r[key].astype(np.float32).ravel() for r in ref])
    for key, got in (("x", x), ("u", u), ("lam", lam), ("y", y)):
        want = cat(key)
        assert np.array_equal(got.numpy()[:want.size], want), key
    assert [s.inner_iters for s in st] == [r["inner_iters"] for r in ref]
    for a, c in zip(ref, again):
        for key in ("x", "u", "lam", "y"):
            assert np.array_equal(a[key], c[key])


def test_async_flat_reads_on_two_streams_equal_the_synchronous_read():
    """Two handles on two streams taking steps in turn (the end-to-end pipeline): every
    asynchronous read, once waited for, equals the synchronous flat read bit for bit."""
    from paper_2506_13624_b300 import bmpc
    ps = scenes.config4(7, 20)
    ref_b = bmpc.Batch(ps)
    ref_b.set_problems_flat(*ref_b.flat_inputs())
    ref_b.solve()
    ref = ref_b.get_solutions_flat(ref_b.flat_outputs())
    ref_b.close()
    pipe = [bmpc.Batch(ps, stream=torch.cuda.Stream()) for _ in range(2)]
    fin = pipe[0].flat_inputs()
    outs = [bb.flat_outputs() for bb in pipe]
    for k in range(5):
        bb = pipe[k % 2]
        if k >= 2:
            bb.wait_solutions(want_stats=False)
        bb.set_problems_flat(*fin)
        bb.solve(graph=True)
        bb.get_solutions_flat_async(outs[k % 2])
    stats = [bb.wait_solutions() for bb in pipe]
    for bb, out, st in zip(pipe, outs, stats):
        for got, want in zip(out, ref[:4]):
            assert torch.equal(got, want)
        assert [s.inner_iters for s in st] == [s.inner_iters for s in ref[4]]
        assert [s.status for s in st] == [s.status for s in ref[4]]
        bb.close()


def test_convergence_outcomes_follow_the_oracle_on_config3():
    """On config-3 scenes the FP32 GPU path converges exactly where the FP64 oracle does: the
    failures (a pass-before/after decision against a crossing car that 50 iterations do not settle)
    are the method's, not FP32's.  A problem that converges at the iteration cap on one side only
    is a borderline case and is not counted."""
    ps = [scenes.config3(k) for k in range(12)]
    gres = _gpu(ps, block_threads=256)
    failures = 0
    for p, g in zip(ps, gres):
        r = _orc(p)
        if max(g["inner_iters"], r["inner_iters"]) >= 45 and (g["status"] == oracle.OK) != (r["status"] == oracle.OK):
            continue
        assert (g["status"] == oracle.OK) == (r["status"] == oracle.OK), (g["status"], r["status"], g["r_kkt"], r["r_kkt"])
        failures += r["status"] != oracle.OK
    assert failures >= 1   # the sample holds scenes the method does not settle


def test_batch_equals_single():
    ps = scenes.config4(4, 6)
    batch = _gpu(ps, block_threads=64)
    for p, g in zip(ps, batch):
        s = _gpu([p], block_threads=64)[0]
        for key in ("x", "u", "lam", "y"):
            assert np.array_equal(g[key], s[key])


@pytest.mark.parametrize("cfg", [2, 3])
def test_level_and_path_variants_agree(cfg):
    """The level-synchronous, per-path, 8-lane per-path and scan sweeps compute the same search
    directions."""
    ps = scenes.instances(cfg, 3 if cfg == 2 else 1, seed0=3)
    lev = _gpu(ps, variant=1)
    for v in (2, 3, 4, 5):
        pth = _gpu(ps, variant=v)
        for p, a, b in zip(ps, lev, pth):
            assert a["status"] == b["status"] == oracle.OK
            assert abs(a["inner_iters"] - b["inner_iters"]) <= 1
            # the scan's FP32 compositions of E^-1 factors carry more rounding than the recursions
            tol = (2e-4 if v == 4 else 1e-4) * max(1.0, np.abs(a["u"]).max())
            np.testing.assert_allclose(a["u"], b["u"], atol=tol)


def test_autotuner_returns_a_valid_configuration():
    from paper_2506_13624_b300 import bmpc
    ps = scenes.config4(4, 32)
    b = bmpc.Batch(ps)
    b.set_problems()
    best, us = b.autotune()
    assert best.block_threads in (32, 64, 128, 256, 512) and best.variant in (1, 2, 3, 4, 5) and best.ls_chunk in (1, 2, 4)
    assert us > 0
    b.solve(best)
    tuned = b.get_solutions()
    b.solve(bmpc.default_opts())
    ref = b.get_solutions()
    b.close()
    for p, a, r in zip(ps, tuned, ref):
        assert a["status"] == r["status"]
        if a["status"] == oracle.OK:
            tol = 1e-4 * max(1.0, np.abs(r["u"]).max())
            np.testing.assert_allclose(a["u"], r["u"], atol=tol)


def test_shifted_warm_start_receding_horizon():
    """Solve, advance the scenes one step, warm-start from the shifted solution: converged, matches
    the oracle on the new problem, and needs fewer iterations than the cold start."""
    from paper_2506_13624_b300 import bmpc
    prev_ps = scenes.instances(2, 6, seed0=20)
    prev = bmpc.Batch(prev_ps)
    prev.set_problems()
    prev.solve()
    pres = prev.get_solutions()
    next_ps = [scenes.advance(p, r["x"][1], seed=k) for k, (p, r) in enumerate(zip(prev_ps, pres))]
    cold = _gpu(next_ps)
    nb = bmpc.Batch(next_ps)
    nb.set_problems()
    nb.shift_from(prev, slot=0)
    nb.solve()
    warm = nb.get_solutions()
    nb.close()
    prev.close()
    assert all(w["start_used"] == 1 for w in warm)
    for p, w in zip(next_ps, warm):
        r = _orc(p)
        if r["status"] == oracle.OK:
            _check_pair(p, w, r)
    assert sum(w["inner_iters"] for w in warm) < sum(c["inner_iters"] for c in cold)


def test_merit_selection_between_starts():
    """warm_select keeps a good primary start and rejects a bad one for the fallback."""
    import torch as T
    from paper_2506_13624_b300 import bmpc
    ps = scenes.instances(1, 4, seed0=30)
    first = _gpu(ps)
    b = bmpc.Batch(ps)
    b.set_problems()
    stride = b.start_stride()
    good = np.zeros((len(ps), stride), np.float32)
    for k, (p, g) in enumerate(zip(ps, first)):
        packed = np.concatenate([g["x"].ravel(), g["u"].ravel(), g["lam"].ravel(), g["y"].ravel()])
        good[k, :packed.size] = packed
    bad = good.copy()
    bad[:, :] = 50.0
    opts = bmpc.default_opts(warm_select=1)
    b.set_warm_device(T.from_numpy(good).cuda(), slot=0)
    b.solve(opts)
    rg = b.get_solutions()
    b.set_problems()
    b.set_warm_device(T.from_numpy(bad).cuda(), slot=0)
    b.solve(opts)
    rb = b.get_solutions()
    b.close()
    for a, c, f in zip(rg, rb, first):
        assert a["start_used"] == 1 and a["status"] == oracle.OK and a["inner_iters"] <= 2
        assert c["start_used"] == 0 and c["status"] == f["status"]
        assert np.array_equal(c["u"], f["u"])


def test_invalid_problem_rejected():
    from paper_2506_13624_b300 import bmpc
    p = dict(scenes.config1(0))
    par = p["parent"].copy()
    par[10] = 12
    p["parent"] = par
    with pytest.raises(RuntimeError):
        bmpc.Batch([p])


def test_full_size_batch_sampled():
    """The launch configuration the benchmark times: 4,096 mixed problems in one launch (the
    autotuned per-model block sizes of the benchmark, 256 threads per kinematic problem and 512 per
    dynamic one).  Sampled problems are drawn from every tree size, in three bands by node count, both
    models.  A problem the oracle solves and the GPU does not is a failure; one exception is allowed
    where the oracle itself needs 40 or more of the 50 iterations (a borderline case at the cap)."""
    ps = scenes.config4(4, 4096)
    gres = _gpu(ps, block_threads=256, block_threads_model=[256, 512, 0])
    conv = np.mean([g["status"] == oracle.OK for g in gres])
    assert conv >= 0.85, conv
    rng = np.random.default_rng(0)
    nodes = np.array([int(p["n"]) for p in ps])
    bands = [(0, 700), (700, 1500), (1500, 10 ** 6)]
    picks = []
    for lo, hi in bands:
        idx = np.where((nodes >= lo) & (nodes < hi))[0]
        picks += list(rng.choice(idx, 4, replace=False))
    assert max(nodes[picks]) >= 1500 and any(int(ps[k]["model"]) == 1 for k in picks)
    counts = {"match": 0, "distinct": 0, "oracle_fail": 0, "borderline": 0}
    dits = []
    for k in picks:
        r = _orc(ps[k])
        g = gres[k]
        if r["status"] != oracle.OK:
            counts["oracle_fail"] += 1
            continue
        if g["status"] != oracle.OK and r["inner_iters"] >= 40:
            counts["borderline"] += 1
            continue
        kind = _check_pair(ps[k], g, r)
        counts[kind] += 1
        if kind == "match":
            dits.append(g["inner_iters"] - r["inner_iters"])
    print(counts, dits, conv)
    assert counts["borderline"] <= 1, counts
    assert counts["match"] >= 0.75 * (counts["match"] + counts["distinct"]) and counts["match"] >= 6, counts
    _iter_rule(dits)


def _fp32(a):
    return np.asarray(a, np.float32).astype(np.float64)


def _one_iteration(p, k, hessian=0):
    """Both sides take one inner iteration from the same FP32 iterate: the cold start (k = 0, each
    side forms its own) or the oracle's iterate after k iterations, rounded to float32 (k is lowered
    below the oracle's own iteration count, so that the iterate is not already converged)."""
    if k == 0:
        warm = None
    else:
        k = max(1, min(k, _orc(p, hessian=hessian)["inner_iters"] - 2))
        it = _orc(p, max_iters=k, hessian=hessian)
        warm = tuple(_fp32(it[key]) for key in ("x", "u", "lam", "y"))
    from paper_2506_13624_b300 import bmpc
    b = bmpc.Batch([p])
    b.set_problems(warm=None if warm is None else [warm])
    b.solve(bmpc.default_opts(max_iters=1, hessian=hessian))
    g = b.get_solutions()[0]
    b.close()
    r = _orc(p, max_iters=1, warm=warm, hessian=hessian)
    return g, r


# One iteration from an identical FP32 iterate, compared relative to each block's magnitude
# (max(1, |.|_inf) of the oracle's block).  The step solves a tree LQR assembled in FP32 from FP32
# data: x moves by a small step on states of tens of metres (an ulp of the state, 6e-8 relative,
# dominates); u and lambda carry the rounding of the linearisation through the N + 1 Riccati steps
# (up to 4e-6 measured on B300, about 60 ulps); y <- max(0, y + rho g) multiplies the FP32 rounding
# of g by rho = 100 (up to 3.5e-5 measured).  Bars: five times the measured worst case.
STEP_TOL = {"x": 1e-6, "u": 2e-5, "lam": 2e-5, "y": 2e-4}


@pytest.mark.parametrize("cfg,k", [(1, 0), (1, 3), (2, 0), (2, 4), (3, 0), (3, 6)])
def test_one_iteration_from_an_identical_iterate(cfg, k):
    for seed in range(3 if cfg < 3 else 2):
        p = scenes.instances(cfg, 1, seed0=seed)[0]
        g, r = _one_iteration(p, k)
        assert g["inner_iters"] == r["inner_iters"] == 1, (g["inner_iters"], r["inner_iters"])
        assert g["status"] == r["status"]
        worst = {}
        for key in ("x", "u", "lam", "y"):
            a, b = g[key], r[key]
            if b.size == 0:
                continue
            scale = max(1.0, float(np.abs(b).max()))
            d = float(np.abs(a - b).max()) / scale
            worst[key] = d
            assert d <= STEP_TOL[key], (cfg, k, seed, key, d)
        print(cfg, k, seed, worst)


# ------------------------------------------------------------------ the unicycle benchmark (Sec. V-B)
def test_unicycle_parity():
    """The constraint benchmark of Sec. V-B (unicycle, N = 50, input bounds, circular obstacles,
    linear-interpolation start): GPU against the oracle on 16 instances."""
    print(_run_config([scenes.unicycle(s) for s in range(16)]))


def test_unicycle_tree_parity():
    """The same benchmark on scenario trees (branches at stages 1 and 10, obstacles shifted per
    branch)."""
    print(_run_config([scenes.unicycle(s, splits={1: 2, 10: 2}) for s in range(4)]))


def test_unicycle_solved_fraction_follows_the_oracle():
    """Sec. V-B reports the fraction of 50 instances solved against the iteration count.  On the GPU
    the fraction solved within k iterations equals the oracle's (same rule) at every k, up to one
    instance."""
    ps = [scenes.unicycle(s) for s in range(50)]
    g = _gpu(ps)
    r = [_orc(p) for p in ps]
    gi = np.array([x["inner_iters"] if x["status"] == oracle.OK else 10 ** 6 for x in g])
    ri = np.array([x["inner_iters"] if x["status"] == oracle.OK else 10 ** 6 for x in r])
    for k in range(1, 51):
        assert abs(int(np.sum(gi <= k)) - int(np.sum(ri <= k))) <= 1, k
    print("solved within 10/20/30/50:", [int(np.sum(gi <= k)) for k in (10, 20, 30, 50)],
          [int(np.sum(ri <= k)) for k in (10, 20, 30, 50)])


# ------------------------------------------------------------------ the alternative rule, the plain iterate
@pytest.mark.parametrize("compensated", [1, 0])
def test_cap_rule_parity(compensated):
    """The cap rule (cap_rule = 1, rho_max = 100: a multiplier step at the cap) on both sides, with
    the compensated iterate and with the plain FP32 one (the rule it was made for)."""
    global RULE
    saved = RULE
    RULE = oracle.CAP_RULE
    try:
        ps = scenes.instances(1, 8) + scenes.instances(2, 4) + scenes.config4(4, 12)
        print(_run_config(ps, cap_rule=1, rho_max=100.0, compensated=compensated))
    finally:
        RULE = saved


def test_plain_iterate_stalls_where_the_compensated_one_converges():
    """Algorithm 1 on the unicycle benchmark: with the plain FP32 iterate most problems stop at the
    iteration cap with the relaxed KKT residual just above the tolerance (rho times the rounding of
    an input on its bound), with the compensated iterate they converge like the oracle."""
    ps = [scenes.unicycle(s) for s in range(16)]
    plain = _gpu(ps, compensated=0)
    comp = _gpu(ps)
    orc = [_orc(p) for p in ps]
    n_orc = sum(r["status"] == oracle.OK for r in orc)
    assert sum(g["status"] == oracle.OK for g in comp) >= n_orc - 1
    assert sum(g["status"] == oracle.OK for g in plain) <= n_orc // 2


# ------------------------------------------------------------------ scan sweeps (Sec. III-B, variant 4)
def test_scan_variant_parity():
    """The scan sweeps (conditional value functions combined along non-branching segments, tree
    Riccati steps at branch nodes, pointer jumping forward) against the oracle on the planning
    configurations."""
    ps = scenes.instances(1, 6) + scenes.instances(2, 3) + scenes.instances(3, 2, seed0=1)
    print(_run_config(ps, variant=4))
    print(_run_config(ps[:6], variant=4, block_threads=512))


def test_jump_forward_variant_parity():
    """Per-path backward sweep with the pointer-jumping forward sweep (variant 5) against the oracle on
    every tree family: the planning configurations, the unicycle path and tree."""
    ps = (scenes.instances(1, 6) + scenes.instances(2, 3) + scenes.instances(3, 2, seed0=1)
          + [scenes.unicycle(s) for s in range(6)] + [scenes.unicycle(s, splits={1: 2, 10: 2}) for s in range(2)])
    print(_run_config(ps, variant=5))
    print(_run_config(ps[-8:], variant=5, block_threads=512))


def test_scan_variant_edge_and_ragged_trees():
    base = scenes.linear_problem(1, N=1, splits={})
    wide = scenes.linear_problem(2, N=4, splits={1: 8, 2: 8, 3: 6})
    deep = scenes.linear_problem(3, N=70, splits={2: 2, 40: 3})
    ragged = scenes.linear_problem(9, N=6, splits={2: 3})
    st, par = ragged["stage"], ragged["parent"]
    keep = np.ones(ragged["n"], bool)
    branch = np.zeros(ragged["n"], int)
    for i in range(1, ragged["n"]):
        branch[i] = branch[par[i]] if st[i] > 2 else (i % 3 if st[i] == 2 else 0)
    keep[(branch != 0) & (st > 4)] = False
    idx = np.where(keep)[0]
    remap = -np.ones(ragged["n"], int)
    remap[idx] = np.arange(len(idx))
    q = dict(ragged)
    q["parent"] = np.array([-1] + [remap[par[i]] for i in idx[1:]], np.int32)
    q["stage"] = st[idx]
    q["n"] = len(idx)
    for key in ("xref", "weight", "obs"):
        q[key] = ragged[key][idx]
    for bt in (32, 256):
        for v in (4, 5):
            print(_run_config([base, wide, deep, q], min_match=1.0, variant=v, block_threads=bt))


@pytest.mark.parametrize("cfg,k", [(1, 3), (2, 4), ("unicycle", 5)])
def test_scan_variant_one_iteration_against_the_oracle_scan(cfg, k):
    """One iteration of the scan sweeps from an identical FP32 iterate against the oracle's own scan
    form of the tree LQR (orc_tree_lqr_scan, option lqr_scan), element by element."""
    from paper_2506_13624_b300 import bmpc
    for seed in range(2):
        p = scenes.unicycle(seed) if cfg == "unicycle" else scenes.instances(cfg, 1, seed0=seed)[0]
        kk = max(1, min(k, _orc(p)["inner_iters"] - 2))
        it = _orc(p, max_iters=kk)
        warm = tuple(_fp32(it[key]) for key in ("x", "u", "lam", "y"))
        b = bmpc.Batch([p])
        b.set_problems(warm=[warm])
        b.solve(bmpc.default_opts(max_iters=1, variant=4))
        g = b.get_solutions()[0]
        b.close()
        r = _orc(p, max_iters=1, warm=warm, lqr_scan=1)
        assert g["inner_iters"] == r["inner_iters"] == 1
        for key in ("x", "u", "lam", "y"):
            a, c = g[key], r[key]
            if c.size:
                d = float(np.abs(a - c).max()) / max(1.0, float(np.abs(c).max()))
                assert d <= STEP_TOL[key], (cfg, seed, key, d)


# ------------------------------------------------------------------ per-branch dynamics (Sec. V-A)
@pytest.mark.parametrize("variant,bt", [(1, 64), (2, 64), (0, 256)])
def test_per_edge_dynamics_one_iteration(variant, bt):
    """Mass-spring trees whose spring constant differs per branch (every edge its own A_m, B_m): the
    linear-quadratic problem is solved in one iteration, equal to the oracle's (which equals the dense
    QP solution, pinned on the CPU)."""
    ps = [scenes.mass_spring(0, N=20, Nr=2), scenes.mass_spring(1, N=12, Nr=3), scenes.mass_spring(2, N=30, Nr=5)]
    gres = _gpu(ps, variant=variant, block_threads=bt)
    for p, g in zip(ps, gres):
        r = _orc(p)
        assert g["status"] == oracle.OK and g["inner_iters"] == 1 == r["inner_iters"]
        np.testing.assert_allclose(g["u"], r["u"], atol=1e-4 * max(1.0, np.abs(r["u"]).max()))
        np.testing.assert_allclose(g["x"], r["x"], atol=1e-4 * max(1.0, np.abs(r["x"]).max()))


def test_per_edge_dynamics_constrained_parity():
    """The same trees with bounded forces (the AL method with active input bounds) against the oracle."""
    ps = [scenes.mass_spring(s, N=20, Nr=3, constrained=True) for s in range(4)]
    print(_run_config(ps, min_match=1.0))
    print(_run_config(ps, min_match=1.0, variant=1))


def test_per_edge_dynamics_refuses_sweeps_without_edges():
    """The 8-lane, scan and jump sweeps read one model per node: a batch with per-edge dynamics is
    refused for them, with nothing launched."""
    from paper_2506_13624_b300 import bmpc
    b = bmpc.Batch([scenes.mass_spring(0)])
    b.set_problems()
    for v in (3, 4, 5):
        with pytest.raises(RuntimeError):
            b.solve(bmpc.default_opts(variant=v))
    b.solve(bmpc.default_opts(variant=2))
    assert b.get_solutions()[0]["status"] == oracle.OK
    b.close()


# ------------------------------------------------------------------ exact Hessian (Sec. IV-A)
def _exact_cases():
    return (scenes.instances(1, 6) + scenes.instances(2, 3) + [scenes.unicycle(s) for s in range(6)]
            + [scenes.unicycle(s, splits={1: 2, 10: 2}) for s in range(2)]
            + [scenes.mass_spring(s, N=20, Nr=3, constrained=True) for s in range(2)])


@pytest.mark.parametrize("variant", [0, 1, 5])
def test_exact_hessian_parity(variant):
    """The exact Hessian of the Lagrangian with eigenvalue modification on both sides (the GPU's
    hyper-dual second derivatives and Jacobi eigen-decomposition in FP32 against the oracle's in
    FP64), whole solves on every model and tree family, under the per-path, level and jump sweeps."""
    ps = _exact_cases()
    if variant == 5:   # the jump sweep reads one model per node: no per-edge dynamics
        ps = [p for p in ps if p.get("Aedge") is None]
    print(_run_config(ps, orc_kw={"hessian": 1}, variant=variant, hessian=1))


@pytest.mark.parametrize("cfg,k", [(1, 0), (1, 3), (2, 0), (2, 4), (3, 0), (3, 6), ("unicycle", 5)])
def test_exact_hessian_one_iteration(cfg, k):
    """One exact-Hessian iteration from an identical FP32 iterate, element by element: the modified
    blocks enter the Riccati recursion, the merit slope and the curvature test, so a wrong second
    derivative or a wrong eigenvalue floor moves the step."""
    for seed in range(2):
        p = scenes.unicycle(seed) if cfg == "unicycle" else scenes.instances(cfg, 1, seed0=seed)[0]
        g, r = _one_iteration(p, k, hessian=1)
        assert g["inner_iters"] == r["inner_iters"] == 1 and g["status"] == r["status"]
        for key in ("x", "u", "lam", "y"):
            a, c = g[key], r[key]
            if c.size:
                d = float(np.abs(a - c).max()) / max(1.0, float(np.abs(c).max()))
                assert d <= STEP_TOL[key], (cfg, k, seed, key, d)


def test_exact_hessian_refuses_diagonal_cost_sweeps():
    """The 8-lane and scan sweeps assume the diagonal cost blocks: with hessian = 1 they are refused
    and nothing runs; the linear-quadratic problem (no curvature beyond the cost) is solved in one
    iteration either way."""
    from paper_2506_13624_b300 import bmpc
    b = bmpc.Batch(scenes.instances(1, 2))
    b.set_problems()
    for v in (3, 4):
        with pytest.raises(RuntimeError):
            b.solve(bmpc.default_opts(variant=v, hessian=1))
    b.close()
    ps = [scenes.mass_spring(0, N=20, Nr=2), scenes.linear_problem(1, N=12, splits={2: 3})]
    for g, p in zip(_gpu(ps, hessian=1), ps):
        r = _orc(p)
        assert g["status"] == oracle.OK and g["inner_iters"] == 1 == r["inner_iters"]
        np.testing.assert_allclose(g["u"], r["u"], atol=1e-4 * max(1.0, np.abs(r["u"]).max()))


def test_exact_hessian_dynamic_bicycle_parity():
    """The exact option on the dynamic bicycle (config 3: n_x = 6, four RK4 substeps, tyre slip
    angles): whole solves against the oracle's exact option, the same bar as Gauss-Newton."""
    ps = scenes.instances(3, 2, seed0=1)
    print(_run_config(ps, min_match=0.5, orc_kw={"hessian": 1}, hessian=1))


@pytest.mark.parametrize("model", [0, 1])
def test_sweep_records_match_the_component_rows(model):
    """The per-path sweeps on node-major records and on the component-major rows give the same
    solution bit for bit: the records carry exactly the rows' values and the forward step does the
    same arithmetic.  A problem solved alone uses the records (its threads' staging fits in shared
    memory); next to a tree with 128 (dynamic) or 256 (kinematic) scenario paths in the same launch
    the staging no longer fits and every problem of the launch sweeps on the rows."""
    if model == 1:
        small = [scenes.config3(0)]
        wide = scenes.batch_problems(7, 1, model=1, N=50, splits={1: 2, 4: 2, 8: 2, 12: 2, 16: 2, 20: 2, 30: 2})
    else:
        small = [scenes.config2(1)]
        wide = scenes.batch_problems(7, 1, model=0, N=24, splits={1: 2, 3: 2, 5: 2, 7: 2, 9: 2, 11: 2, 13: 2, 15: 2})
    assert int(wide[0]["n"]) > 1000
    alone = _gpu(small, block_threads=512, variant=2)[0]
    mixed = _gpu(small + wide, block_threads=512, variant=2)[0]
    assert alone["status"] == oracle.OK
    for key in ("x", "u", "lam", "y"):
        assert np.array_equal(alone[key], mixed[key]), key
    for key in ("status", "inner_iters", "outer_iters", "ls_evals"):
        assert alone[key] == mixed[key], key
