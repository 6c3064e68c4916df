"""Host-only checks of the C ABI: the library loads, exports every symbol that
include/bmpc.h declares, and its host-side validation and sizing work without a GPU."""
import ctypes as C
import os
import re

import numpy as np
import pytest

import scenes
from paper_2506_13624_b300 import bmpc

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    src = open(os.path.join(ROOT, "include", "bmpc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = set(re.findall(r"\b(bmpc_[a-z_]+)\s*\(", src))
    return sorted(names)


def test_library_exports_every_declared_symbol():
    L = bmpc.lib()
    declared = _declared_functions()
    assert len(declared) >= 15
    for name in declared:
        assert hasattr(L, name), name
    assert set(declared) == set(bmpc.EXPORTED)


def test_library_exports_every_mlp_symbol():
    src = open(os.path.join(ROOT, "include", "bmpc_mlp.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = set(re.findall(r"\b(bmpc_mlp_[a-z_]+)\s*\(", src))
    assert len(names) >= 9
    L = bmpc.lib()
    for name in names:
        assert hasattr(L, name), name


def test_library_exports_every_tree_lqr_symbol():
    src = open(os.path.join(ROOT, "include", "bmpc_lqr.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = set(re.findall(r"\b(bmpc_lqr_[a-z_]+)\s*\(", src))
    assert names == {"bmpc_lqr_create", "bmpc_lqr_solve", "bmpc_lqr_status", "bmpc_lqr_stages", "bmpc_lqr_destroy",
                     "bmpc_lqr_set_schedule", "bmpc_lqr_fused"}
    L = bmpc.lib()
    for name in names:
        assert hasattr(L, name), name


@pytest.mark.parametrize("case", ["nx", "nu", "batch", "root", "order", "levels", "empty"])
def test_tree_lqr_rejects_bad_trees_and_sizes_on_the_host(case):
    """bmpc_lqr_create validates before any device call: sizes beyond n_x = 32 or n_u = 16, a
    root with a parent, a parent after its child, stages out of level order, an empty tree."""
    from paper_2506_13624_b300 import lqr
    parent, nx, nu, batch = np.array([-1, 0, 0, 1, 2], np.int32), 4, 2, 1
    if case == "nx":
        nx = 33
    elif case == "nu":
        nu = 17
    elif case == "batch":
        batch = 0
    elif case == "root":
        parent[0] = 0
    elif case == "order":
        parent = np.array([-1, 2, 0], np.int32)
    elif case == "levels":
        parent = np.array([-1, 0, 1, 0], np.int32)   # node 3 (stage 1) after node 2 (stage 2)
    n = 0 if case == "empty" else len(parent)
    h = C.c_void_p()
    rc = lqr._lib().bmpc_lqr_create(n, parent.ctypes.data_as(C.POINTER(C.c_int32)), nx, nu, batch, None,
                                    C.byref(h))
    assert rc == bmpc.ERR_INVALID and not h.value


def test_version_and_status_strings():
    assert b"sm_103a" in bmpc.lib().bmpc_version()
    for s in (0, 1, 2, -1, -2, -3, -4, -5):
        assert bmpc.status_str(s) != "unknown status"


def _sizes(problems):
    descs = (bmpc.TreeDesc * len(problems))()
    keep = []
    for k, p in enumerate(problems):
        d, par = bmpc.tree_desc(p)
        descs[k] = d
        keep.append(par)
    db, sb, hb = C.c_size_t(), C.c_size_t(), C.c_size_t()
    rc = bmpc.lib().bmpc_batch_bytes(descs, len(problems), C.byref(db), C.byref(sb), C.byref(hb))
    return rc, db.value, sb.value, hb.value


def test_batch_bytes_scale_with_nodes():
    rc1, d1, s1, h1 = _sizes([scenes.config1(0)])
    rc3, d3, s3, h3 = _sizes([scenes.config3(0)])
    assert rc1 == 0 and rc3 == 0
    assert s3 > 20 * s1 and d3 > 10 * d1
    # staging mirrors the data arena up to the statistics; the device-only flat-transfer region
    # (at least one float per node and state component) follows
    p1 = scenes.config1(0)
    assert h1 < d1 and d1 - h1 >= 4 * p1["n"] * (p1["nx"] + 1)
    rc, d, s, h = _sizes(scenes.config4(4, 16))
    assert rc == 0 and s % 4 == 0


@pytest.mark.parametrize("mutate", ["not_level_order", "parent_after", "bad_root", "bad_model", "too_many_obs",
                                    "one_node", "bad_substeps", "edge_on_vehicle"])
def test_invalid_trees_rejected_on_host(mutate):
    p = dict(scenes.config1(0))
    par = p["parent"].copy()
    if mutate == "not_level_order":
        par[5], par[6] = par[6], par[5]          # children of a node not contiguous
        par[4] = 30
    elif mutate == "parent_after":
        par[10] = 11
    elif mutate == "bad_root":
        par[0] = 0
    elif mutate == "bad_model":
        p["model"] = 1                            # nx = 4 with the dynamic model
    elif mutate == "too_many_obs":
        p["n_obs"] = 9
    elif mutate == "one_node":
        par = par[:1]
        p["n"] = 1
    elif mutate == "bad_substeps":
        p["params"] = p["params"].copy()
        p["params"][9] = 0.0
    elif mutate == "edge_on_vehicle":               # per-edge dynamics exist for the linear model only
        p["Aedge"] = np.zeros((p["n"], 4, 4))
        p["Bedge"] = np.zeros((p["n"], 4, 2))
    p["parent"] = par
    rc, *_ = _sizes([p])
    assert rc == bmpc.ERR_INVALID


def test_default_opts_match_the_oracle_constants():
    """The library's defaults are the oracle's constants (Algorithm 1's failure branch, rho up to 1e6)
    with the library's convergence margin (oracle.PRODUCT_RULE); the cap rule is the option
    cap_rule = 1 on both sides."""
    import oracle
    o, r = bmpc.default_opts(), oracle.default_opts(**oracle.PRODUCT_RULE)
    for f in ("max_iters", "max_outer", "n_alpha", "cap_rule"):
        assert getattr(o, f) == getattr(r, f)
    for f in ("tau", "omega0", "eta0", "a_omega", "b_omega", "a_eta", "b_eta", "rho0", "rho_max",
              "mu0", "beta", "ls_rel_eps"):
        assert np.float32(getattr(o, f)) == np.float32(getattr(r, f)), f
    assert np.float32(o.eps_tol * o.kkt_margin) == np.float32(r.eps_tol)
    paper = oracle.default_opts()
    assert paper.cap_rule == 0 and paper.rho_max == 1e6 and o.cap_rule == 0
    cap = oracle.default_opts(**oracle.CAP_RULE)
    assert cap.cap_rule == 1 and cap.rho_max == 100.0


def test_single_tree_calls_cite_the_problem_statement():
    """Each call of the single-tree interface carries, in the comment right above its declaration,
    the passage of the paper that defines what it does."""
    src = open(os.path.join(ROOT, "include", "bmpc.h")).read()
    for name in ("bmpc_create_tree", "bmpc_set_problem", "bmpc_solve", "bmpc_get_solution"):
        m = re.search(r"/\*((?:(?!\*/).)*)\*/\s*int\s+" + name + r"\(", src, flags=re.S)
        assert m, name
        assert re.search(r"(Eq\.|Sec\.|Algorithm) ", m.group(1)), name


def test_set_stream_rejects_a_null_handle():
    assert bmpc.lib().bmpc_set_stream(None, None) == bmpc.ERR_INVALID



def test_async_read_and_wait_reject_null_handles():
    """The asynchronous flat read and its wait check their handle before any CUDA call."""
    L = bmpc.lib()
    assert L.bmpc_get_solutions_flat_async(None, None, None, None, None) == bmpc.ERR_INVALID
    assert L.bmpc_wait_solutions(None, None) == bmpc.ERR_INVALID


def test_wait_selftest_rejects_out_of_range_limits():
    """The bounded-wait self-test checks its limit before launching anything."""
    from paper_2506_13624_b300 import mlp
    L = mlp._setup()
    assert L.bmpc_mlp_selftest_wait(0, None) == -1
    assert L.bmpc_mlp_selftest_wait(10 ** 9, None) == -1


def test_default_options_match_their_documentation():
    """bmpc_default_opts (host only) sets the constants include/bmpc.h documents: the readings of the
    paper's unstated constants (rho0 = 10, rho_max = 1e6, mu0 = 1, Armijo beta = 1e-4, alpha_i = 2^-i
    for i < 10, 50 inner iterations), Algorithm 1's failure branch, the compensated iterate and
    automatic launch geometry."""
    o = bmpc.default_opts()
    assert (o.max_iters, o.max_outer, o.n_alpha) == (50, 60, 10)
    assert o.eps_tol == np.float32(1e-5) and o.tau == 100.0
    assert (o.omega0, o.a_omega, o.b_omega, o.a_eta) == (1.0, 1.0, 1.0, np.float32(0.1))
    assert o.eta0 == np.float32(0.1) and o.b_eta == np.float32(0.9)
    assert (o.rho0, o.rho_max, o.mu0, o.cap_rule) == (10.0, 1e6, 1.0, 0)
    assert o.kkt_margin == np.float32(0.8) and o.compensated == 1 and o.hessian == 0
    assert o.beta == np.float32(1e-4) and o.ls_rel_eps == np.float32(1e-6)
    assert (o.block_threads, o.blocks_per_sm, o.variant, o.warm_select, o.queue_order) == (0, 0, 0, 0, 1)
    assert list(o.block_threads_model) == [0, 0, 0, 0]
    assert o.select_mu == 100.0 and o.select_rho == 1e4
    assert C.sizeof(bmpc.Opts) == 32 * 4   # 32 four-byte fields, as in bmpc_opts
