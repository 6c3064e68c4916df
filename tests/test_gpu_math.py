"""Elementary functions of the device dynamics against their error bound.

The vehicle right-hand sides (Sec. V, kinematic and dynamic bicycle) take sin and cos of the heading
at every RK4 stage from the library's own Cody-Waite reduction plus Taylor polynomials; the bound
stated for them in include/bmpc.h (about 1.5 ulp for |a| < 1e3) is checked here against float64
sin and cos, to 2 ulp of the true value.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _ulp_err(v, t):
    return np.abs(v - t) / np.spacing(np.abs(t).astype(np.float32)).astype(np.float64)


def test_sincos_within_two_ulp():
    import torch
    from paper_2506_13624_b300 import bmpc
    rng = np.random.default_rng(5)
    a = np.concatenate([
        rng.uniform(-np.pi, np.pi, 200_000),                        # headings
        rng.uniform(-1e3, 1e3, 200_000),                            # many turns
        10.0 ** rng.uniform(-30, 0, 50_000) * rng.choice([-1, 1], 50_000),   # small angles: sin a ~ a
        np.arange(-1273, 1274) * np.pi / 4,                         # near the zeros of sin and cos
        [0.0, -0.0, 1e-38, -1e-38],
    ]).astype(np.float32)
    s, c = bmpc.selftest_sincos(torch.from_numpy(a).cuda())
    torch.cuda.synchronize()
    s, c = s.cpu().numpy().astype(np.float64), c.cpu().numpy().astype(np.float64)
    a64 = a.astype(np.float64)
    es, ec = _ulp_err(s, np.sin(a64)), _ulp_err(c, np.cos(a64))
    assert es.max() <= 2.0, (es.max(), a[es.argmax()])
    assert ec.max() <= 2.0, (ec.max(), a[ec.argmax()])
    # tan(delta) = sin / cos of the kinematic model stays within a few ulp on the steering range
    d = np.abs(a64) <= 0.6
    t = s[d] / c[d]
    assert _ulp_err(t, np.tan(a64[d])).max() <= 4.0


def test_selftest_rejects_bad_arguments():
    from paper_2506_13624_b300 import bmpc
    assert bmpc.lib().bmpc_selftest_sincos(None, None, None, -1, None) == bmpc.ERR_INVALID
    assert bmpc.lib().bmpc_selftest_sincos(None, None, None, 4, None) == bmpc.ERR_INVALID
    assert bmpc.lib().bmpc_selftest_sincos(None, None, None, 0, None) == 0


def _spectral(rng, n, ev):
    Qm, _ = np.linalg.qr(rng.standard_normal((n, n)))
    return (Qm * ev) @ Qm.T


@pytest.mark.parametrize("n", [6, 8])
def test_eigenvalue_modification_against_the_oracle(n):
    """The exact-Hessian option's eigenvalue modification on the GPU (a Cholesky test, then cyclic
    Jacobi rotations in FP32) against the oracle's FP64 Jacobi on the same FP32 inputs: definite
    blocks come back bit for bit; indefinite, rank-deficient and badly scaled ones equal the
    oracle's modified blocks to FP32 accuracy (1e-5 of the block's magnitude per entry, a few times
    the rounding of an n-step reconstruction) and have every eigenvalue at the floor or above."""
    import torch

    import oracle
    from paper_2506_13624_b300 import bmpc
    rng = np.random.default_rng(40 + n)
    mats = []
    for _ in range(16):                                       # well-conditioned, definite
        F = rng.standard_normal((n, n))
        mats.append(F @ F.T + np.eye(n))
    for _ in range(16):                                       # indefinite
        mats.append(_spectral(rng, n, rng.uniform(-5.0, 5.0, n)))
    for _ in range(16):                                       # rank-deficient (zero-weight directions)
        ev = rng.uniform(0.5, 2.0, n)
        ev[: n // 2] = 0.0
        mats.append(_spectral(rng, n, ev))
    for _ in range(16):                                       # large, with a negative direction
        ev = rng.uniform(1.0, 1e3, n)
        ev[0] = -rng.uniform(1.0, 10.0)
        mats.append(_spectral(rng, n, ev))
    S = np.array(mats, np.float32)
    S = 0.5 * (S + np.transpose(S, (0, 2, 1)))
    got = bmpc.selftest_eig_modify(torch.tensor(S, device="cuda")).cpu().numpy().astype(np.float64)
    assert np.array_equal(got[:16], S[:16].astype(np.float64))
    for k in range(16, len(S)):
        want = oracle.eig_modify(S[k].astype(np.float64))
        scale = max(1.0, float(np.abs(want).max()))
        assert np.abs(got[k] - want).max() <= 1e-5 * scale, (k, float(np.abs(got[k] - want).max()), scale)
        ev = np.linalg.eigvalsh(0.5 * (got[k] + got[k].T))
        floor = 1e-6 * max(1.0, float(np.abs(np.linalg.eigvalsh(S[k].astype(np.float64))).max()))
        assert ev.min() >= 0.5 * floor, (k, ev.min(), floor)


def test_eigenvalue_selftest_rejects_bad_arguments():
    import ctypes as C

    from paper_2506_13624_b300 import bmpc
    L = bmpc.lib()
    assert L.bmpc_selftest_eig_modify(None, 6, 1, None) == bmpc.ERR_INVALID
    assert L.bmpc_selftest_eig_modify(C.c_void_p(16), 7, 1, None) == bmpc.ERR_INVALID
    assert L.bmpc_selftest_eig_modify(C.c_void_p(16), 8, 0, None) == bmpc.ERR_INVALID


@pytest.mark.parametrize("which", ["kinematic", "dynamic", "unicycle"])
def test_dynamics_second_derivatives_against_the_oracle(which):
    """The exact-Hessian option's sum_i mu_i d^2 f_i / dz dz of the RK4 map on the GPU (hyper-dual
    FP32) against the oracle's (hyper-dual FP64, pinned on the CPU against central differences of
    the analytic Jacobian) at the same FP32 points, element by element: within 1e-4 of the
    block's magnitude (FP32 rounding carried through four RK4 stages of n_sub substeps)."""
    import torch

    import oracle
    import scenes
    from paper_2506_13624_b300 import bmpc
    rng = np.random.default_rng({"kinematic": 1, "dynamic": 2, "unicycle": 3}[which])
    p = {"kinematic": lambda: scenes.config1(0), "dynamic": lambda: scenes.config3(0),
         "unicycle": lambda: scenes.unicycle(0)}[which]()
    nx, count = int(p["nx"]), 64
    x = np.zeros((count, nx))
    x[:, 0] = rng.uniform(-20, 20, count)
    x[:, 1] = rng.uniform(-5, 5, count)
    x[:, 2] = rng.uniform(-0.6, 0.6, count)
    x[:, 3] = rng.uniform(2.0, 10.0, count)
    if nx == 6:
        x[:, 4] = rng.uniform(-0.5, 0.5, count)
        x[:, 5] = rng.uniform(-0.3, 0.3, count)
    u = np.stack([rng.uniform(-3, 3, count), rng.uniform(-0.5, 0.5, count)], axis=1)
    mu = rng.standard_normal((count, nx))
    x, u, mu = (np.asarray(a, np.float32) for a in (x, u, mu))
    dev = lambda a: torch.tensor(a, device="cuda")
    H = bmpc.selftest_dyn_hessian(int(p["model"]), np.asarray(p["params"], np.float32), float(np.float32(p["dt"])),
                                  dev(x), dev(u), dev(mu)).cpu().numpy().astype(np.float64)
    worst = 0.0
    for k in range(count):
        want = oracle.dyn_hessian(p, x[k].astype(np.float64), u[k].astype(np.float64), mu[k].astype(np.float64))
        scale = max(1.0, float(np.abs(want).max()))
        d = float(np.abs(H[k] - want).max()) / scale
        worst = max(worst, d)
        assert d <= 1e-4, (which, k, d)
        assert np.allclose(H[k], H[k].T, atol=1e-6 * scale)
    print(which, "worst", worst)
