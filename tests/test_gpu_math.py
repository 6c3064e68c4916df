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
