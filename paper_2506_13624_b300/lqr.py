"""Binding of the general-size tree LQR (include/bmpc_lqr.h): argument marshalling only.

The solve runs in ``libbmpc.so``: the backward Riccati recursion with per-edge dynamics, then the
forward sweep, either as a launch per stage and sweep or as one block per problem (the header's
schedules).  Inputs and outputs are float32 CUDA tensors in the header's layout; there is no CPU
path.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import bmpc

_done = False


def _lib():
    global _done
    L = bmpc.lib()
    if not _done:
        L.bmpc_lqr_create.argtypes = [C.c_int32, C.POINTER(C.c_int32), C.c_int32, C.c_int32, C.c_int32, C.c_void_p,
                                      C.POINTER(C.c_void_p)]
        L.bmpc_lqr_solve.argtypes = [C.c_void_p] + [C.c_void_p] * 16
        L.bmpc_lqr_status.argtypes = [C.c_void_p]
        L.bmpc_lqr_stages.argtypes = [C.c_void_p]
        L.bmpc_lqr_set_schedule.argtypes = [C.c_void_p, C.c_int32]
        L.bmpc_lqr_fused.argtypes = [C.c_void_p]
        L.bmpc_lqr_destroy.argtypes = [C.c_void_p]
        L.bmpc_lqr_destroy.restype = None
        _done = True
    return L


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


class TreeLQR:
    """A batch of `batch` tree LQR problems on one tree (parent array in level order), n_x <= 32,
    n_u <= 16, bound to a CUDA stream (default: torch's current stream)."""

    def __init__(self, parent, nx: int, nu: int, batch: int = 1, stream=None, schedule: int = 0):
        import torch
        self.torch = torch
        self.parent = np.ascontiguousarray(parent, dtype=np.int32)
        self.n, self.nx, self.nu, self.batch = int(self.parent.shape[0]), int(nx), int(nu), int(batch)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        h = C.c_void_p()
        bmpc._check(_lib().bmpc_lqr_create(self.n, self.parent.ctypes.data_as(C.POINTER(C.c_int32)), self.nx,
                                           self.nu, self.batch, C.c_void_p(self.stream.cuda_stream), C.byref(h)),
                    "bmpc_lqr_create")
        self.handle = h
        bmpc._check(_lib().bmpc_lqr_set_schedule(h, int(schedule)), "bmpc_lqr_set_schedule")
        dev = torch.device("cuda", torch.cuda.current_device())
        b, n, nx, nu = self.batch, self.n, self.nx, self.nu
        z = lambda *s: torch.zeros(s, dtype=torch.float32, device=dev)
        self.out = dict(K=z(b, n, nu, nx), k=z(b, n, nu), P=z(b, n, nx, nx), p=z(b, n, nx), x=z(b, n, nx),
                        u=z(b, n, nu), lam=z(b, n, nx))

    @property
    def stages(self) -> int:
        return int(_lib().bmpc_lqr_stages(self.handle))

    @property
    def fused(self) -> bool:
        """True when solves run as one block per problem (one launch), False when per stage."""
        return bool(_lib().bmpc_lqr_fused(self.handle))

    def solve(self, Q, R, q, r, A, B, c, x0, M=None, check=True):
        """Queues one solve on the handle's stream; returns the output tensors (K, k, P, p, x, u, lam).
        With check, waits and raises on a non-positive-definite H."""
        torch = self.torch
        for name, t in (("Q", Q), ("R", R), ("q", q), ("r", r), ("A", A), ("B", B), ("c", c), ("x0", x0)):
            if not (t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()):
                raise ValueError(f"{name}: a contiguous float32 CUDA tensor is required")
        o = self.out
        bmpc._check(_lib().bmpc_lqr_solve(self.handle, _ptr(Q), _ptr(M), _ptr(R), _ptr(q), _ptr(r), _ptr(A),
                                          _ptr(B), _ptr(c), _ptr(x0), _ptr(o["K"]), _ptr(o["k"]), _ptr(o["P"]),
                                          _ptr(o["p"]), _ptr(o["x"]), _ptr(o["u"]), _ptr(o["lam"])),
                    "bmpc_lqr_solve")
        if check:
            self.status()
        return o

    def status(self):
        return bmpc._check(_lib().bmpc_lqr_status(self.handle), "bmpc_lqr (H not positive definite)")

    def close(self):
        if self.handle:
            _lib().bmpc_lqr_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
