"""Thin binding of the learned warm-start network (include/bmpc_mlp.h).

Torch tensors hold the weights, AdamW moments, gradients and activations; every
computation (tensor-core GEMMs, GELU, loss, back-propagation, AdamW, feature and
start kernels) runs in libbmpc.so.
"""
from __future__ import annotations

import ctypes as C

from .bmpc import _check, lib

MAX_LAYERS = 8
_u16p = C.POINTER(C.c_uint16)
_fp = C.POINTER(C.c_float)


class Layer(C.Structure):
    _fields_ = [("in_", C.c_int32), ("out", C.c_int32), ("w_bf16", C.c_void_p), ("w", C.c_void_p),
                ("w_m", C.c_void_p), ("w_v", C.c_void_p), ("b", C.c_void_p), ("b_m", C.c_void_p),
                ("b_v", C.c_void_p), ("dw", C.c_void_p), ("db", C.c_void_p)]


class Work(C.Structure):
    _fields_ = [("pre", C.c_void_p * MAX_LAYERS), ("act", C.c_void_p * MAX_LAYERS), ("dy0", C.c_void_p),
                ("dy1", C.c_void_p), ("pred", C.c_void_p), ("loss", C.c_void_p), ("splitk", C.c_void_p),
                ("splitk_floats", C.c_int64)]


def _setup():
    L = lib()
    if getattr(L, "_mlp_ready", False):
        return L
    L.bmpc_mlp_init.argtypes = [C.POINTER(Layer), C.c_int32, C.c_uint64, C.c_void_p]
    L.bmpc_mlp_forward.argtypes = [C.POINTER(Layer), C.c_int32, C.c_void_p, C.c_int32, C.POINTER(Work), C.c_void_p]
    L.bmpc_mlp_train_step.argtypes = [C.POINTER(Layer), C.c_int32, C.c_void_p, C.c_void_p, C.c_int32, C.c_float,
                                      C.c_float, C.c_int32, C.POINTER(Work), C.c_void_p]
    L.bmpc_mlp_gemm.argtypes = [C.c_void_p, C.c_int32, C.c_int32, C.c_void_p, C.c_int32, C.c_int32, C.c_void_p,
                                C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.c_void_p]
    L.bmpc_mlp_status.argtypes = [C.c_void_p]
    L.bmpc_mlp_selftest_wait.argtypes = [C.c_int64, C.c_void_p]
    L.bmpc_mlp_workspace_floats.argtypes = [C.POINTER(Layer), C.c_int32, C.c_int32]
    L.bmpc_mlp_workspace_floats.restype = C.c_int64
    L.bmpc_mlp_features.argtypes = [C.c_void_p, C.c_void_p, C.c_int32, C.c_int32, C.c_int32]
    L.bmpc_mlp_targets.argtypes = [C.c_void_p, C.c_void_p, C.c_int64, C.c_int32]
    L.bmpc_mlp_start.argtypes = [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64,
                                 C.c_int32]
    L.bmpc_mlp_standardize.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_int32,
                                       C.c_void_p]
    L._mlp_ready = True
    return L


def _stream(torch):
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def gemm(A, B, trans_a=False, trans_b=False):
    """C = op(A) op(B) in fp32 from bf16 CUDA tensors (M, N multiples of 128, K of 64)."""
    import torch
    L = _setup()
    M = A.shape[1] if trans_a else A.shape[0]
    K = A.shape[0] if trans_a else A.shape[1]
    N = B.shape[0] if trans_b else B.shape[1]
    Cm = torch.empty((M, N), dtype=torch.float32, device=A.device)
    rc = L.bmpc_mlp_gemm(A.data_ptr(), A.shape[1], int(trans_a), B.data_ptr(), B.shape[1], int(trans_b),
                         Cm.data_ptr(), N, M, N, K, _stream(torch))
    if rc != 0:
        raise RuntimeError(f"bmpc_mlp_gemm failed: {rc}")
    return Cm


class MLP:
    """Multilayer perceptron dims[0] -> ... -> dims[-1] (GELU between layers), widths multiples of 128."""

    def __init__(self, dims, device="cuda", seed=0):
        import torch
        assert all(d % 128 == 0 for d in dims) and 2 <= len(dims) <= MAX_LAYERS + 1
        self.torch = torch
        self.dims = list(dims)
        self.device = torch.device(device)
        self.params = []
        self.c_layers = (Layer * (len(dims) - 1))()
        for l, (a, b) in enumerate(zip(dims[:-1], dims[1:])):
            f32 = dict(dtype=torch.float32, device=self.device)
            t = dict(w_bf16=torch.empty((a, b), dtype=torch.bfloat16, device=self.device),
                     w=torch.empty((a, b), **f32), w_m=torch.empty((a, b), **f32), w_v=torch.empty((a, b), **f32),
                     b=torch.empty(b, **f32), b_m=torch.empty(b, **f32), b_v=torch.empty(b, **f32),
                     dw=torch.empty((a, b), **f32), db=torch.empty(b, **f32))
            self.params.append(t)
            cl = self.c_layers[l]
            cl.in_, cl.out = a, b
            for k, v in t.items():
                setattr(cl, k, v.data_ptr())
        _check(_setup().bmpc_mlp_init(self.c_layers, len(self.params), seed, _stream(torch)), "bmpc_mlp_init")
        self._work = {}
        self.step_count = 0

    def work(self, batch: int):
        if batch in self._work:
            return self._work[batch]
        torch = self.torch
        w = Work()
        keep = []
        for l, d in enumerate(self.dims[1:-1]):
            pre = torch.empty((batch, d), dtype=torch.bfloat16, device=self.device)
            act = torch.empty((batch, d), dtype=torch.bfloat16, device=self.device)
            keep += [pre, act]
            w.pre[l], w.act[l] = pre.data_ptr(), act.data_ptr()
        widest = max(self.dims[1:])
        dy0 = torch.empty((batch, widest), dtype=torch.bfloat16, device=self.device)
        dy1 = torch.empty((batch, widest), dtype=torch.bfloat16, device=self.device)
        pred = torch.empty((batch, self.dims[-1]), dtype=torch.float32, device=self.device)
        loss = torch.zeros(1, dtype=torch.float32, device=self.device)
        nws = _setup().bmpc_mlp_workspace_floats(self.c_layers, len(self.params), batch)
        ws = torch.empty(max(nws, 1), dtype=torch.float32, device=self.device)
        keep += [dy0, dy1, pred, loss, ws]
        w.dy0, w.dy1, w.pred, w.loss = dy0.data_ptr(), dy1.data_ptr(), pred.data_ptr(), loss.data_ptr()
        w.splitk, w.splitk_floats = (ws.data_ptr(), nws) if nws > 0 else (None, 0)
        self._work[batch] = (w, keep, pred, loss)
        return self._work[batch]

    def forward(self, x):
        """x: bf16 CUDA tensor [batch, dims[0]] -> fp32 prediction [batch, dims[-1]] (a view)."""
        w, _, pred, _ = self.work(x.shape[0])
        _check(_setup().bmpc_mlp_forward(self.c_layers, len(self.params), x.data_ptr(), x.shape[0], C.byref(w),
                                         _stream(self.torch)), "bmpc_mlp_forward")
        return pred

    def train_step(self, x, target, lr, weight_decay=0.0):
        """One AdamW step on (x, target), both bf16 [batch, ...]; returns the loss tensor (device)."""
        w, _, _, loss = self.work(x.shape[0])
        self.step_count += 1
        _check(_setup().bmpc_mlp_train_step(self.c_layers, len(self.params), x.data_ptr(), target.data_ptr(),
                                            x.shape[0], lr, weight_decay, self.step_count, C.byref(w),
                                            _stream(self.torch)), "bmpc_mlp_train_step")
        return loss


def status():
    """Synchronise the current stream; raise if a GEMM gave up waiting for its MMAs."""
    import torch
    _check(_setup().bmpc_mlp_status(_stream(torch)), "bmpc_mlp_status")


def status_code() -> int:
    """Synchronise the current stream; the raw status (0, -4 a GEMM wait gave up, -2 CUDA error)."""
    import torch
    return int(_setup().bmpc_mlp_status(_stream(torch)))


def selftest_wait(cycles: int):
    """Launch the bounded-wait self-test: a wait for a barrier phase that nothing completes, given
    up after `cycles` SM cycles and recorded like a GEMM timeout."""
    import torch
    _check(_setup().bmpc_mlp_selftest_wait(int(cycles), _stream(torch)), "bmpc_mlp_selftest_wait")


def features(batch, out, n_scen, n_obs):
    _check(_setup().bmpc_mlp_features(batch.handle, out.data_ptr(), out.shape[1], n_scen, n_obs), "bmpc_mlp_features")


def targets(batch, out, y_sqrt=1):
    _check(_setup().bmpc_mlp_targets(batch.handle, out.data_ptr(), out.shape[1], int(y_sqrt)), "bmpc_mlp_targets")


def starts(batch, pred, mean, std, out, y_sqrt=1):
    _check(_setup().bmpc_mlp_start(batch.handle, pred.data_ptr(), pred.shape[1], mean.data_ptr(), std.data_ptr(),
                                   out.data_ptr(), out.shape[1], int(y_sqrt)), "bmpc_mlp_start")


def standardize(raw, mean, std, out):
    import torch
    _check(_setup().bmpc_mlp_standardize(raw.data_ptr(), mean.data_ptr(), std.data_ptr(), out.data_ptr(),
                                         raw.shape[0], raw.shape[1], _stream(torch)), "bmpc_mlp_standardize")


def _main(argv=None):
    """Times C = A B on the tcgen05 GEMM for the given shape (used for profiling)."""
    import argparse
    import torch
    ap = argparse.ArgumentParser(description="time one tcgen05 GEMM shape")
    ap.add_argument("M", type=int)
    ap.add_argument("N", type=int)
    ap.add_argument("K", type=int)
    ap.add_argument("--ta", action="store_true")
    ap.add_argument("--tb", action="store_true")
    ap.add_argument("--reps", type=int, default=20)
    a = ap.parse_args(argv)
    torch.manual_seed(0)
    A = torch.randn((a.K, a.M) if a.ta else (a.M, a.K), device="cuda").to(torch.bfloat16)
    B = torch.randn((a.N, a.K) if a.tb else (a.K, a.N), device="cuda").to(torch.bfloat16)
    for _ in range(3):
        gemm(A, B, a.ta, a.tb)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(a.reps):
        gemm(A, B, a.ta, a.tb)
    e1.record()
    status()
    ms = e0.elapsed_time(e1) / a.reps
    print(f"M={a.M} N={a.N} K={a.K} ta={int(a.ta)} tb={int(a.tb)}: {ms:.3f} ms, "
          f"{2.0 * a.M * a.N * a.K / ms / 1e9:.1f} TFLOP/s")


if __name__ == "__main__":
    _main()
