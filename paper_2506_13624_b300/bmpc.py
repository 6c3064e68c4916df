"""Thin Python binding of the bmpc C ABI (include/bmpc.h).

Only argument marshalling lives here: every step of the solver runs in the
CUDA library ``libbmpc.so``.  PyTorch provides the device arenas, the pinned
host staging buffer and the CUDA stream.  There is no CPU fallback: importing
the binding without the built library, or calling it without a CUDA device,
raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libbmpc.so")

OK, MAX_ITER, LS_FAIL = 0, 1, 2
ERR_INVALID, ERR_CUDA, ERR_NUMERIC, ERR_TIMEOUT, ERR_SPACE = -1, -2, -3, -4, -5
MAX_NX, NU, MAX_OBS = 6, 2, 8
MODEL_KINEMATIC, MODEL_DYNAMIC, MODEL_LINEAR, MODEL_UNICYCLE = 0, 1, 2, 3

_fp = C.POINTER(C.c_float)
_ip = C.POINTER(C.c_int32)


class TreeDesc(C.Structure):
    _fields_ = [("num_nodes", C.c_int32), ("parent", _ip), ("nx", C.c_int32), ("nu", C.c_int32),
                ("model", C.c_int32), ("n_obs", C.c_int32), ("box_on", C.c_int32), ("lane_on", C.c_int32),
                ("dt", C.c_float), ("params", C.c_float * 10), ("edge_dynamics", C.c_int32)]


class Problem(C.Structure):
    _fields_ = [("x0", _fp), ("xref", _fp), ("weight", _fp), ("Qw", C.c_float * MAX_NX),
                ("QNw", C.c_float * MAX_NX), ("Rw", C.c_float * NU), ("u_lo", C.c_float * NU),
                ("u_hi", C.c_float * NU), ("lane_lo", C.c_float), ("lane_hi", C.c_float), ("obs", _fp),
                ("Alin", _fp), ("Blin", _fp), ("warm_x", _fp), ("warm_u", _fp), ("warm_lam", _fp),
                ("warm_y", _fp), ("Aedge", _fp), ("Bedge", _fp)]


class Opts(C.Structure):
    _fields_ = [("max_iters", C.c_int32), ("max_outer", C.c_int32), ("n_alpha", C.c_int32),
                ("eps_tol", C.c_float), ("tau", C.c_float), ("omega0", C.c_float), ("eta0", C.c_float),
                ("a_omega", C.c_float), ("b_omega", C.c_float), ("a_eta", C.c_float), ("b_eta", C.c_float),
                ("rho0", C.c_float), ("rho_max", C.c_float), ("mu0", C.c_float), ("beta", C.c_float),
                ("ls_rel_eps", C.c_float), ("ls_chunk", C.c_int32), ("block_threads", C.c_int32),
                ("blocks_per_sm", C.c_int32), ("variant", C.c_int32), ("warm_select", C.c_int32),
                ("select_mu", C.c_float), ("select_rho", C.c_float), ("queue_order", C.c_int32),
                ("block_threads_model", C.c_int32 * 4), ("cap_rule", C.c_int32),
                ("kkt_margin", C.c_float), ("compensated", C.c_int32), ("hessian", C.c_int32)]


class Stats(C.Structure):
    _fields_ = [("status", C.c_int32), ("inner_iters", C.c_int32), ("outer_iters", C.c_int32),
                ("ls_fail_total", C.c_int32), ("ls_evals", C.c_int32), ("start_used", C.c_int32),
                ("r_kkt", C.c_float), ("c", C.c_float), ("rho", C.c_float),
                ("mu", C.c_float), ("cycles_linearise", C.c_int64), ("cycles_backward", C.c_int64),
                ("cycles_forward", C.c_int64), ("cycles_linesearch", C.c_int64), ("cycles_total", C.c_int64)]


_lib = None


def lib() -> C.CDLL:
    """Load the in-tree CUDA library (fails loudly when it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: run paper_2506_13624_b300/build.py (nvcc, sm_103a)")
        L = C.CDLL(LIB_PATH)
        L.bmpc_status_str.restype = C.c_char_p
        L.bmpc_version.restype = C.c_char_p
        sz = C.POINTER(C.c_size_t)
        L.bmpc_batch_bytes.argtypes = [C.POINTER(TreeDesc), C.c_int32, sz, sz, sz]
        L.bmpc_create_batch.argtypes = [C.POINTER(TreeDesc), C.c_int32, C.c_void_p, C.c_size_t, C.c_void_p,
                                        C.c_size_t, C.c_void_p, C.c_size_t, C.c_void_p, C.POINTER(C.c_void_p)]
        L.bmpc_set_problems.argtypes = [C.c_void_p, C.POINTER(Problem)]
        L.bmpc_solve_batch.argtypes = [C.c_void_p, C.POINTER(Opts)]
        L.bmpc_solve_batch_graph.argtypes = [C.c_void_p, C.POINTER(Opts)]
        L.bmpc_get_solutions.argtypes = [C.c_void_p, _fp, _fp, _fp, _fp, C.POINTER(Stats)]
        L.bmpc_destroy_batch.argtypes = [C.c_void_p]
        L.bmpc_default_opts.argtypes = [C.POINTER(Opts)]
        L.bmpc_autotune.argtypes = [C.c_void_p, C.POINTER(Opts), C.POINTER(Opts), C.POINTER(C.c_float)]
        L.bmpc_set_warm_start_device.argtypes = [C.c_void_p, C.c_void_p, C.c_int64, C.c_int32]
        L.bmpc_shift_warm_start.argtypes = [C.c_void_p, C.c_void_p, C.c_int32]
        L.bmpc_create_batch_static.argtypes = [C.POINTER(TreeDesc), C.c_int32, C.c_void_p, C.c_size_t, C.c_void_p,
                                               C.c_size_t, C.c_void_p, C.POINTER(C.c_void_p)]
        L.bmpc_problem_device_outputs.argtypes = [C.c_void_p, C.c_int32, C.POINTER(C.c_void_p),
                                                  C.POINTER(C.c_void_p), C.POINTER(C.c_void_p),
                                                  C.POINTER(C.c_void_p), C.POINTER(C.c_int32)]
        L.bmpc_get_queue_order.argtypes = [C.c_void_p, C.POINTER(C.c_int32)]
        L.bmpc_transfer_bytes.argtypes = [C.c_void_p, C.POINTER(C.c_size_t), C.POINTER(C.c_size_t),
                                          C.POINTER(C.c_size_t)]
        L.bmpc_transfer_bytes_flat.argtypes = [C.c_void_p, C.POINTER(C.c_size_t), C.POINTER(C.c_size_t)]
        L.bmpc_set_problems_flat.argtypes = [C.c_void_p, C.POINTER(Problem), C.c_void_p, C.c_void_p, C.c_void_p]
        L.bmpc_get_solutions_flat.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                              C.POINTER(Stats)]
        L.bmpc_selftest_sincos.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p]
        L.bmpc_selftest_eig_modify.argtypes = [C.c_void_p, C.c_int32, C.c_int32, C.c_void_p]
        L.bmpc_selftest_dyn_hessian.argtypes = [C.c_int32, C.POINTER(C.c_float), C.c_float, C.c_void_p, C.c_void_p,
                                                C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p]
        L.bmpc_get_solutions_flat_async.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
        L.bmpc_wait_solutions.argtypes = [C.c_void_p, C.POINTER(Stats)]
        L.bmpc_set_stream.argtypes = [C.c_void_p, C.c_void_p]
        L.bmpc_selftest_fma.argtypes = [C.c_void_p, C.c_int32, C.c_int32, C.c_void_p]
        _lib = L
    return _lib


EXPORTED = ["bmpc_default_opts", "bmpc_batch_bytes", "bmpc_create_batch", "bmpc_set_problems", "bmpc_solve_batch",
            "bmpc_solve_batch_graph", "bmpc_get_solutions", "bmpc_problem_device_outputs", "bmpc_destroy_batch",
            "bmpc_tree_bytes", "bmpc_create_tree", "bmpc_set_problem", "bmpc_solve", "bmpc_get_solution",
            "bmpc_destroy_tree", "bmpc_status_str", "bmpc_version", "bmpc_create_batch_static", "bmpc_autotune",
            "bmpc_set_warm_start_device", "bmpc_shift_warm_start", "bmpc_get_queue_order", "bmpc_transfer_bytes",
            "bmpc_set_problems_flat", "bmpc_get_solutions_flat", "bmpc_transfer_bytes_flat", "bmpc_selftest_sincos",
            "bmpc_get_solutions_flat_async", "bmpc_wait_solutions", "bmpc_set_stream", "bmpc_selftest_fma",
            "bmpc_selftest_eig_modify", "bmpc_selftest_dyn_hessian"]

STATIC_SCRATCH_BYTES = 16 << 20


def selftest_sincos(a):
    """Device sine and cosine of the vehicle dynamics on a float32 CUDA tensor of angles."""
    import torch
    assert a.is_cuda and a.dtype == torch.float32 and a.is_contiguous()
    s, c = torch.empty_like(a), torch.empty_like(a)
    with torch.cuda.device(a.device):
        _check(lib().bmpc_selftest_sincos(a.data_ptr(), s.data_ptr(), c.data_ptr(), a.numel(),
                                          torch.cuda.current_stream(a.device).cuda_stream), "bmpc_selftest_sincos")
    return s, c


def selftest_eig_modify(S):
    """The exact-Hessian option's eigenvalue modification on a float32 CUDA tensor [count, n, n]
    (n = 6 or 8); returns the modified copy."""
    import torch
    assert S.is_cuda and S.dtype == torch.float32 and S.dim() == 3 and S.shape[1] == S.shape[2]
    out = S.contiguous().clone()
    with torch.cuda.device(S.device):
        _check(lib().bmpc_selftest_eig_modify(out.data_ptr(), S.shape[1], S.shape[0],
                                              torch.cuda.current_stream(S.device).cuda_stream),
               "bmpc_selftest_eig_modify")
    return out


def selftest_dyn_hessian(model, params, dt, x, u, mu):
    """The exact-Hessian option's second derivatives of the dynamics on the device: float32 CUDA
    tensors x, mu [count, nx], u [count, 2]; returns H [count, nx + 2, nx + 2]."""
    import torch
    x, u, mu = x.contiguous(), u.contiguous(), mu.contiguous()
    count, nx = x.shape
    H = torch.empty((count, nx + 2, nx + 2), dtype=torch.float32, device=x.device)
    prm = (C.c_float * 10)(*[float(v) for v in params])
    with torch.cuda.device(x.device):
        _check(lib().bmpc_selftest_dyn_hessian(int(model), prm, float(dt), x.data_ptr(), u.data_ptr(), mu.data_ptr(),
                                               H.data_ptr(), count, torch.cuda.current_stream(x.device).cuda_stream),
               "bmpc_selftest_dyn_hessian")
        torch.cuda.current_stream(x.device).synchronize()
    return H


def fp32_peak_tflops(reps: int = 5) -> float:
    """Measured FP32 FMA throughput of the current device (TFLOP/s): the library's FMA kernel over
    8 blocks of 256 threads per SM, timed with CUDA events on the current stream, best of `reps`."""
    import torch
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    blocks, iters = 8 * sms, 50000
    out = torch.empty(blocks * 256, dtype=torch.float32, device="cuda")
    s = torch.cuda.current_stream()
    best = 0.0
    for r in range(reps + 1):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        _check(lib().bmpc_selftest_fma(out.data_ptr(), blocks, iters, C.c_void_p(s.cuda_stream)), "bmpc_selftest_fma")
        e1.record(s)
        e1.synchronize()
        if r:
            best = max(best, 2.0 * 8 * iters * 256 * blocks / (e0.elapsed_time(e1) * 1e-3) / 1e12)
    return best


def status_str(s: int) -> str:
    return lib().bmpc_status_str(int(s)).decode()


def _check(rc: int, what: str):
    if rc < 0:
        raise RuntimeError(f"{what} failed: {rc} ({status_str(rc)})")
    return rc


def default_opts(**kw) -> Opts:
    o = Opts()
    lib().bmpc_default_opts(C.byref(o))
    for k, v in kw.items():
        if k == "block_threads_model":
            v = (C.c_int32 * 4)(*v)
        setattr(o, k, v)
    return o


def n_con(p) -> int:
    return 2 * NU * int(p["box_on"]) + int(p["n_obs"]) + 2 * int(p["lane_on"])


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def tree_desc(p) -> tuple[TreeDesc, np.ndarray]:
    parent = np.ascontiguousarray(p["parent"], dtype=np.int32)
    d = TreeDesc()
    d.num_nodes = int(p["n"])
    d.parent = parent.ctypes.data_as(_ip)
    d.nx, d.nu, d.model = int(p["nx"]), int(p["nu"]), int(p["model"])
    d.n_obs, d.box_on, d.lane_on = int(p["n_obs"]), int(p["box_on"]), int(p["lane_on"])
    d.dt = float(p["dt"])
    for j, v in enumerate(np.asarray(p["params"], dtype=np.float64)[:10]):
        d.params[j] = float(v)
    d.edge_dynamics = 1 if p.get("Aedge") is not None else 0
    return d, parent


class _ProblemData:
    """float32 copies of one problem's arrays, kept alive while the C struct points at them."""

    def __init__(self, p, warm=None):
        nx = int(p["nx"])
        self.keep = [_f32(p["x0"]), _f32(p["xref"]), _f32(p["weight"]), _f32(p["obs"]),
                     _f32(p["Alin"]), _f32(p["Blin"])]
        s = Problem()
        s.x0, s.xref, s.weight, s.obs, s.Alin, s.Blin = (a.ctypes.data_as(_fp) for a in self.keep)
        if p.get("Aedge") is not None:
            ae, be = _f32(p["Aedge"]), _f32(p["Bedge"])
            self.keep += [ae, be]
            s.Aedge, s.Bedge = ae.ctypes.data_as(_fp), be.ctypes.data_as(_fp)
        for j in range(nx):
            s.Qw[j], s.QNw[j] = float(p["Qw"][j]), float(p["QNw"][j])
        for j in range(NU):
            s.Rw[j], s.u_lo[j], s.u_hi[j] = float(p["Rw"][j]), float(p["u_lo"][j]), float(p["u_hi"][j])
        s.lane_lo, s.lane_hi = float(p["lane_lo"]), float(p["lane_hi"])
        if warm is not None:
            nc = n_con(p)
            w = [_f32(a) for a in warm]
            if nc == 0:
                w[3] = np.zeros((int(p["n"]), 1), np.float32)
            self.keep += w
            s.warm_x, s.warm_u, s.warm_lam, s.warm_y = (a.ctypes.data_as(_fp) for a in w)
        self.s = s


class Batch:
    """A batch of BMPC problems resident on one GPU (a single tree is a batch of one).

    Device arenas and the pinned staging buffer are torch tensors owned by this object.
    """

    def __init__(self, problems, device=None, stream=None, pinned: bool = True):
        import torch

        if not torch.cuda.is_available():
            raise RuntimeError("bmpc needs a CUDA device (no CPU fallback)")
        self.torch = torch
        self.problems = list(problems)
        self.n = len(self.problems)
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        descs = (TreeDesc * self.n)()
        self._parents = []
        for k, p in enumerate(self.problems):
            d, par = tree_desc(p)
            descs[k] = d
            self._parents.append(par)
        self._descs = descs
        db, sb, hb = C.c_size_t(), C.c_size_t(), C.c_size_t()
        _check(lib().bmpc_batch_bytes(descs, self.n, C.byref(db), C.byref(sb), C.byref(hb)), "bmpc_batch_bytes")
        self.data_bytes, self.scratch_bytes, self.staging_bytes = db.value, sb.value, hb.value
        with torch.cuda.device(self.device):
            self._data = torch.empty(self.data_bytes + 256, dtype=torch.uint8, device=self.device)
            self._scr = torch.empty(self.scratch_bytes + 256, dtype=torch.uint8, device=self.device)
        self._stage = torch.empty(self.staging_bytes, dtype=torch.uint8, pin_memory=pinned)
        dptr = (self._data.data_ptr() + 255) // 256 * 256
        sptr = (self._scr.data_ptr() + 255) // 256 * 256
        h = C.c_void_p()
        with torch.cuda.device(self.device):
            _check(lib().bmpc_create_batch(descs, self.n, dptr, self.data_bytes, sptr, self.scratch_bytes,
                                           self._stage.data_ptr(), self.staging_bytes,
                                           C.c_void_p(self.stream.cuda_stream), C.byref(h)), "bmpc_create_batch")
        self.handle = h
        self.nodes = np.array([int(p["n"]) for p in self.problems])
        self.nx = np.array([int(p["nx"]) for p in self.problems])
        self.nc = np.array([n_con(p) for p in self.problems])

    def set_problems(self, problems=None, warm=None, reuse: bool = False):
        """Upload problem data (and optional warm starts: list of (x, u, lam, y) or None).

        With reuse=True the problem descriptors of the previous call are uploaded again: the caller
        has updated the same float32 arrays in place (x0, xref, obstacles, ...), as a control loop
        that keeps one buffer per problem does."""
        if not (reuse and getattr(self, "_arr", None) is not None):
            probs = self.problems if problems is None else list(problems)
            arr = (Problem * self.n)()
            self._pd = [_ProblemData(p, None if warm is None else warm[k]) for k, p in enumerate(probs)]
            for k, pd in enumerate(self._pd):
                arr[k] = pd.s
            self._arr = arr
        with self.torch.cuda.device(self.device):
            _check(lib().bmpc_set_problems(self.handle, self._arr), "bmpc_set_problems")

    def transfer_bytes(self):
        """(host-to-device bytes per set_problems cold, with warm starts, device-to-host bytes per
        get_solutions with arrays)."""
        h, w, d = C.c_size_t(), C.c_size_t(), C.c_size_t()
        _check(lib().bmpc_transfer_bytes(self.handle, C.byref(h), C.byref(w), C.byref(d)), "bmpc_transfer_bytes")
        return h.value, w.value, d.value

    def flat_inputs(self, pinned: bool = True):
        """The batch's per-node inputs as node-major float32 tensors concatenated in problem order:
        (xref [sum n*nx], weight [sum n], obs [sum n*n_obs*5]) in pinned host memory, for
        set_problems_flat.  A control loop keeps them and overwrites them in place."""
        torch = self.torch
        cat = lambda key: np.concatenate([np.asarray(p[key], np.float32).reshape(-1) for p in self.problems])
        arrs = (cat("xref"), cat("weight"), cat("obs"))
        out = []
        for a in arrs:
            t = torch.from_numpy(np.ascontiguousarray(a))
            out.append(t.pin_memory() if pinned else t)
        return tuple(out)

    def flat_outputs(self, pinned: bool = True):
        """Reusable node-major float32 tensors (x, u, lam, y) for get_solutions_flat."""
        torch = self.torch
        sizes = (int(np.sum(self.nodes * self.nx)), int(np.sum(self.nodes * NU)), int(np.sum(self.nodes * self.nx)),
                 int(np.sum(self.nodes * self.nc)))
        return tuple((torch.empty(max(s, 1), dtype=torch.float32).pin_memory() if pinned
                      else torch.empty(max(s, 1), dtype=torch.float32)) for s in sizes)

    def set_problems_flat(self, xref, weight, obs):
        """Upload from flat node-major tensors (see flat_inputs); per-problem scalars come from the
        problem dicts.  Warm-start slots are cleared."""
        if getattr(self, "_arr", None) is None:
            arr = (Problem * self.n)()
            self._pd = [_ProblemData(p) for p in self.problems]
            for k, pd in enumerate(self._pd):
                arr[k] = pd.s
            self._arr = arr
        ptr = lambda t: None if t is None else C.c_void_p(t.data_ptr())
        with self.torch.cuda.device(self.device):
            _check(lib().bmpc_set_problems_flat(self.handle, self._arr, ptr(xref), ptr(weight), ptr(obs)),
                   "bmpc_set_problems_flat")

    def get_solutions_flat(self, out=None):
        """Synchronise and return node-major arrays x, u, lam, y of all problems concatenated in
        problem order (into `out`, a tuple from flat_outputs, when given) and the statistics as a
        ctypes array."""
        torch = self.torch
        if out is None:
            out = self.flat_outputs(pinned=False)
        st = (Stats * self.n)()
        with torch.cuda.device(self.device):
            _check(lib().bmpc_get_solutions_flat(self.handle, *(C.c_void_p(t.data_ptr()) for t in out), st),
                   "bmpc_get_solutions_flat")
        return (*out, st)

    def get_solutions_flat_async(self, out):
        """Enqueue the packing and the copies of the solutions into `out` (a tuple from
        flat_outputs, pinned) and of the statistics, without waiting; see wait_solutions."""
        with self.torch.cuda.device(self.device):
            _check(lib().bmpc_get_solutions_flat_async(self.handle, *(C.c_void_p(t.data_ptr()) for t in out)),
                   "bmpc_get_solutions_flat_async")

    def wait_solutions(self, want_stats: bool = True):
        """Wait for the batch's stream; the statistics of the last asynchronous read (ctypes array)."""
        st = (Stats * self.n)() if want_stats else None
        with self.torch.cuda.device(self.device):
            _check(lib().bmpc_wait_solutions(self.handle, st), "bmpc_wait_solutions")
        return st

    def transfer_bytes_flat(self):
        """(host-to-device bytes per set_problems_flat, device-to-host bytes per get_solutions_flat)."""
        h, d = C.c_size_t(), C.c_size_t()
        _check(lib().bmpc_transfer_bytes_flat(self.handle, C.byref(h), C.byref(d)), "bmpc_transfer_bytes_flat")
        return h.value, d.value

    def set_stream(self, stream):
        """Issue the batch's later work on `stream` (a torch.cuda.Stream), ordered after the old one."""
        with self.torch.cuda.device(self.device):
            _check(lib().bmpc_set_stream(self.handle, C.c_void_p(stream.cuda_stream)), "bmpc_set_stream")
        self.stream = stream

    def solve(self, opts: Opts | None = None, graph: bool = False):
        """Launch the persistent solver (asynchronous on the batch's stream)."""
        o = opts if opts is not None else default_opts()
        fn = lib().bmpc_solve_batch_graph if graph else lib().bmpc_solve_batch
        with self.torch.cuda.device(self.device):
            _check(fn(self.handle, C.byref(o)), "bmpc_solve_batch")

    def start_stride(self) -> int:
        """Floats per problem of a packed device start (x | u | lam | y, node-major), over the batch."""
        return int(max(int(n) * (2 * int(nx) + NU + int(nc)) for n, nx, nc in zip(self.nodes, self.nx, self.nc)))

    def set_warm_device(self, starts, slot: int = 0):
        """Warm-start slot from a float32 CUDA tensor [n_problems, stride] of packed starts."""
        t = starts
        assert t.is_cuda and t.dtype == self.torch.float32 and t.is_contiguous() and t.shape[0] == self.n
        with self.torch.cuda.device(self.device):
            _check(lib().bmpc_set_warm_start_device(self.handle, t.data_ptr(), int(t.shape[1]), slot),
                   "bmpc_set_warm_start_device")

    def shift_from(self, prev: "Batch", slot: int = 0):
        """Warm-start slot from the receding-horizon shift of prev's solution (same trees)."""
        with self.torch.cuda.device(self.device):
            _check(lib().bmpc_shift_warm_start(self.handle, prev.handle, slot), "bmpc_shift_warm_start")

    def autotune(self, base: Opts | None = None) -> tuple[Opts, float]:
        """Pick threads per problem, sweep variant and line-search chunk by timing them on this batch."""
        o = base if base is not None else default_opts()
        best, us = Opts(), C.c_float()
        with self.torch.cuda.device(self.device):
            _check(lib().bmpc_autotune(self.handle, C.byref(o), C.byref(best), C.byref(us)), "bmpc_autotune")
        return best, us.value

    def device_order(self):
        """The queue order of the last solve (problem ids, grouped by model)."""
        out = np.zeros(self.n, np.int32)
        with self.torch.cuda.device(self.device):
            _check(lib().bmpc_get_queue_order(self.handle, out.ctypes.data_as(C.POINTER(C.c_int32))),
                   "bmpc_get_queue_order")
        return out

    def get_solutions(self, want_arrays: bool = True):
        """Synchronise and return per-problem dicts with x, u, lam, y and the solver statistics."""
        tot_x = int(np.sum(self.nodes * self.nx))
        tot_u = int(np.sum(self.nodes * NU))
        tot_y = int(np.sum(self.nodes * self.nc))
        x = np.zeros(max(tot_x, 1), np.float32)
        u = np.zeros(max(tot_u, 1), np.float32)
        lam = np.zeros(max(tot_x, 1), np.float32)
        y = np.zeros(max(tot_y, 1), np.float32)
        st = (Stats * self.n)()
        args = [a.ctypes.data_as(_fp) if want_arrays else None for a in (x, u, lam, y)]
        with self.torch.cuda.device(self.device):
            _check(lib().bmpc_get_solutions(self.handle, *args, st), "bmpc_get_solutions")
        out = []
        ox = ou = oy = 0
        for k in range(self.n):
            n_, nx, nc = int(self.nodes[k]), int(self.nx[k]), int(self.nc[k])
            s = st[k]
            rec = dict(status=s.status, inner_iters=s.inner_iters, outer_iters=s.outer_iters,
                       ls_fail_total=s.ls_fail_total, ls_evals=s.ls_evals, start_used=s.start_used, r_kkt=s.r_kkt, c=s.c, rho=s.rho, mu=s.mu,
                       cycles=dict(linearise=s.cycles_linearise, backward=s.cycles_backward,
                                   forward=s.cycles_forward, linesearch=s.cycles_linesearch,
                                   total=s.cycles_total))
            if want_arrays:
                rec["x"] = x[ox:ox + n_ * nx].reshape(n_, nx).astype(np.float64)
                rec["lam"] = lam[ox:ox + n_ * nx].reshape(n_, nx).astype(np.float64)
                rec["u"] = u[ou:ou + n_ * NU].reshape(n_, NU).astype(np.float64)
                rec["y"] = y[oy:oy + n_ * nc].reshape(n_, nc).astype(np.float64)
            ox += n_ * nx
            ou += n_ * NU
            oy += n_ * nc
            out.append(rec)
        return out

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            lib().bmpc_destroy_batch(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def solve(problems, opts: Opts | None = None, warm=None, graph: bool = False):
    """Create a batch, upload, solve and return the per-problem results."""
    b = Batch(problems)
    b.set_problems(warm=warm)
    b.solve(opts, graph=graph)
    res = b.get_solutions()
    b.close()
    return res


class StaticScratchBatch(Batch):
    """A batch whose solver scratch is the library's fixed 16 MiB device array.

    For callers that cannot allocate device memory for the solver (real-time loops, plug-ins
    whose framework owns the device buffers): only the data arena (inputs and outputs) is
    supplied here; bmpc_create_batch_static allocates nothing.  All such batches share the one
    array, so their solves must not overlap on the GPU.
    """

    def __init__(self, problems, device=None, stream=None, pinned: bool = True):
        import torch

        if not torch.cuda.is_available():
            raise RuntimeError("bmpc needs a CUDA device (no CPU fallback)")
        self.torch = torch
        self.problems = list(problems)
        self.n = len(self.problems)
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        descs = (TreeDesc * self.n)()
        self._parents = []
        for k, p in enumerate(self.problems):
            d, par = tree_desc(p)
            descs[k] = d
            self._parents.append(par)
        self._descs = descs
        db, sb, hb = C.c_size_t(), C.c_size_t(), C.c_size_t()
        _check(lib().bmpc_batch_bytes(descs, self.n, C.byref(db), C.byref(sb), C.byref(hb)), "bmpc_batch_bytes")
        self.data_bytes, self.scratch_bytes, self.staging_bytes = db.value, sb.value, hb.value
        with torch.cuda.device(self.device):
            self._data = torch.empty(self.data_bytes + 256, dtype=torch.uint8, device=self.device)
        self._stage = torch.empty(self.staging_bytes, dtype=torch.uint8, pin_memory=pinned)
        dptr = (self._data.data_ptr() + 255) // 256 * 256
        h = C.c_void_p()
        with torch.cuda.device(self.device):
            _check(lib().bmpc_create_batch_static(descs, self.n, dptr, self.data_bytes, self._stage.data_ptr(),
                                                  self.staging_bytes, C.c_void_p(self.stream.cuda_stream),
                                                  C.byref(h)), "bmpc_create_batch_static")
        self.handle = h
        self.nodes = np.array([int(p["n"]) for p in self.problems])
        self.nx = np.array([int(p["nx"]) for p in self.problems])
        self.nc = np.array([n_con(p) for p in self.problems])
