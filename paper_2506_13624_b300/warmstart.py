"""Learned warm start for branch MPC: data from the solver's own solutions, training of the
network, and the receding-horizon comparison of cold, shifted and learned starts.

Features (per problem): the measured state without its X coordinate and, for every scenario
and obstacle, the predicted obstacle position at the middle and the end of the scenario and
its final heading, positions relative to the ego's X.  Targets: the converged solution
(states with X relative to the ego, controls, dynamics multipliers, AL multipliers), both
standardised with statistics of the training set.  At run time the network's start goes into
warm-start slot 0 and the shifted previous solution into slot 1; the solver starts from the
network's start only when its merit is not above the shifted start's (bmpc_opts.warm_select).

Bookkeeping of the data set (concatenation, statistics, shuffling) uses torch tensor ops;
features, targets, standardisation, the network and the starts run in libbmpc.so.
"""
from __future__ import annotations

import math
import time

import numpy as np

from . import bmpc, mlp

N_SCEN, N_OBS = 64, 5


def round128(v: int) -> int:
    return (v + 127) // 128 * 128


def feature_dim(p) -> int:
    return round128(int(p["nx"]) - 1 + 5 * N_SCEN * N_OBS)


def target_dim(p) -> int:
    return round128(int(p["n"]) * (2 * int(p["nx"]) + 2 + bmpc.n_con(p)))


def solve_batch(problems, opts=None, prev=None, warm_from=None):
    b = bmpc.Batch(problems)
    b.set_problems()
    if prev is not None:
        b.shift_from(prev, slot=0)
    b.solve(opts if opts is not None else bmpc.default_opts())
    return b


def build_dataset(make, total, chunk, opts=None, device="cuda", log=print):
    """Solve `total` problems from make(chunk_index, count) in chunks; keep the converged ones.

    Returns (X_raw, Y_raw) fp32 CUDA tensors [kept, feature_dim], [kept, target_dim] and timing."""
    import torch
    X, Y = [], []
    t_gen = t_solve = 0.0
    kept = 0
    done = 0
    c = 0
    while done < total:
        cnt = min(chunk, total - done)
        t0 = time.perf_counter()
        ps = make(c, cnt)
        t_gen += time.perf_counter() - t0
        t0 = time.perf_counter()
        b = solve_batch(ps, opts)
        res = b.get_solutions(want_arrays=False)
        ok = torch.tensor([r["status"] == 0 for r in res], device=device)
        fx = torch.empty((cnt, feature_dim(ps[0])), dtype=torch.float32, device=device)
        fy = torch.empty((cnt, target_dim(ps[0])), dtype=torch.float32, device=device)
        mlp.features(b, fx, N_SCEN, N_OBS)
        mlp.targets(b, fy)
        torch.cuda.synchronize()
        X.append(fx[ok])
        Y.append(fy[ok])
        kept += int(ok.sum())
        b.close()
        t_solve += time.perf_counter() - t0
        done += cnt
        c += 1
        if log and c % 10 == 0:
            log(f"  dataset {done}/{total} solved, {kept} converged")
    X = torch.cat(X)
    Y = torch.cat(Y)
    return X, Y, dict(generate_s=t_gen, solve_s=t_solve, kept=kept, total=total)


def standardise(X_raw, Y_raw):
    """Statistics of the training set and bf16 standardised copies (kernels do the conversion)."""
    import torch
    fm, fs = X_raw.mean(0), X_raw.std(0).clamp_min(1e-3)
    tm, ts = Y_raw.mean(0), Y_raw.std(0).clamp_min(1e-4)
    Xb = torch.empty(X_raw.shape, dtype=torch.bfloat16, device=X_raw.device)
    Yb = torch.empty(Y_raw.shape, dtype=torch.bfloat16, device=Y_raw.device)
    mlp.standardize(X_raw, fm, fs, Xb)
    mlp.standardize(Y_raw, tm, ts, Yb)
    return Xb, Yb, dict(fm=fm, fs=fs, tm=tm, ts=ts)


def train(net, Xb, Yb, epochs, batch=512, lr=1e-3, weight_decay=1e-4, seed=0, log=print):
    """AdamW on shuffled minibatches with a cosine learning-rate decay; returns per-epoch loss."""
    import torch
    g = torch.Generator(device=Xb.device)
    g.manual_seed(seed)
    n = Xb.shape[0] // batch * batch
    steps = epochs * (n // batch)
    hist = []
    k = 0
    t0 = time.perf_counter()
    for ep in range(epochs):
        perm = torch.randperm(Xb.shape[0], device=Xb.device, generator=g)[:n]
        tot = torch.zeros((), device=Xb.device)
        for s in range(n // batch):
            idx = perm[s * batch:(s + 1) * batch]
            x = Xb.index_select(0, idx)
            y = Yb.index_select(0, idx)
            lr_k = lr * 0.5 * (1.0 + math.cos(math.pi * k / max(1, steps)))
            tot += net.train_step(x, y, lr_k, weight_decay)
            k += 1
        hist.append(float(tot) / (n // batch))
        if log:
            log(f"  epoch {ep + 1}/{epochs}: loss {hist[-1]:.4f}")
    torch.cuda.synchronize()
    return hist, time.perf_counter() - t0


def learned_starts(net, b, stats, batch_pad=128):
    """Features -> standardised bf16 -> network -> packed starts in warm slot 0 of batch b."""
    import torch
    n = b.n
    rows = (n + batch_pad - 1) // batch_pad * batch_pad
    fx = torch.zeros((rows, net.dims[0]), dtype=torch.float32, device=b.device)
    mlp.features(b, fx, N_SCEN, N_OBS)
    xb = torch.empty((rows, net.dims[0]), dtype=torch.bfloat16, device=b.device)
    mlp.standardize(fx, stats["fm"], stats["fs"], xb)
    pred = net.forward(xb)
    st = torch.empty((n, b.start_stride()), dtype=torch.float32, device=b.device)
    mlp.starts(b, pred, stats["tm"], stats["ts"], st)
    b.set_warm_device(st, slot=0)


def timed_solve(b, opts):
    import torch
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(b.stream)
    b.solve(opts)
    e1.record(b.stream)
    res = b.get_solutions(want_arrays=False)
    return res, e0.elapsed_time(e1)


def evaluate(net, stats, make_prev, count, opts=None, seed=0):
    """Receding-horizon comparison on held-out scenes: solve the previous problems, advance each
    scene one step, then solve the next problems from the cold start, the shifted previous
    solution, and the learned start (shifted start as fallback by merit)."""
    import torch

    import scenes
    opts = opts if opts is not None else bmpc.default_opts()
    prev_ps = make_prev(count)
    prev = solve_batch(prev_ps, opts)
    pres = prev.get_solutions()
    next_ps = [scenes.advance(p, r["x"][1], seed=seed * 100000 + k) for k, (p, r) in enumerate(zip(prev_ps, pres))]
    out = {}
    b = bmpc.Batch(next_ps)
    # cold
    b.set_problems()
    b.solve(opts)
    b.get_solutions(want_arrays=False)
    b.set_problems()
    out["cold"] = timed_solve(b, opts)
    # shifted
    b.set_problems()
    b.shift_from(prev, slot=0)
    out["shifted"] = timed_solve(b, opts)
    # learned, shifted as fallback
    sel = bmpc.Opts.from_buffer_copy(opts)
    sel.warm_select = 1
    b.set_problems()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(b.stream)
    learned_starts(net, b, stats)
    b.shift_from(prev, slot=1)
    e1.record(b.stream)
    res, ms = timed_solve(b, sel)
    torch.cuda.synchronize()
    out["learned"] = (res, ms + e0.elapsed_time(e1))
    prev.close()
    b.close()
    summary = {}
    for k, (res, ms) in out.items():
        it = np.array([r["inner_iters"] for r in res])
        conv = np.array([r["status"] == 0 for r in res])
        summary[k] = dict(mean_iters=float(it.mean()), median_iters=float(np.median(it)),
                          converged=float(conv.mean()), ms_total=ms, us_per_solve=1e3 * ms / len(res),
                          used_primary=float(np.mean([r["start_used"] == 1 for r in res])))
    return summary
