"""Learned warm start for branch MPC: data from the solver's own solutions, training of the
network, and the receding-horizon comparison of cold, shifted and learned starts.

Features (per problem): the measured state without its X coordinate and, for every scenario
and obstacle, the predicted obstacle position at the middle and the end of the scenario and
its final heading, positions relative to the ego's X.  Targets: the converged solution
(states with X relative to the ego, controls, dynamics multipliers, AL multipliers, the latter
as sqrt(y) by default), both standardised with statistics of the training set.  At run time the
network's start goes into warm-start slot 0 and the shifted previous solution (or nothing: the cold start) into slot 1; the
solver starts from the network's start only when its merit, with a large constraint penalty, is
not above the fallback's (bmpc_opts.warm_select, select_rho).

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
    """Targets per problem, padded to a multiple of 256: the output layer's GEMMs then run on the
    128 x 256 output tiles."""
    return (int(p["n"]) * (2 * int(p["nx"]) + 2 + bmpc.n_con(p)) + 255) // 256 * 256


def solve_batch(problems, opts=None, prev=None, warm_from=None):
    b = bmpc.Batch(problems)
    b.set_problems()
    if prev is not None:
        b.shift_from(prev, slot=0)
    b.solve(opts if opts is not None else bmpc.default_opts())
    return b


def build_dataset(make, total, chunk, opts=None, device="cuda", log=print, y_sqrt=1, y_alt=False):
    """Solve `total` problems from make(chunk_index, count) in chunks; keep the converged ones.

    Returns (X_raw, Y_raw) fp32 CUDA tensors [kept, feature_dim], [kept, target_dim] and timing;
    with y_alt the targets with the other multiplier form are in info["Y_alt"]."""
    import torch
    X, Y, Y2 = [], [], []
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
        mlp.targets(b, fy, y_sqrt)
        if y_alt:
            fy2 = torch.empty_like(fy)
            mlp.targets(b, fy2, 1 - y_sqrt)
            Y2.append(fy2[ok])
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
    info = dict(generate_s=t_gen, solve_s=t_solve, kept=kept, total=total)
    if y_alt:
        info["Y_alt"] = torch.cat(Y2)
    return X, Y, info


def standardise(X_raw, Y_raw, y_sqrt=1):
    """Statistics of the training set and bf16 standardised copies (kernels do the conversion).
    y_sqrt records the multiplier form of the targets, which the starts invert."""
    import torch
    fm, fs = X_raw.mean(0), X_raw.std(0).clamp_min(1e-3)
    tm, ts = Y_raw.mean(0), Y_raw.std(0).clamp_min(1e-4)
    Xb = torch.empty(X_raw.shape, dtype=torch.bfloat16, device=X_raw.device)
    Yb = torch.empty(Y_raw.shape, dtype=torch.bfloat16, device=Y_raw.device)
    mlp.standardize(X_raw, fm, fs, Xb)
    mlp.standardize(Y_raw, tm, ts, Yb)
    return Xb, Yb, dict(fm=fm, fs=fs, tm=tm, ts=ts, y_sqrt=y_sqrt)


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
            tot += net.train_step(x, y, lr_k, weight_decay)[0]
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
    mlp.starts(b, pred, stats["tm"], stats["ts"], st, stats.get("y_sqrt", 1))
    b.set_warm_device(st, slot=0)
    return st


def start_errors(problems, starts, sols):
    """Accuracy of packed starts against converged solutions (converged problems only): per block
    (x, u, lam, y) the relative error sqrt(sum |start - sol|^2 / sum |sol|^2), and for y the
    fraction of constraint rows whose activity (y > 1e-6) the start gets right."""
    acc = {k: [0.0, 0.0] for k in ("x", "u", "lam", "y")}
    agree = total = 0
    for p, s, r in zip(problems, starts, sols):
        if r["status"] != 0:
            continue
        n, nx = int(p["n"]), int(p["nx"])
        nc = bmpc.n_con(p)
        o = [0, n * nx, n * nx + 2 * n, 2 * n * nx + 2 * n, 2 * n * nx + 2 * n + n * nc]
        for j, k in enumerate(("x", "u", "lam", "y")):
            a, ref = np.asarray(s[o[j]:o[j + 1]], np.float64), np.asarray(r[k], np.float64).ravel()
            acc[k][0] += float(np.sum((a - ref) ** 2))
            acc[k][1] += float(np.sum(ref ** 2))
        ys, yr = np.asarray(s[o[3]:o[4]]) > 1e-6, np.asarray(r["y"]).ravel() > 1e-6
        agree += int(np.sum(ys == yr))
        total += ys.size
    out = {f"rel_{k}": math.sqrt(v[0] / max(v[1], 1e-30)) for k, v in acc.items()}
    out["y_activity_agreement"] = agree / max(total, 1)
    return out


def timed_solve(b, opts):
    import torch
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(b.stream)
    b.solve(opts)
    e1.record(b.stream)
    res = b.get_solutions(want_arrays=False)
    return res, e0.elapsed_time(e1)


def summarise(res, ms):
    it = np.array([r["inner_iters"] for r in res])
    conv = np.array([r["status"] == 0 for r in res])
    return dict(mean_iters=float(it.mean()), median_iters=float(np.median(it)), converged=float(conv.mean()),
                ms_total=ms, us_per_solve=1e3 * ms / len(res),
                used_primary=float(np.mean([r["start_used"] == 1 for r in res])))


def evaluate(net, stats, make_prev, count, opts=None, seed=0):
    """Two comparisons on held-out scenes.

    First solve (no previous solution): cold start against the learned start alone and against the
    learned start with the cold start as fallback.  Receding horizon: solve the scenes, advance
    each one step, then solve the next problems from the cold start, the shifted previous solution,
    and the learned start with the shifted start as fallback.  Learned times include the network
    (features, forward pass, starts)."""
    import torch

    import scenes
    opts = opts if opts is not None else bmpc.default_opts()
    sel = bmpc.Opts.from_buffer_copy(opts)
    sel.warm_select = 1
    prev_ps = make_prev(count)
    prev = bmpc.Batch(prev_ps)
    first = {}

    def learned(b, fallback):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(b.stream)
        learned_starts(net, b, stats)
        if fallback is not None:
            b.shift_from(fallback, slot=1)
        e1.record(b.stream)
        res, ms = timed_solve(b, sel)
        torch.cuda.synchronize()
        return res, ms + e0.elapsed_time(e1)

    prev.set_problems()
    timed_solve(prev, opts)                       # warm-up of the launch path
    prev.set_problems()
    first["cold"] = timed_solve(prev, opts)
    cold_sols = prev.get_solutions()
    prev.set_problems()
    o1 = bmpc.Opts.from_buffer_copy(opts)
    st = learned_starts(net, prev, stats).cpu().numpy()
    accuracy = start_errors(prev_ps, st, cold_sols)
    first["learned"] = timed_solve(prev, o1)
    prev.set_problems()
    first["learned_or_cold"] = learned(prev, None)
    prev.set_problems()
    timed_solve(prev, opts)                       # the previous solutions the next problems shift
    pres = prev.get_solutions()
    next_ps = [scenes.advance(p, r["x"][1], seed=seed * 100000 + k) for k, (p, r) in enumerate(zip(prev_ps, pres))]
    nxt = {}
    b = bmpc.Batch(next_ps)
    b.set_problems()
    nxt["cold"] = timed_solve(b, opts)
    b.set_problems()
    b.shift_from(prev, slot=0)
    nxt["shifted"] = timed_solve(b, opts)
    b.set_problems()
    nxt["learned_or_shifted"] = learned(b, prev)
    prev.close()
    b.close()
    return dict(first_solve={k: summarise(*v) for k, v in first.items()},
                receding_horizon={k: summarise(*v) for k, v in nxt.items()}, start_accuracy=accuracy)


# ------------------------------------------------------------------ command line: the config-5 experiment
def _gen_chunk(args):
    import scenes
    seed, count = args
    ps = scenes.batch_problems(seed, count)
    for p in ps:
        p["obs"] = p["obs"].astype(np.float32)
    return ps


def main(argv=None):
    import argparse
    import json
    import multiprocessing as mp

    ap = argparse.ArgumentParser(description="train and evaluate the learned warm start (config-3 scenes)")
    ap.add_argument("--train", type=int, default=200000)
    ap.add_argument("--chunk", type=int, default=4096)
    ap.add_argument("--epochs", type=int, default=10)
    ap.add_argument("--batch", type=int, default=512)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--hidden", type=int, default=512)
    ap.add_argument("--eval", type=int, default=2000)
    ap.add_argument("--train-seed", type=int, default=5)
    ap.add_argument("--eval-seed", type=int, default=6)
    ap.add_argument("--workers", type=int, default=12)
    ap.add_argument("--out", default="")
    ap.add_argument("--y-form", choices=("sqrt", "linear", "both"), default="sqrt",
                    help="form of the AL-multiplier targets; 'both' trains one network on each")
    a = ap.parse_args(argv)
    pool = mp.get_context("spawn").Pool(a.workers)          # started before the first CUDA call
    import torch
    import scenes

    def make(c, cnt):
        per = (cnt + a.workers - 1) // a.workers
        jobs = [(a.train_seed * 1000003 + c * 64 + w, min(per, cnt - w * per)) for w in range(a.workers)
                if cnt - w * per > 0]
        out = []
        for part in pool.map(_gen_chunk, jobs):
            out += part
        return out

    opts = bmpc.default_opts()
    probe = bmpc.Batch(make(0, 512))
    probe.set_problems()
    opts, _ = probe.autotune(opts)
    probe.close()
    t0 = time.perf_counter()
    y_sqrt = 0 if a.y_form == "linear" else 1
    X, Y, info = build_dataset(make, a.train, a.chunk, opts, y_sqrt=y_sqrt, y_alt=a.y_form == "both")
    info["dataset_s"] = time.perf_counter() - t0
    forms = [(y_sqrt, Y)] + ([(1 - y_sqrt, info.pop("Y_alt"))] if a.y_form == "both" else [])
    del Y
    eval_make = lambda cnt: scenes.batch_problems(a.eval_seed * 1000003, cnt)
    res = dict(dataset=info, opts=dict(block_threads=opts.block_threads, variant=opts.variant,
                                       ls_chunk=opts.ls_chunk), runs={})
    while forms:
        ys, Yf = forms.pop(0)
        Xb, Yb, stats = standardise(X, Yf, y_sqrt=ys)
        del Yf
        torch.cuda.empty_cache()
        dims = [Xb.shape[1], a.hidden, a.hidden, a.hidden, Yb.shape[1]]
        net = mlp.MLP(dims, seed=1)
        hist, t_train = train(net, Xb, Yb, a.epochs, a.batch, a.lr)
        flops = 6.0 * a.batch * sum(x * y for x, y in zip(dims[:-1], dims[1:])) * a.epochs * (Xb.shape[0] // a.batch)
        del Xb, Yb
        torch.cuda.empty_cache()
        res["runs"]["sqrt" if ys else "linear"] = dict(
            dims=dims, train_loss=hist, train_s=t_train, train_tflops=flops / t_train / 1e12,
            eval=evaluate(net, stats, eval_make, a.eval, opts))
        del net
    pool.close()
    print(json.dumps(res))
    if a.out:
        with open(a.out, "w") as f:
            json.dump(res, f, indent=1)
    return res


if __name__ == "__main__":
    main()
