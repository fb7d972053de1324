"""Learned warm start: training data from the solver, training, and the
warm-start measurement, all through the C ABI (bfcs_solve_batched,
bfcs_net_prepare, bfcs_net_train_step, bfcs_net_predict).  This module only
marshals arguments and runs loops; every arithmetic step runs in libbfcs.so.

Workload (random sphere microstructures of volume fraction 0.1-0.3 in 16^3
cells, contrast 10, BFCS radius a in [4, 12] voxels at a random voxel corner)
is generated by workloads.config_c5_sample(seed, n).

Command line:
  python -m paper_2601_00822_gb300.surrogate train --samples 4096 --steps 6000 --out W.bin
  python -m paper_2601_00822_gb300.surrogate bench --weights W.bin --batch 64
"""
from __future__ import annotations

import argparse
import json
import math
import os
import time

import numpy as np
import torch

from . import api, workloads as W

PKG = os.path.dirname(os.path.abspath(__file__))
DEFAULT_WEIGHTS = os.path.join(PKG, "weights", "unet_c5_64.bin")
TRAIN_SEED0 = 1_000_000      # training samples use seeds TRAIN_SEED0 + i; evaluation seeds are below


def material():
    p = W.config_c5_sample(0)
    return [tuple(q) for q in p.phases], tuple(p.c0)


def sample_inputs(seed, n, precision="fp64"):
    """(phase, b) of config_c5_sample(seed, n) on the device."""
    p = W.config_c5_sample(seed, n)
    ph = api.voxelize(p.dims, p.cell, p.spheres)
    b = api.body_force(p.dims, p.bf_centre, p.bf_radius, precision)
    return ph, b


def generate(seeds, n, solve_batch=64, tol=1e-4, maxit=5000, log=print):
    """Solver-generated training pairs: X (S, 4, n, n, n) and T (S, 6, n, n, n),
    float32 on the device (FP32 batched solves to tol)."""
    phases, c0 = material()
    dims = (n, n, n)
    S = len(seeds)
    X = torch.empty((S, 4, n, n, n), dtype=torch.float32, device="cuda")
    T = torch.empty((S, 6, n, n, n), dtype=torch.float32, device="cuda")
    net = api.Net(dims, max_batch=1)
    t0 = time.time()
    iters = []
    with api.Plan(dims, "fp32", max_batch=solve_batch) as plan:
        for i0 in range(0, S, solve_batch):
            chunk = seeds[i0:i0 + solve_batch]
            members = []
            for s in chunk:
                ph, b = sample_inputs(s, n, "fp32")
                members.append(dict(phase=ph, b=b, sig_out=None, u_out=None))
            members, infos = plan.solve_batched(members, phases, c0, tol=tol, maxit=maxit)
            iters += [i.iters for i in infos]
            for k, mem in enumerate(members):
                net.prepare(mem["b"], mem["phase"], phases, eps=mem["eps_out"], x_out=X[i0 + k],
                            target_out=T[i0 + k])
    torch.cuda.synchronize()
    log(f"generated {S} samples at {n}^3 in {time.time() - t0:.1f} s (mean sweeps {np.mean(iters):.1f})")
    return X, T


def init_params(seed=0):
    """He-uniform weights, zero biases (the network oracle's initialisation, here
    with numpy so that this module does not depend on the oracle)."""
    rng = np.random.default_rng(seed)
    parts = []
    for kind, cin, cout in LAYERS:
        k = 27 if kind == "conv3" else 1 if kind == "conv1" else 8
        fan_in = cin * (27 if kind == "conv3" else 1)
        bound = math.sqrt(6.0 / fan_in) * (0.5 if kind == "conv1" else 1.0)
        parts.append(rng.uniform(-bound, bound, size=k * cin * cout))
        parts.append(np.zeros(cout))
    flat = np.concatenate(parts).astype(np.float32)
    assert flat.size == api.Net.param_count()
    return torch.from_numpy(flat).cuda()


LAYERS = (("conv3", 4, 32), ("conv3", 32, 32), ("conv3", 32, 32), ("conv3", 32, 32), ("conv3", 32, 32),
          ("conv3", 32, 32), ("conv3", 32, 48), ("conv3", 48, 48), ("up", 48, 32), ("conv3", 64, 32),
          ("conv3", 32, 32), ("up", 32, 32), ("conv3", 64, 32), ("conv3", 32, 32), ("up", 32, 32),
          ("conv3", 64, 32), ("conv3", 32, 32), ("conv1", 32, 6))


def train(X, T, steps, batch=8, lr=1e-3, seed=0, params=None, log=print, log_every=200, warmup=300):
    """Adam with a linear warm-up and a cosine learning-rate decay over
    contiguous minibatches of a shuffled-once sample order; returns (params, losses)."""
    S = X.shape[0]
    dims = tuple(X.shape[2:][::-1])
    net = api.Net(dims, max_batch=batch, train=True)
    params = params if params is not None else init_params(seed)
    grad = torch.zeros_like(params)
    m = torch.zeros_like(params)
    v = torch.zeros_like(params)
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    losses = []
    nb = S // batch
    t0 = time.time()
    for t in range(1, steps + 1):
        i = ((t - 1) % nb) * batch
        lr_t = lr * min(1.0, t / max(warmup, 1)) * 0.5 * (1 + math.cos(math.pi * (t - 1) / steps))
        net.train_step(params, grad, m, v, t, lr_t, X[i:i + batch], T[i:i + batch], loss=loss)
        if t % log_every == 0 or t == steps:
            losses.append((t, float(loss.item())))
            log(f"step {t} loss {losses[-1][1]:.4f} ({time.time() - t0:.0f} s)")
    torch.cuda.synchronize()
    return params, losses


def validation_loss(params, X, T, batch=8):
    dims = tuple(X.shape[2:][::-1])
    net = api.Net(dims, max_batch=batch, train=True)
    tot, cnt = 0.0, 0
    for i in range(0, X.shape[0] - batch + 1, batch):
        _, loss = net.grad(params, X[i:i + batch], T[i:i + batch])
        tot += float(loss.item()) * batch
        cnt += batch
    return tot / max(cnt, 1)


def save(params, path):
    os.makedirs(os.path.dirname(path), exist_ok=True)
    params.detach().cpu().numpy().astype("<f4").tofile(path)


def load(path):
    a = np.fromfile(path, dtype="<f4")
    if a.size != api.Net.param_count():
        raise ValueError(f"{path}: {a.size} values, expected {api.Net.param_count()}")
    return torch.from_numpy(a).cuda()


def warm_start_benchmark(params, seeds, n, tol=1e-6, maxit=20000, batch=64, plain=True, repeats=1):
    """Solves/s to residual tol of the same problems (mixed-precision ladder):
    plain (one cold solve at a time), batched cold, batched with the network's
    warm start (inference included in the timing).  The warm results are
    compared with the cold solver's: relative L2 of eps."""
    phases, c0 = material()
    dims = (n, n, n)
    inputs = [sample_inputs(s, n, "fp64") for s in seeds]
    B = len(seeds)
    out = {"grid": n, "solves": B, "tol": tol}
    with api.Plan(dims, "mixed", max_batch=min(batch, 64)) as pb, api.Plan(dims, "mixed") as p1:
        net = api.Net(dims, max_batch=min(B, 16))

        def cold_batched():
            mem = [dict(phase=ph, b=b, sig_out=None, u_out=None) for ph, b in inputs]
            return pb.solve_batched(mem, phases, c0, tol=tol, maxit=maxit)

        def warm_batched():
            init = net.predict(params, [b for _, b in inputs], [ph for ph, _ in inputs], phases)
            mem = [dict(phase=ph, b=b, eps_init=e, sig_out=None, u_out=None) for (ph, b), e in zip(inputs, init)]
            return pb.solve_batched(mem, phases, c0, tol=tol, maxit=maxit)

        def plain_cold():
            res = []
            for ph, b in inputs:
                eps, _, _, info = p1.solve(ph, phases, c0, b, tol=tol, maxit=maxit, want_sig=False, want_u=False)
                res.append((eps, info))
            return res

        def timed(fn):
            fn()       # warm-up (graph instantiation, allocations)
            torch.cuda.synchronize()
            best = float("inf")
            res = None
            for _ in range(repeats):
                t0 = time.perf_counter()
                res = fn()
                torch.cuda.synchronize()
                best = min(best, time.perf_counter() - t0)
            return best, res

        tc, (mc, ic) = timed(cold_batched)
        tw, (mw, iw) = timed(warm_batched)
        out["batched_cold"] = {"solves_per_s": B / tc, "mean_sweeps": float(np.mean([i.iters for i in ic])),
                               "max_resid": max(i.resid for i in ic)}
        out["batched_warm"] = {"solves_per_s": B / tw, "mean_sweeps": float(np.mean([i.iters for i in iw])),
                               "max_resid": max(i.resid for i in iw)}
        errs = [float(torch.linalg.vector_norm(a["eps_out"] - c["eps_out"]) / torch.linalg.vector_norm(c["eps_out"]))
                for a, c in zip(mw, mc)]
        out["warm_vs_cold_eps_rel_l2_max"] = max(errs)
        # quality of the prediction itself: relative L2 against the cold solution
        init = net.predict(params, [b for _, b in inputs], [ph for ph, _ in inputs], phases)
        out["prediction_rel_l2_mean"] = float(np.mean([
            float(torch.linalg.vector_norm(e - c["eps_out"]) / torch.linalg.vector_norm(c["eps_out"]))
            for e, c in zip(init, mc)]))
        if plain:
            tp, rp = timed(plain_cold)
            out["plain_cold"] = {"solves_per_s": B / tp, "mean_sweeps": float(np.mean([i.iters for _, i in rp]))}
            out["speedup_batched_warm_vs_plain"] = out["batched_warm"]["solves_per_s"] / out["plain_cold"]["solves_per_s"]
        out["speedup_warm_vs_cold_batched"] = out["batched_warm"]["solves_per_s"] / out["batched_cold"]["solves_per_s"]
    return out


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    sub = ap.add_subparsers(dest="cmd", required=True)
    t = sub.add_parser("train")
    t.add_argument("--samples", type=int, default=4096)
    t.add_argument("--val", type=int, default=64)
    t.add_argument("--grid", type=int, default=64)
    t.add_argument("--steps", type=int, default=6000)
    t.add_argument("--batch", type=int, default=8)
    t.add_argument("--lr", type=float, default=1e-3)
    t.add_argument("--out", default=DEFAULT_WEIGHTS)
    t.add_argument("--log", default=None)
    b = sub.add_parser("bench")
    b.add_argument("--weights", default=DEFAULT_WEIGHTS)
    b.add_argument("--grid", type=int, default=64)
    b.add_argument("--batch", type=int, default=64)
    b.add_argument("--tol", type=float, default=1e-6)
    st = sub.add_parser("step", help="time training steps and a forward pass on random data (profiling aid)")
    st.add_argument("--grid", type=int, default=64)
    st.add_argument("--batch", type=int, default=8)
    st.add_argument("--steps", type=int, default=4)
    a = ap.parse_args(argv)
    if a.cmd == "step":
        n, B = a.grid, a.batch
        gen = torch.Generator(device="cuda").manual_seed(0)
        X = torch.randn((B, 4, n, n, n), device="cuda", generator=gen)
        T = torch.randn((B, 6, n, n, n), device="cuda", generator=gen)
        net = api.Net((n, n, n), max_batch=B, train=True)
        params = init_params(0)
        grad, m, v = torch.zeros_like(params), torch.zeros_like(params), torch.zeros_like(params)
        for t in range(1, 4):
            net.train_step(params, grad, m, v, t, 1e-4, X, T)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        torch.cuda.synchronize()
        ev[0].record()
        for t in range(4, 4 + a.steps):
            net.train_step(params, grad, m, v, t, 1e-4, X, T)
        ev[1].record()
        net.forward(params, X)
        ev[2].record()
        torch.cuda.synchronize()
        print(json.dumps({"grid": n, "batch": B, "train_step_ms": ev[0].elapsed_time(ev[1]) / a.steps,
                          "forward_ms": ev[1].elapsed_time(ev[2])}))
        return
    if a.cmd == "train":
        logf = open(a.log, "w") if a.log else None

        def log(msg):
            print(msg, flush=True)
            if logf:
                logf.write(msg + "\n")
                logf.flush()
        rng = np.random.default_rng(12345)
        seeds = [TRAIN_SEED0 + int(i) for i in rng.permutation(a.samples)]
        X, T = generate(seeds, a.grid, log=log)
        Xv, Tv = generate(list(range(TRAIN_SEED0 - a.val, TRAIN_SEED0)), a.grid, log=log)
        params, losses = train(X, T, a.steps, batch=a.batch, lr=a.lr, log=log)
        vl = validation_loss(params, Xv, Tv, batch=a.batch)
        log(f"validation loss {vl:.4f}")
        save(params, a.out)
        log(json.dumps({"train_loss_last": losses[-1][1], "val_loss": vl, "samples": a.samples,
                        "steps": a.steps, "batch": a.batch, "grid": a.grid}))
    else:
        params = load(a.weights)
        res = warm_start_benchmark(params, list(range(a.batch)), a.grid, tol=a.tol, batch=a.batch)
        print(json.dumps(res))


if __name__ == "__main__":
    main()
