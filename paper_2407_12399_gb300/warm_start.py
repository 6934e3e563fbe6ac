"""Learned warm start (not in the paper): data, training and the warm-started
solve, all on the GPU through the library's C ABI.

1. Pairs (f, g): seeded 64^3 inputs from `synthetic.warm_start_input`
   (generated on the host by a spawn pool), each simplified by the plain
   solver (Algorithm 1, stop rule L <= 0.01 L_0); g is the simplified field.
2. Training: the U-Net (tsf_unet_*) by Adam on mean((g0 - g)^2), one pair
   per step, pairs in a seeded random order each epoch.
3. Warm-started solve of a field f: g0 = net(f, tau); the solver takes f's
   own target diagram (the signal pairs of D(f), Section 3), starts from g0
   instead of f and iterates Algorithm 1 to its stop rule.
"""
from __future__ import annotations

import multiprocessing as mp
import os
import time

import numpy as np

from . import Field, UNet, params, tsf_create_field, tsf_destroy_field, tsf_set_signal_threshold, \
    tsf_set_start_field, tsf_simplify
from . import synthetic

TRAIN_SHAPE = (64, 64, 64)


def _gen(args):
    i, n, seed, shape = args
    f, tau = synthetic.warm_start_input(i, n, seed, shape)
    return i, f, tau


def generate_inputs(n, seed=4, shape=TRAIN_SHAPE, workers=None):
    """The n training inputs, generated by a spawn pool (numpy only)."""
    workers = workers or min(16, os.cpu_count() or 1)
    jobs = [(i, n, seed, shape) for i in range(n)]
    out = [None] * n
    if workers <= 1:
        for j in jobs:
            i, f, tau = _gen(j)
            out[i] = (f, tau)
        return out
    with mp.get_context("spawn").Pool(workers) as pool:
        for i, f, tau in pool.imap_unordered(_gen, jobs, chunksize=4):
            out[i] = (f, tau)
    return out


def solve_pairs(inputs, stop_s=0.01, max_iters=1000):
    """g for every input by the plain solver on the GPU; returns a list of
    (f, tau, g, iterations) with f and g as torch CUDA tensors."""
    import torch
    out = []
    for f, tau in inputs:
        fd = torch.from_numpy(np.ascontiguousarray(f)).cuda()
        fld = Field(fd)
        fld.set_threshold(float(tau))
        g_host, st = fld.simplify(stop_s=stop_s, max_iters=max_iters)
        g = torch.from_numpy(g_host).cuda()
        fld.close()
        out.append((fd, float(tau), g, int(st["iters"])))
    return out


def train(net, pairs, epochs=4, lr=1e-3, seed=0, log=None):
    """Adam steps over the pairs, one pair per step, in a seeded shuffled
    order per epoch; returns the mean loss of every epoch."""
    rng = np.random.default_rng(seed)
    hist = []
    for ep in range(epochs):
        order = rng.permutation(len(pairs))
        tot = 0.0
        for k in order:
            f, tau, g = pairs[k][:3]
            tot += net.train_step(f, g, tau, lr)
        hist.append(tot / max(len(pairs), 1))
        if log:
            log(f"epoch {ep}: mean loss {hist[-1]:.3e}")
    return hist


def solve(f_host, tau, stream=None, g0=None, stop_s=0.01, max_iters=1000):
    """The solve of f through the C ABI from host memory: the target diagram
    of f; the start field g0 (device tensor, None = f itself); simplify to
    the stop rule.  Returns (g as a host array, stats, seconds)."""
    f_host = np.ascontiguousarray(f_host, np.float32)
    lz, ly, lx = f_host.shape
    cs = stream.cuda_stream if stream is not None else 0
    t = time.perf_counter()
    h = tsf_create_field(lx, ly, lz, f_host.ctypes.data, 0, cs)
    try:
        tsf_set_signal_threshold(h, tau)
        if g0 is not None:
            tsf_set_start_field(h, g0.data_ptr(), 1)
        out = np.empty_like(f_host)
        st = tsf_simplify(h, params(stop_s=stop_s, max_iters=max_iters), out.ctypes.data, 0)
    finally:
        tsf_destroy_field(h)
    return out, st, time.perf_counter() - t


def warm_solve(net, f_host, tau, stream=None, stop_s=0.01, max_iters=1000):
    """Inference (g0 = net(f)) then the solve from g0 against f's targets,
    timed together from host memory to the host result."""
    import torch
    t = time.perf_counter()
    fd = torch.from_numpy(np.ascontiguousarray(f_host, np.float32)).cuda()
    g0 = net.forward(fd, tau)
    torch.cuda.synchronize()
    t_inf = time.perf_counter() - t
    g, st, t_solve = solve(f_host, tau, stream=stream, g0=g0, stop_s=stop_s, max_iters=max_iters)
    return g, st, time.perf_counter() - t, t_inf


def save(net, path):
    np.save(path, net.params())


def load(path, stream=None):
    return UNet(np.load(path), stream=stream)


__all__ = ["generate_inputs", "solve_pairs", "train", "solve", "warm_solve", "save", "load", "TRAIN_SHAPE"]


WEIGHTS = os.path.join(os.path.dirname(os.path.abspath(__file__)), "unet_warm_start.npy")


def train_default(n_pairs=2000, epochs=4, lr=1e-3, seed=4, out=WEIGHTS, log=print):
    """The warm-start network of this package: n_pairs 64^3 solver pairs from
    the mixture and filament generators, trained from unet_init(0); writes
    the fp32 parameters to `out`.  Returns (net, training report)."""
    import torch
    t0 = time.perf_counter()
    inputs = generate_inputs(n_pairs, seed=seed)
    t1 = time.perf_counter()
    pairs = solve_pairs(inputs)
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    net = UNet(seed=0)
    hist = train(net, pairs, epochs=epochs, lr=lr, seed=seed, log=log)
    torch.cuda.synchronize()
    t3 = time.perf_counter()
    if out:
        save(net, out)
    base = float(np.mean([float(((p[0] - p[2]) ** 2).mean()) for p in pairs]))
    rep = {"pairs": n_pairs, "shape": list(TRAIN_SHAPE), "epochs": epochs, "lr": lr, "seed": seed,
           "generate_s": t1 - t0, "solve_s": t2 - t1, "train_s": t3 - t2,
           "solver_iterations_mean": float(np.mean([p[3] for p in pairs])),
           "epoch_loss": hist, "identity_loss": base}
    return net, rep


if __name__ == "__main__":
    import argparse
    import json
    ap = argparse.ArgumentParser(description="train the warm-start network on solver pairs (GPU)")
    ap.add_argument("--pairs", type=int, default=2000)
    ap.add_argument("--epochs", type=int, default=4)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--out", default=WEIGHTS)
    a = ap.parse_args()
    _, rep = train_default(a.pairs, a.epochs, a.lr, out=a.out)
    print(json.dumps(rep))
