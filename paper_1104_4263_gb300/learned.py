"""Training data, training loop and evaluation of the learned preconditioner.

Every computation runs in libdie (through the ctypes binding in die.py): the operator
products and solves that generate the pairs, the encoding of a pair, the network's
forward and backward passes and Adam (tensor-core kernels), and flexible GMRES.  This
module only schedules those calls and draws seeded inputs (workloads.py).

Pairs (contrast, right-hand side) -> solution come from the solver in two ways:
  * "solve": u from a regularised GMRES solve of A u = b_inc for the incident plane wave
    of the field's angle, and b = A u (one more product), so that u = A^-1 b holds to
    rounding even where the solve stopped early; b differs from b_inc by the solve's
    residual (the physical pairs the initial guess is for);
  * "product": u = a smooth random field (correlation 0.1 wavelength), b = A u from one
    FFT-speed product, so u = A^-1 b exactly (general inputs such as Krylov vectors, the
    preconditioner's use).
"""
from __future__ import annotations

import dataclasses
import math
import time

import numpy as np

from . import die, workloads as W

HELD_OUT_BASE = 1_000_000     # seed indices of the held-out fields (training uses 0 .. count-1)


@dataclasses.dataclass
class Dataset:
    x: "object"        # torch float32 (count, 6, n, n), on the device
    t: "object"        # torch float32 (count, 4, n, n)
    kinds: list
    gen_s: float


def _solve_u(op, b, tol, max_iters):
    u, rep = op.solve(b, restart=60, tol=tol, max_iters=max_iters, regularized=True, inner=die.DIE_FP32_INNER)
    return u, rep


def make_dataset(count: int, n: int = 128, solve_every: int = 40, solve_tol: float = 1e-5, first: int = 0,
                 solve_iters: int = 2000) -> Dataset:
    """`count` training pairs on n x n grids (h = 1/60): pair i uses the random field of seed
    first + i; every `solve_every`-th pair is a "solve" pair, the rest "product" pairs."""
    import torch
    t0 = time.perf_counter()
    p0 = W.config4_field(first, n)
    op = die.Operator(p0.eps_r, p0.h)
    X = torch.empty((count, 6, n, n), dtype=torch.float32, device="cuda")
    T = torch.empty((count, 4, n, n), dtype=torch.float32, device="cuda")
    kinds = []
    for i in range(count):
        p = W.config4_field(first + i, n)
        op.set_permittivity(p.eps_r)
        if solve_every and i % solve_every == 0:
            u, _ = _solve_u(op, op.plane_wave(p.psi[0]), solve_tol, solve_iters)
            b = op.apply(u)
            kinds.append("solve")
        else:
            u = torch.from_numpy(W.smooth_random_vector(W.rng_for(40, first + i), n, n, p.h)).cuda()
            b = op.apply(u)
            kinds.append("product")
        die.encode_pair(op, b, u, X[i], T[i])
    torch.cuda.synchronize()
    return Dataset(X, T, kinds, time.perf_counter() - t0)


def default_network(n: int = 128, max_batch: int = 16, seed: int = 0):
    """The 4-layer, 16-mode, width-32 network (hidden 128) with He-style random weights
    (the spectral weights scaled by 1 / width^2, as in the FNO reference)."""
    net = die.FNO(6, 4, 32, 16 if n >= 64 else max(1, n // 4), 4, 128, n, n, max_batch)
    rng = np.random.default_rng(seed)
    parts = []
    width, hid, m = 32, 128, net.desc.modes

    def lin(o, i):
        return [rng.standard_normal((o, i)) / math.sqrt(i), np.zeros(o)]

    parts += lin(width, 6)
    for _ in range(4):
        parts += lin(width, width)
        for _ in range(2):
            parts.append((rng.standard_normal((width, width, m, m, 2))) / (width * width))
    parts += lin(hid, width)
    parts += [np.zeros((4, hid)), np.zeros(4)]      # zero output layer: the network starts as M(v) = v
    net.set_params(np.concatenate([np.ravel(a) for a in parts]).astype(np.float32))
    return net


def train(net, data: Dataset, epochs: int = 10, batch: int = 16, lr: float = 1e-3, seed: int = 0):
    """Adam over shuffled mini-batches; returns the per-epoch mean losses and seconds."""
    import torch
    rng = np.random.default_rng(seed)
    count = data.x.shape[0]
    hist = []
    t0 = time.perf_counter()
    for ep in range(epochs):
        order = torch.from_numpy(rng.permutation(count)).cuda()
        lr_ep = lr * 0.5 * (1 + math.cos(math.pi * ep / max(epochs, 1)))
        tot, nb = 0.0, 0
        for s in range(0, count - batch + 1, batch):
            idx = order[s:s + batch]
            xb = data.x.index_select(0, idx).contiguous()
            tb = data.t.index_select(0, idx).contiguous()
            tot += net.train_step(xb, tb, lr_ep)
            nb += 1
        hist.append(tot / max(nb, 1))
    torch.cuda.synchronize()
    return hist, time.perf_counter() - t0


def relative_error(net, data: Dataset, batch: int = 16) -> float:
    """Relative 2-norm error of the network's outputs against the targets."""
    import torch
    num = den = 0.0
    for s in range(0, data.x.shape[0], batch):
        xb = data.x[s:s + batch].contiguous()
        if xb.shape[0] != batch:
            break
        y = net.forward(xb)
        num += float(((y - data.t[s:s + batch]) ** 2).sum())
        den += float((data.t[s:s + batch] ** 2).sum())
    return math.sqrt(num / den) if den > 0 else float("nan")


def evaluate(net, count: int, n: int = 128, tol: float = 1e-6, restart: int = 30, base_restart: int = 100,
             r_defl: int = 8, max_iters: int = 8000, flex_iters: int = 600, first: int = HELD_OUT_BASE,
             re_lo: float = -4.0):
    """On `count` held-out fields (plane-wave right-hand sides; Re eps_r in [re_lo, 16]):
      * without the network: regularised, deflated (r_defl), FP32-inner GMRES(base_restart)
        from x0 = 0 (the method of Sections 4-5; restart 30 stagnates on these fields);
      * with it: flexible GMRES(restart) with the network as initial guess and right
        preconditioner for up to flex_iters steps, then the former method from its iterate.
    Both run to tol on ||b - A u|| / ||b|| (the regularised solve's own tolerance is
    tightened until that holds), within max_iters steps in all.  Seconds exclude the
    deflation build, which is reported apart."""
    import torch
    rows = []
    p0 = W.config4_field(first, n, re_lo=re_lo)
    op = die.Operator(p0.eps_r, p0.h)
    for i in range(count):
        p = W.config4_field(first + i, n, re_lo=re_lo)
        op.set_permittivity(p.eps_r)
        b = op.plane_wave(p.psi[0])
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        D = die.Deflation(op, r_defl, tol=1e-4, regularized=True, inner=die.DIE_FP32_INNER)
        torch.cuda.synchronize()
        t_defl = time.perf_counter() - t0
        t0 = time.perf_counter()
        tol_r, iters, rep = tol, 0, None
        x = torch.zeros_like(b)
        for _ in range(4):
            x, rep = op.solve(b, x=x, restart=base_restart, tol=tol_r, max_iters=max_iters - iters,
                              regularized=True, inner=die.DIE_FP32_INNER, deflation=D)
            iters += rep["iters"]
            if rep["rel_res_orig"] <= tol or not rep["converged"] or iters >= max_iters:
                break
            tol_r *= 0.1
        torch.cuda.synchronize()
        base = {"iters": iters, "s": time.perf_counter() - t0, "rel_res_orig": rep["rel_res_orig"],
                "converged": rep["rel_res_orig"] <= tol}
        t0 = time.perf_counter()
        _, rf = die.fgmres(op, b, net=net, deflation=D, restart=restart, tol=tol, max_iters=flex_iters,
                           fallback_restart=base_restart, fallback_iters=max_iters - flex_iters)
        torch.cuda.synchronize()
        t_net = time.perf_counter() - t0
        # the network's initial guess alone, then the method without it
        t0 = time.perf_counter()
        x0 = net.precondition(op, b)
        res0 = float(torch.linalg.norm(op.apply(x0) - b) / torch.linalg.norm(b))
        tol_r, it_g, rg = tol, 0, None
        for _ in range(4):
            x0, rg = op.solve(b, x=x0, restart=base_restart, tol=tol_r, max_iters=max_iters - it_g,
                              regularized=True, inner=die.DIE_FP32_INNER, deflation=D)
            it_g += rg["iters"]
            if rg["rel_res_orig"] <= tol or not rg["converged"] or it_g >= max_iters:
                break
            tol_r *= 0.1
        torch.cuda.synchronize()
        guess = {"iters": it_g, "s": time.perf_counter() - t0, "rel_res_orig": rg["rel_res_orig"],
                 "converged": rg["rel_res_orig"] <= tol}
        rows.append({"field": first + i, "deflation_build_s": t_defl, "without_network": base,
                     "with_network": {"iters": rf["iters"], "s": t_net, "rel_res_orig": rf["rel_res_orig"],
                                      "converged": rf["converged"], "used_fallback": rf["used_fallback"]},
                     "initial_guess_only": guess, "initial_guess_rel_res": res0})
        del D
    return rows
