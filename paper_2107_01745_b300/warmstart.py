"""Learned warm start for families of scenario-tree problems that share the tree and the
dynamics (host orchestration; every computation runs in the library's kernels).

1. Labels: the batched NAMA (Algorithm 2) solves the training draws; its duals y* are the
   targets (the network learns the scaled dual ybar* = y*/sqrt(pi), Section III-E).
2. Training: the library's tensor-core perceptron, Adam on batches of (draw, node) samples.
3. Use: predicted y0 for new draws; per draw the start is kept only if its forward-backward
   envelope is not above that of y0 = 0 (phi_lambda is what both algorithms decrease), else the
   draw starts cold.  The paper's own warm start is a few accelerated dual gradient steps
   (Section III-E); this replaces them.
"""
from __future__ import annotations

import time

import numpy as np
import torch

from . import workloads as W
from .stotree import StoBatch, StoWarm


def _events():
    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


def batch_lambda(system: W.Group, device="cuda:0") -> float:
    """Step size for the family: 0.9 / L from the power iteration on one draw (the dual Hessian
    depends on neither x0 nor c)."""
    g = W.warm_start_draws(system, 0, 1)
    sb = StoBatch([g], device=device)
    sb.factor()
    lam = float(sb.group_lambdas()[0])
    sb.close()
    return lam


def solve_draws(group: W.Group, lam: float, tol=1e-4, max_iter=500, y0=None, device="cuda:0"):
    """Batched NAMA on every draw of the group; y0 [D, m] unscaled or None (cold)."""
    sb = StoBatch([group], device=device)
    sb.factor()
    D = group.num_instances
    m = int(sb.sizes[0])
    yin = None if y0 is None else y0.reshape(-1).contiguous()
    torch.cuda.synchronize()
    e0, e1 = _events()
    e0.record()
    res = sb.nama(np.array([lam]), tol=tol, max_iter=max_iter, y0=yin, outputs=False)
    e1.record()
    torch.cuda.synchronize()
    out = dict(y=res["y"].reshape(D, m), infos=res["infos"], ms=e0.elapsed_time(e1), sb=sb)
    return out


def make_dataset(system: W.Group, first_seed: int, count: int, lam: float, chunk=2048, tol=1e-4,
                 device="cuda:0"):
    """Draws first_seed .. first_seed + count - 1 with their solved duals, on the device."""
    nn = system.c.shape[1]
    x0 = torch.empty(count, system.nx, dtype=torch.float32, device=device)
    c = torch.empty(count, nn, system.nx, dtype=torch.float32, device=device)
    y = None
    iters = np.zeros(count, dtype=np.int64)
    t_solve = 0.0
    for k0 in range(0, count, chunk):
        n = min(chunk, count - k0)
        g = W.warm_start_draws(system, first_seed + k0, n, dtype=np.float32)
        r = solve_draws(g, lam, tol=tol, device=device)
        r["sb"].close()
        if y is None:
            y = torch.empty(count, r["y"].shape[1], dtype=torch.float32, device=device)
        y[k0:k0 + n] = r["y"]
        x0[k0:k0 + n] = torch.as_tensor(g.x0, device=device)
        c[k0:k0 + n] = torch.as_tensor(g.c, device=device)
        iters[k0:k0 + n] = [i["iters"] for i in r["infos"]]
        if any(i["status"] != 0 for i in r["infos"]):
            raise RuntimeError("a training draw did not converge")
        t_solve += r["ms"]
    return dict(x0=x0, c=c, y=y, iters=iters, solve_ms=t_solve, first_seed=first_seed)


class WarmStarter:
    def __init__(self, system: W.Group, hidden=256, batch=8192, seed=0, device="cuda:0"):
        self.system = system
        self.tree = system.tree()
        self.net = StoWarm(self.tree, system.nx, system.nu, hidden=hidden, batch=batch, seed=seed, device=device)

    def fit(self, data: dict, epochs=10, lr=1e-3, shuffle_seed=0):
        self.net.set_draws(data["x0"], data["c"], data["y"])
        samples = data["x0"].shape[0] * self.tree.num_nodes
        steps = epochs * (samples // self.net.batch)
        torch.cuda.synchronize()
        e0, e1 = _events()
        e0.record()
        hist = self.net.train(steps, lr=lr, seed=shuffle_seed)
        e1.record()
        torch.cuda.synchronize()
        return dict(loss=hist.cpu().numpy(), steps=steps, ms=e0.elapsed_time(e1))

    def predict(self, x0: torch.Tensor, c: torch.Tensor) -> torch.Tensor:
        self.net.set_draws(x0, c)
        return self.net.predict(0, x0.shape[0])


def choose_start(group: W.Group, lam: float, y0: torch.Tensor, device="cuda:0"):
    """Per draw: y0 if phi_lambda(y0) <= phi_lambda(0), else zeros.  Returns the start and the
    number of draws that fell back."""
    sb = StoBatch([group], device=device)
    sb.factor()
    D = group.num_instances
    f_warm = sb.nama(np.array([lam]), max_iter=0, y0=y0.reshape(-1).contiguous(), outputs=False,
                     allow_not_converged=True)["infos"]
    f_cold = sb.nama(np.array([lam]), max_iter=0, outputs=False, allow_not_converged=True)["infos"]
    sb.close()
    keep = torch.tensor([fw["fbe"] <= fc["fbe"] for fw, fc in zip(f_warm, f_cold)], device=y0.device)
    start = torch.where(keep[:, None], y0.reshape(D, -1), torch.zeros_like(y0.reshape(D, -1)))
    return start, int(D - keep.sum().item())


def warm_vs_cold(system: W.Group, starter: WarmStarter, eval_group: W.Group, lam: float, tol=1e-4,
                 device="cuda:0"):
    """Batched NAMA on the evaluation draws from y0 = 0 and from the learned start (inference
    and the fallback test included in the warm time)."""
    cold = solve_draws(eval_group, lam, tol=tol, device=device)
    cold["sb"].close()
    x0 = torch.as_tensor(eval_group.x0, dtype=torch.float32, device=device)
    c = torch.as_tensor(eval_group.c, dtype=torch.float32, device=device)
    torch.cuda.synchronize()
    e0, e1 = _events()
    e0.record()
    y0 = starter.predict(x0, c)
    start, fallbacks = choose_start(eval_group, lam, y0, device=device)
    e1.record()
    torch.cuda.synchronize()
    prep_ms = e0.elapsed_time(e1)
    warm = solve_draws(eval_group, lam, tol=tol, y0=start, device=device)
    warm["sb"].close()
    ci = np.array([i["iters"] for i in cold["infos"]])
    wi = np.array([i["iters"] for i in warm["infos"]])
    ok = all(i["status"] == 0 for i in cold["infos"] + warm["infos"])
    return dict(draws=eval_group.num_instances, cold_ms=cold["ms"], warm_ms=warm["ms"] + prep_ms,
                warm_solve_ms=warm["ms"], warm_prep_ms=prep_ms, cold_iters_mean=float(ci.mean()),
                warm_iters_mean=float(wi.mean()), cold_iters_max=int(ci.max()), warm_iters_max=int(wi.max()),
                fallbacks=fallbacks, converged=ok, y_warm=warm["y"], y_cold=cold["y"])
