"""Learned warm start for families of scenario-tree problems that share the tree and the
dynamics (host orchestration; every computation runs in the library's kernels).

1. Labels: the batched NAMA (Algorithm 2) solves the training draws; its duals y* are the
   targets (the network learns the scaled dual ybar* = y*/sqrt(pi), Section III-E).
2. Training: the library's tensor-core perceptron, Adam on batches of (draw, node) samples.
3. Use: predicted y0 for new draws; per draw the start is kept only if its forward-backward
   envelope is not above that of y0 = 0 (phi_lambda is what both algorithms decrease), else the
   draw starts cold.  The paper's own warm start is a few accelerated dual gradient steps
   (Section III-F); this replaces them.
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
    def __init__(self, system: W.Group, hidden=256, batch=8192, seed=0, device="cuda:0", infer_batch=65536):
        self.system = system
        self.tree = system.tree()
        self.net = StoWarm(self.tree, system.nx, system.nu, hidden=hidden, batch=batch, seed=seed, device=device)
        # inference runs the trained weights in a second network with a larger row batch: each
        # product is then large enough to keep the tensor cores busy (training keeps its batch)
        self._infer_args = dict(hidden=hidden, batch=max(batch, infer_batch), seed=seed, device=device)
        self._infer = None
        self._infer_version = -1
        self._version = 0

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
        self._version += 1
        return dict(loss=hist.cpu().numpy(), steps=steps, ms=e0.elapsed_time(e1))

    def predict(self, x0: torch.Tensor, c: torch.Tensor) -> torch.Tensor:
        net = self.net
        if self._infer_args["batch"] > self.net.batch:
            if self._infer is None:
                self._infer = StoWarm(self.tree, self.system.nx, self.system.nu, **self._infer_args)
            if self._infer_version != self._version:
                self._infer.set_params(self.net.params())
                self._infer_version = self._version
            net = self._infer
        net.set_draws(x0, c)
        return net.predict(0, x0.shape[0])


class EvalSet:
    """Evaluation draws in one factored batch, reused by the cold and the warm solve."""

    def __init__(self, group: W.Group, lam: float, device="cuda:0"):
        self.group, self.lam, self.device = group, lam, device
        self.sb = StoBatch([group], device=device)
        self.sb.factor()
        self.D = group.num_instances
        self.m = int(self.sb.sizes[0])
        self.x0 = torch.as_tensor(group.x0, dtype=torch.float32, device=device)
        self.c = torch.as_tensor(group.c, dtype=torch.float32, device=device)

    def nama(self, y0=None, tol=1e-4, max_iter=500):
        yin = None if y0 is None else y0.reshape(-1).contiguous()
        res = self.sb.nama(np.array([self.lam]), tol=tol, max_iter=max_iter, y0=yin, outputs=False)
        return res["y"].reshape(self.D, self.m), res["infos"]

    def phi(self, y0=None):
        """phi_lambda at the start point of every draw (a zero-iteration NAMA)."""
        yin = None if y0 is None else y0.reshape(-1).contiguous()
        infos = self.sb.nama(np.array([self.lam]), max_iter=0, y0=yin, outputs=False,
                             allow_not_converged=True)["infos"]
        return np.array([i["fbe"] for i in infos])

    def close(self):
        self.sb.close()


def choose_start(ev: EvalSet, y0: torch.Tensor):
    """Per draw: y0 if phi_lambda(y0) <= phi_lambda(0), else zeros.  Returns the start and the
    number of draws that fell back."""
    keep = torch.as_tensor(ev.phi(y0) <= ev.phi(None), device=y0.device)
    start = torch.where(keep[:, None], y0, torch.zeros_like(y0))
    return start, int(ev.D - int(keep.sum().item()))


def warm_vs_cold(starter: WarmStarter, ev: EvalSet, tol=1e-4):
    """Batched NAMA on the evaluation draws from y0 = 0 and from the learned start; the warm time
    includes inference and the fallback test.  The learned start is also timed without the
    fallback test ("direct": inference and the solve from every prediction)."""
    torch.cuda.synchronize()
    e0, e1 = _events()
    e0.record()
    y_cold, cold = ev.nama(None, tol=tol)
    e1.record()
    torch.cuda.synchronize()
    cold_ms = e0.elapsed_time(e1)
    e0, e1 = _events()
    e2, e3 = _events()
    e0.record()
    y0 = starter.predict(ev.x0, ev.c)
    e1.record()
    start, fallbacks = choose_start(ev, y0)
    e2.record()
    y_warm, warm = ev.nama(start, tol=tol)
    e3.record()
    torch.cuda.synchronize()
    # the same start taken without the fallback test (every draw from its prediction)
    e4, e5 = _events()
    e4.record()
    y1 = starter.predict(ev.x0, ev.c)
    _, direct = ev.nama(y1, tol=tol)
    e5.record()
    torch.cuda.synchronize()
    ci = np.array([i["iters"] for i in cold])
    wi = np.array([i["iters"] for i in warm])
    di = np.array([i["iters"] for i in direct])
    ok = all(i["status"] == 0 for i in cold + warm + direct)
    return dict(draws=ev.D, cold_ms=cold_ms, warm_ms=e0.elapsed_time(e3), warm_infer_ms=e0.elapsed_time(e1),
                warm_fallback_test_ms=e1.elapsed_time(e2), warm_solve_ms=e2.elapsed_time(e3),
                cold_iters_mean=float(ci.mean()), warm_iters_mean=float(wi.mean()), cold_iters_max=int(ci.max()),
                warm_iters_max=int(wi.max()), fallbacks=fallbacks, converged=ok, y_warm=y_warm, y_cold=y_cold,
                y0=y0, direct_ms=e4.elapsed_time(e5), direct_iters_mean=float(di.mean()),
                direct_iters_max=int(di.max()))
