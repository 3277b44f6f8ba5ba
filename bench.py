#!/usr/bin/env python
"""Benchmark: milliseconds to ||z - Hx||_inf <= 1e-4 for NAMA (Algorithm 2) on the paper-scale
scenario tree (horizon 20, binary for 10 stages then one child, 1024 scenarios, 12,287 nodes,
nx = 100, nu = 50: 1.79M primal and dual variables), FP32 solve path with the FP64 factor.

One step = one cold-started NAMA solve (y0 = 0) to tolerance, inputs resident on the device;
the factor and the step-size estimate are set-up and are not timed.  MINFBE (Algorithm 1) is
timed beside it.  The solve rounds (Algorithm 3/4) are timed inside the library with CUDA
events on the launching stream for the roofline line.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
                    [--warm-train-draws D] [--warm-eval-draws E] [--spring-mass 0|1]
                    [--profile nama|minfbe|batched|warm|infer|warm_round|warm_round_full|uneven_round]

Beside the headline the line carries the batched workload (512 instances), the learned warm
start (training, inference, warm vs cold), the factor, GPAD (warm start and to tolerance), the
step-size backtracking rules, soft state bounds and the spring-mass experiment of Section IV-A.

Under torchrun each rank solves its own replica of the instance (independent problems, no
collective on the data path; scaling "weak"); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "ms to KKT tol 1e-4 (MINFBE/NAMA), batched/warm vs plain; solve-step GB/s"
GPAD_MAX_ITER = 5000
TOL = 1e-4
WORKLOAD = ("paper_scale: horizon 20, branching 2 for stages 0-9 then 1 (1024 scenarios, 12287 nodes), "
            "nx=100, nu=50, per-node A_j = A + 0.05 N(0,1) (rho(A)=0.98), B_j ~ N(0,1/nx), w ~ N(0,0.05^2), "
            "Q=diag(U[0.5,2]), R=0.1I, P_N=I, box = 80% of the unconstrained range (not below the first two "
            "stages), x0 ~ U[-3,3], seed 2; NAMA cold start to ||z-Hx||_inf <= 1e-4")


def _traffic_per_launch(rounds, rhs):
    """DRAM traffic per solve round from the committed ncu summary, if it was taken on the current
    kernel source (else None).  Weighted by the mix of 1- and 2-RHS rounds in the timed region."""
    import hashlib
    import re
    path = os.path.join(ROOT, "profiles", "k_tree_paper_scale.md")
    src = os.path.join(ROOT, "paper_2107_01745_b300", "csrc", "solve.cu")
    if not os.path.exists(path):
        return None
    text = open(path).read()
    m = re.search(r"sha256 `([0-9a-f]{64})`", text)
    t1 = re.search(r"traffic_bytes_per_round_1rhs: (\d+)", text)
    t2 = re.search(r"traffic_bytes_per_round_2rhs: (\d+)", text)
    if not (m and t1 and t2):
        return None
    if hashlib.sha256(open(src, "rb").read()).hexdigest() != m.group(1):
        return None
    n2 = rhs - rounds  # rounds with two right-hand sides (the others have one)
    n1 = rounds - n2
    return (n1 * int(t1.group(1)) + n2 * int(t2.group(1))) / max(rounds, 1)


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6400.0, "fallback"


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None
        self._out = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        self._out = open(self.path, "w")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=self._out, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        # start timing only once the sampler is running (its first line is written)
        t0 = time.time()
        while self.proc is not None and time.time() - t0 < 3.0:
            if os.path.getsize(self.path) > 0:
                break
            time.sleep(0.01)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.proc.wait(timeout=5)
        self._out.close()

    def summary(self):
        if not self.path or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                except ValueError:
                    continue
                for n, v in zip(names, parts[5:9]):
                    if v.lower() == "active":
                        reasons.add(n)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def _max_over_ranks(pg, value: float, device) -> float:
    """The largest of every rank's value (the job's time is its slowest rank's); pg = None or
    torch.distributed with an initialised process group (NCCL on GPUs, gloo on CPU)."""
    if pg is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def _config(world, m_dual, n_primal):
    """The workload description both arms print (no measured or estimated quantities)."""
    return {"workload": WORKLOAD, "method": "nama", "solver_tol": TOL, "lbfgs_mem": 5,
            "step_size": "0.9 / L, L from 50 power iterations of the dual Hessian (seeded start)",
            "m_dual": int(m_dual), "n_primal": int(n_primal),
            "l2": "inputs larger than L2: each solve round streams 2.04 GB of factor arrays",
            "parallelism": f"replicas x{world}"}


def run_ours(args):
    import torch
    from paper_2107_01745_b300 import workloads as W
    from paper_2107_01745_b300.stotree import StoTree

    world, rank, local = _dist()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
        pg = dist
    p = W.paper_scale(2)
    st = StoTree(p, precision="fp32", device=dev)
    st.factor()
    factor = run_factor(st, p)
    r0 = torch.as_tensor(np.random.default_rng(7).standard_normal(st.m), dtype=torch.float32, device=dev)
    lam, Lhat = st.estimate_lambda(r0, iters=50, safety=0.9)
    x0 = st.to_dev(p.x0)
    stream = torch.cuda.current_stream()

    def one(method, y0=None):
        res = st.solve(method, lam, x0=x0, y0=y0, tol=TOL, mem=5, max_iter=500)
        if res["info"]["res_inf"] > TOL:
            raise RuntimeError(f"{method} stopped at residual {res['info']['res_inf']}")
        return res

    for _ in range(args.warmup):
        one("nama")
        one("minfbe")

    def timed(method, k):
        infos = []
        if pg is not None:
            pg.barrier()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(k):
            infos.append(one(method)["info"])
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / k
        return _max_over_ranks(pg, ms, dev), infos

    st.set_timing(True)
    st.get_timing()  # reset counters
    with ClockSampler(local) as clk:
        nama_ms, nama_infos = timed("nama", args.steps)
        solve_ms, rounds, rhs = st.get_timing()
        st.set_timing(False)
        minfbe_ms, minfbe_infos = timed("minfbe", args.steps)
    gpad = run_gpad(st, lam, x0, stream, pg, dev, args.steps)
    backtrack = run_backtrack(st, Lhat, x0)
    soft = run_soft(st, lam, x0)
    spring = run_spring_mass(dev) if args.spring_mass else None
    largest = run_largest(dev, max(1, min(args.steps, 3))) if args.largest else None

    mat_bytes, vec_bytes = st.solve_bytes()
    alg_bytes = rounds * mat_bytes + rhs * vec_bytes
    achieved = alg_bytes / (solve_ms * 1e-3) / 1e9
    peak, peak_kind = _peaks()

    # end to end through the public API: pinned host inputs in, results out, every step
    x0_h = torch.as_tensor(p.x0, dtype=torch.float32).pin_memory()
    y0_h = torch.zeros(st.m, dtype=torch.float32).pin_memory()
    y_h = torch.empty(st.m, dtype=torch.float32).pin_memory()
    x_h = torch.empty((st.Nn, st.nx), dtype=torch.float32).pin_memory()
    u_h = torch.empty((st.Np, st.nu), dtype=torch.float32).pin_memory()
    x0_d = torch.empty_like(x0)
    y0_d = torch.empty(st.m, dtype=torch.float32, device=dev)
    if pg is not None:
        pg.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        x0_d.copy_(x0_h, non_blocking=True)
        y0_d.copy_(y0_h, non_blocking=True)
        res = st.solve("nama", lam, x0=x0_d, y0=y0_d, tol=TOL, mem=5, max_iter=500)
        y_h.copy_(res["y"], non_blocking=True)
        x_h.copy_(res["x"], non_blocking=True)
        u_h.copy_(res["u"], non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1) / args.steps
    e2e_ms = _max_over_ranks(pg, e2e_ms, dev)
    h2d = 4 * (st.nx + st.m)
    d2h = 4 * (st.m + st.Nn * st.nx + st.Np * st.nu)
    # the last e2e solution through the library's FP64 optimality check (untimed)
    kkt = st.kkt_check(x0, res["x"], res["u"], res["y"], tol_active=1e-3)
    kkt = {k: float(f"{v:.4g}") for k, v in kkt.items()}
    kkt["note"] = ("FP64 residuals of the returned (x, u, y) (stotree_kkt_check; tol_active 1e-3): max "
                   "violations, and the Fenchel-Young duality gap summed over the 1.79 M duals")

    batched = run_batched(dev, max(1, min(args.steps, 3)))
    warm = run_warm(dev, args.warm_train_draws, args.warm_eval_draws) if args.warm_train_draws > 0 else None
    line = None
    if rank == 0:
        cpu = cpu_baseline(p, lam, nama_infos[0]["iters"])
        launches = int(sum(i["launches"] for i in nama_infos))
        line = {
            "metric": METRIC, "value": round(nama_ms, 4), "unit": "ms", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(nama_ms, 4), "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": _config(world, st.m, st.n),
            "step_size": {"lambda": lam, "L_estimate": Lhat, "rule": "0.9 / L, L from 50 power iterations"},
            "nama": {"ms": round(nama_ms, 4), "iters": nama_infos[0]["iters"],
                     "solve_calls": nama_infos[0]["solve_calls"], "ls_zero": nama_infos[0]["ls_zero"]},
            "minfbe": {"ms": round(minfbe_ms, 4), "iters": minfbe_infos[0]["iters"],
                       "solve_calls": minfbe_infos[0]["solve_calls"]},
            "roofline": {"kernel": "k_tree (one Algorithm 3/4 solve round = a backward-pass launch + a forward-pass launch)", "bound": "hbm",
                         "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                         "frac": round(achieved / peak, 4), "peak_source": peak_kind,
                         "traffic": _traffic_per_launch(rounds, rhs), "rounds": rounds, "rhs": rhs,
                         "algorithmic_bytes_per_round": mat_bytes, "vector_bytes_per_rhs": vec_bytes,
                         "avg_round_ms": round(solve_ms / max(rounds, 1), 5)},
            "solve_step_gbs": round(achieved, 1),
            "e2e": {"value": round(e2e_ms, 4), "unit": "ms", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "gpu_launches": launches,
            "kkt": kkt,
            "factor": factor,
            "gpad": gpad,
            "backtracking": backtrack,
            "soft_states": soft,
            "spring_mass": spring,
            "largest": largest,
            "batched": batched,
            "warm_start": warm,
            "clocks": clk.summary(),
            "cpu_baseline": cpu,
        }
    if pg is not None:
        pg.barrier()
        pg.destroy_process_group()
    return line


def run_factor(st, p):
    """The offline factor (Section III-D) of the paper-scale instance, FP64 on the device: its
    time (set-up, not part of the headline), an operation count of its products, and the
    FP64 rate of a cuBLAS DGEMM on this GPU for comparison (the factor is bound by the FP64
    pipe).  Flops counted: per child j, P^j [A^j | B^j] and [A^j | B^j]' (P^j [A^j | B^j]);
    per parent, the Cholesky factor of Rbar, K = -Rbar^-1 M and the update M' K."""
    import torch
    nx, nu = p.nx, p.nu
    t = p.tree
    nc, npn = t.num_nodes - 1, t.num_nonleaf
    flops = nc * (2.0 * nx * nx * (nx + nu) + 2.0 * (nx + nu) ** 2 * nx) + \
        npn * (nu ** 3 / 3.0 + 2.0 * nu * nu * nx + 2.0 * nx * nx * nu)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    stream = torch.cuda.current_stream()
    ms = []
    for _ in range(3):
        torch.cuda.synchronize()
        e0.record(stream)
        st.factor()
        e1.record(stream)
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    fac_ms = min(ms)
    a = torch.randn(4096, 4096, dtype=torch.float64, device=st.device)
    torch.matmul(a, a)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(5):
        torch.matmul(a, a)
    e1.record(stream)
    torch.cuda.synchronize()
    dgemm_tf = 5 * 2.0 * 4096 ** 3 / (e0.elapsed_time(e1) * 1e-3) / 1e12
    return {"ms": round(fac_ms, 2), "gflop": round(flops / 1e9, 1), "tflops": round(flops / (fac_ms * 1e-3) / 1e12, 3),
            "fp64_dgemm_tflops_measured": round(dgemm_tf, 3), "frac_of_dgemm": round(flops / (fac_ms * 1e-3) / 1e12 / dgemm_tf, 3)}


def run_gpad(st, lam, x0, stream, pg, dev, steps):
    """GPAD (accelerated dual projected gradient) on the same instance: its five-step warm start
    of Section III-F followed by NAMA, timed as one step, and one cold GPAD run to the same
    tolerance (the comparison method of Section IV)."""
    import torch

    def warm_nama():
        g = st.solve("gpad", lam, x0=x0, tol=TOL, max_iter=5, allow_not_converged=True, outputs=False)
        res = st.solve("nama", lam, x0=x0, y0=g["y"], tol=TOL, mem=5, max_iter=500, outputs=False)
        if res["info"]["res_inf"] > TOL:
            raise RuntimeError(f"NAMA after GPAD stopped at residual {res['info']['res_inf']}")
        return g["info"], res["info"]

    warm_nama()
    if pg is not None:
        pg.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        gi, ni = warm_nama()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    cold = st.solve("gpad", lam, x0=x0, tol=TOL, max_iter=GPAD_MAX_ITER, allow_not_converged=True, outputs=False)
    ci = cold["info"]
    return {"warm5_then_nama_ms": round(ms, 4), "gpad5_ms": round(gi["ms"], 4), "nama_iters_after_gpad5": ni["iters"],
            "gpad_to_tol": {"ms": round(ci["ms"], 3), "iters": ci["iters"], "res_inf": ci["res_inf"],
                            "converged": ci["status"] == 0, "max_iter": GPAD_MAX_ITER}}


def run_backtrack(st, Lhat, x0):
    """NAMA with the step-size backtracking of Section III-B when L is not known: started from
    ten times the power-iteration estimate of 1/L, one solve per rule."""
    out = {"lambda0": 10.0 / Lhat}
    for rule, param in (("simple", 0.25), ("original", 0.1)):
        st.solve("nama", 10.0 / Lhat, x0=x0, tol=TOL, max_iter=500, backtrack=rule, bt_param=param, outputs=False)
        i = st.solve("nama", 10.0 / Lhat, x0=x0, tol=TOL, max_iter=500, backtrack=rule, bt_param=param,
                     outputs=False)["info"]
        out[rule] = {"param": param, "ms": round(i["ms"], 3), "iters": i["iters"], "halvings": i["halvings"],
                     "lambda_final": i["lambda_"], "solve_calls": i["solve_calls"], "res_inf": i["res_inf"]}
    return out


def run_soft(st, lam, x0):
    """The same instance with soft state bounds (Section II-B: rho = 1 times the distance of
    each state to its interval; inputs stay hard): NAMA to the same tolerance, one timed solve
    after one warm-up.  The hard box is restored afterwards."""
    n = st.nx + st.nu
    st.set_penalty([1] * st.nx + [0] * st.nu, 1.0, 1.0)
    try:
        st.solve("nama", lam, x0=x0, tol=TOL, max_iter=500, outputs=False)
        i = st.solve("nama", lam, x0=x0, tol=TOL, max_iter=500, outputs=False)["info"]
    finally:
        st.set_penalty([0] * n, 0.0, 1.0)
    return {"rho": 1.0, "ms": round(i["ms"], 3), "iters": i["iters"], "solve_calls": i["solve_calls"],
            "res_inf": i["res_inf"], "converged": i["status"] == 0}


def run_largest(dev, steps):
    """The largest single instance (horizon 24, binary for 12 stages, 57,343 nodes, nx = 200,
    nu = 100: 16.8 M primal variables; per-node data generated in seeded 512-node blocks): NAMA to
    the tolerance, one warm-up solve and `steps` timed ones, the solve rounds' HBM roofline (the
    library's algorithmic bytes over the rounds' CUDA-event time), and the FP64 optimality check
    of the result.  Set-up (data generation, upload, FP64 factor, lambda) is untimed."""
    import time
    import torch
    from paper_2107_01745_b300 import workloads as W
    from paper_2107_01745_b300.stotree import StoTree
    t0 = time.time()
    p = W.largest(5)
    st = StoTree(p, precision="fp32", device=dev, chunk_nodes=4096)
    st.factor()
    r0 = torch.as_tensor(np.random.default_rng(7).standard_normal(st.m), dtype=torch.float32, device=dev)
    lam, _ = st.estimate_lambda(r0, iters=50, safety=0.9)
    x0 = st.to_dev(p.x0)
    st.solve("nama", lam, x0=x0, tol=TOL, max_iter=1000, outputs=False)
    setup_s = time.time() - t0
    stream = torch.cuda.current_stream()
    st.set_timing(True)
    st.get_timing()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        res = st.solve("nama", lam, x0=x0, tol=TOL, max_iter=1000)
    e1.record(stream)
    torch.cuda.synchronize()
    solve_ms, rounds, rhs = st.get_timing()
    st.set_timing(False)
    info = res["info"]
    if info["status"] != 0 or info["res_inf"] > TOL:
        raise RuntimeError(f"largest instance: NAMA stopped at residual {info['res_inf']}")
    mat_bytes, vec_bytes = st.solve_bytes()
    gbs = (rounds * mat_bytes + rhs * vec_bytes) / (solve_ms * 1e-3) / 1e9
    peak, peak_kind = _peaks()
    kkt = st.kkt_check(x0, res["x"], res["u"], res["y"], tol_active=1e-3)
    del res, r0, x0
    out = {"workload": "largest: horizon 24, binary for stages 0-11 then one child (4096 scenarios, 57,343 nodes), "
                       "nx=200, nu=100 (16.8 M primal variables), A_j = A + 0.02 N(0,1) with rho(A)=0.98, "
                       "B_j ~ N(0,1/nx), c ~ N(0,0.05^2), Q=I, R=0.1I, P_N=I, stored input box; seed 5; NAMA to 1e-4",
           "ms": round(e0.elapsed_time(e1) / steps, 3), "steps": steps, "iters": info["iters"],
           "solve_calls": info["solve_calls"], "res_inf": info["res_inf"],
           "roofline": {"kernel": "k_tree solve rounds", "bound": "hbm", "achieved": round(gbs, 1), "peak": peak,
                        "unit": "GB/s", "frac": round(gbs / peak, 4), "peak_source": peak_kind,
                        "algorithmic_bytes_per_round": mat_bytes, "avg_round_ms": round(solve_ms / max(rounds, 1), 4)},
           "kkt": {k: float(f"{v:.4g}") for k, v in kkt.items()},
           "setup_s": round(setup_s, 1)}
    st.close()
    del st
    torch.cuda.empty_cache()  # about 70 GB of workspace, returned before the later sections
    return out


def run_spring_mass(dev):
    """The experiment of Section IV-A: 300 initial states of the spring-mass array (stored, uniform
    on the problem's domain), each solved from y0 = 0 to ||z - Hx||_inf <= 5e-4 by NAMA, MINFBE
    (L-BFGS memory 5) and GPAD; the oracle calls (right-hand sides through Algorithm 3/4) per
    problem, summarised as in the paper: the share solved within 50 calls and the median.  One
    tree and factor serve every initial state (x0 enters only the solve).  FP64 path: the duals
    are of order 100 and near the tolerance the steps fall below FP32's resolution of them."""
    import torch
    from paper_2107_01745_b300 import workloads as W
    from paper_2107_01745_b300.stotree import StoTree
    X, meta = W.spring_mass_x0s()
    p = W.spring_mass(X[0], p_max=meta["p_max"])
    st = StoTree(p, precision="fp64", device=dev)
    st.factor()
    r0 = torch.as_tensor(np.random.default_rng(0).standard_normal(st.m), dtype=torch.float64, device=dev)
    lam, _ = st.estimate_lambda(r0, iters=50, safety=0.9)
    x0s = [st.to_dev(x) for x in X]
    out = {"problems": len(X), "tol": 5e-4, "lambda": lam, "p_max": meta["p_max"], "dtype": "f64",
           "paper": {"share_le50_calls_nama_minfbe": 0.84, "gpad_median_calls": 188}}
    for method in ("nama", "minfbe", "gpad"):
        cap = 2000 if method == "gpad" else 1000
        st.solve(method, lam, x0=x0s[0], tol=5e-4, max_iter=cap, outputs=False)  # warm-up
        calls, iters, ms, bad = [], [], [], 0
        for x in x0s:
            i = st.solve(method, lam, x0=x, tol=5e-4, max_iter=cap, outputs=False, allow_not_converged=True)["info"]
            calls.append(i["solve_calls"])
            iters.append(i["iters"])
            ms.append(i["ms"])
            bad += i["status"] != 0
        calls = np.asarray(calls)
        out[method] = {"share_le50_calls": round(float(np.mean(calls <= 50)), 4),
                       "median_calls": float(np.median(calls)), "mean_iters": round(float(np.mean(iters)), 2),
                       "mean_ms": round(float(np.mean(ms)), 3), "total_s": round(float(np.sum(ms)) / 1e3, 3),
                       "not_converged": int(bad), "max_iter": cap}
    st.close()
    return out


def run_warm(dev, train_draws, eval_draws):
    """Learned warm start on the warm-start workload: labels from the batched NAMA, Adam training
    of the tensor-core perceptron, then batched NAMA on held-out draws from y0 = 0 and from the
    learned start (inference and the phi fallback test counted in the warm time)."""
    import torch
    from paper_2107_01745_b300 import warmstart as WS
    from paper_2107_01745_b300 import workloads as W
    system = W.warm_start_system(4)
    lam = WS.batch_lambda(system, device=dev)
    t0 = time.time()
    data = WS.make_dataset(system, W.WARM_TRAIN_SEED, train_draws, lam, device=dev)
    label_s = time.time() - t0
    label_solve_ms, label_iters = data["solve_ms"], float(data["iters"].mean())
    starter = WS.WarmStarter(system, hidden=256, batch=8192, seed=0, device=dev)
    fit = starter.fit(data, epochs=10, lr=1e-3)
    del data
    ev = WS.EvalSet(W.warm_start_draws(system, W.WARM_EVAL_SEED, eval_draws, dtype=np.float32), lam, device=dev)
    WS.warm_vs_cold(starter, ev)  # warm-up (graph capture)
    r = WS.warm_vs_cold(starter, ev)
    ev.close()
    net = starter.net
    # algorithmic FLOPs of one training step (unpadded widths): forward 3 products, backward 2
    # data products (no input gradient) and 3 weight products
    flops = 2.0 * net.batch * (2 * net.d_in * net.hidden + 3 * net.hidden ** 2 + 3 * net.hidden * net.d_out)
    step_ms = fit["ms"] / max(1, fit["steps"])
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    peak = float(peaks.get("bf16_tflops_sustained", 1400.0))
    achieved = flops / (step_ms * 1e-3) / 1e12
    L = fit["loss"]
    return {"workload": "warm start: horizon 15, branching 4 for stages 0-3 (256 scenarios, 3157 nodes), nx=20, "
                        "nu=10, shared A (rho 0.95), B ~ N(0,1), Q=I, R=0.1I, P_N=I, |u|<=0.3, |x|<=5, per draw "
                        "x0 ~ U[-3,3], c ~ N(0,0.1^2), seed 4; train draws seeds 40000+, eval draws 90000+",
            "train_draws": train_draws, "eval_draws": eval_draws, "label_s": round(label_s, 2),
            "label_solve_ms": round(label_solve_ms, 1), "label_iters_mean": label_iters,
            "train_steps": fit["steps"], "train_ms": round(fit["ms"], 1), "train_step_us": round(1e3 * step_ms, 1),
            "loss_first": float(L[:10].mean()), "loss_last": float(L[-100:].mean()),
            "train_roofline": {"bound": "tensor", "achieved": round(achieved, 2), "peak": peak, "unit": "TFLOP/s",
                               "frac": round(achieved / peak, 4), "peak_source": "measured bf16 sustained" if peaks
                               else "fallback", "flops_per_step": flops},
            "cold_ms": round(r["cold_ms"], 2), "warm_ms": round(r["warm_ms"], 2),
            "warm_infer_ms": round(r["warm_infer_ms"], 2), "warm_fallback_test_ms": round(r["warm_fallback_test_ms"], 2),
            "cold_iters_mean": r["cold_iters_mean"], "warm_iters_mean": r["warm_iters_mean"],
            "cold_iters_max": r["cold_iters_max"], "warm_iters_max": r["warm_iters_max"],
            "fallbacks": r["fallbacks"], "all_converged": r["converged"],
            "warm_direct_ms": round(r["direct_ms"], 2), "warm_direct_iters_mean": r["direct_iters_mean"],
            "warm_direct_iters_max": r["direct_iters_max"],
            "warm_direct_speedup": round(r["cold_ms"] / r["direct_ms"], 3)}


def batched_round_bytes(groups, affine=True):
    """Algorithmic bytes of one batched solve round (one right-hand side per instance, FP32): y read
    and Hx written (m each), s and ubar of every nonleaf node written and read once, the state of
    every non-root node written and read once, and for the affine round (Algorithm 3) the
    disturbances c and the constant terms gamma read once.  The stage matrices (a few KB per
    group) are not counted."""
    total = 0.0
    for g in groups:
        t = g.tree()
        nn, npl = t.num_nodes, t.num_nonleaf
        m_i = npl * (g.nx + g.nu) + t.num_leaves * g.nx
        per = 2 * m_i + 2 * g.nx * npl + 2 * g.nu * npl + 2 * g.nx * (nn - 1)
        if affine:
            per += g.nx * (nn - 1) + (g.nx + g.nu) * npl
        total += 4.0 * per * g.num_instances
    return total


def time_batched_rounds(groups, dev, reps=20):
    """Mean time of `reps` batched solve rounds (Algorithm 3, one right-hand side per instance) and
    their HBM roofline: algorithmic bytes (batched_round_bytes) over the CUDA-event time on the
    launching stream; the tuner's choice of round kernel beside it."""
    import torch
    from paper_2107_01745_b300.stotree import StoBatch
    sb = StoBatch(groups, device=dev)
    sb.factor()
    stream = torch.cuda.current_stream()
    y = torch.randn(sb.M, device=dev, generator=torch.Generator(device=dev).manual_seed(1)) * 0.01
    for _ in range(3):
        sb.solve_step(y)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        sb.solve_step(y)
    e1.record(stream)
    torch.cuda.synchronize()
    sb.round_status()
    ms = e0.elapsed_time(e1) / reps
    nbytes = batched_round_bytes(groups)
    peak, peak_kind = _peaks()
    gbs = nbytes / (ms * 1e-3) / 1e9
    cfg = sb.round_config(1)
    sb.close()
    return {"round_ms": round(ms, 4), "algorithmic_bytes": nbytes, "dual_variables": sb.M,
            "roofline": {"bound": "hbm", "achieved": round(gbs, 1), "peak": peak, "unit": "GB/s",
                         "frac": round(gbs / peak, 4), "peak_source": peak_kind},
            "round_kernel": cfg}


def run_batched(dev, steps):
    """Batched uneven workload: 512 instances (16 shape groups x 32) solved by one batched NAMA
    per step, against the plain single-instance FP32 path run instance after instance (every
    instance timed, the times summed)."""
    import torch
    from paper_2107_01745_b300 import workloads as W
    from paper_2107_01745_b300.stotree import StoBatch, StoTree
    groups = W.batched_uneven(3)
    sb = StoBatch(groups, device=dev)
    sb.factor()
    lams = sb.group_lambdas()
    stream = torch.cuda.current_stream()
    sb.nama(lams, tol=TOL, max_iter=500)  # warm-up (graph capture)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        res = sb.nama(lams, tol=TOL, max_iter=500, outputs=False)
    e1.record(stream)
    torch.cuda.synchronize()
    batched_ms = e0.elapsed_time(e1) / steps
    infos = res["infos"]
    if not all(i["status"] == 0 and i["res_inf"] <= TOL for i in infos):
        raise RuntimeError("batched NAMA: some instance did not reach the tolerance")
    # algorithmic vector bytes of the solve rounds: every right-hand side an active instance
    # pushes through Algorithm 3/4 reads y and writes Hx (m reals each) and writes and reads the
    # per-node scratch s, ubar, x, u once; NAMA pushes 1 + 3 k right-hand sides in k iterations
    vec_bytes = 0.0
    inst = 0
    for g in groups:
        t = g.tree()
        m_i = t.num_nonleaf * (g.nx + g.nu) + t.num_leaves * g.nx
        per_rhs = 4.0 * (2 * m_i + 2 * (g.nu * t.num_nonleaf + g.nx * t.num_nodes))
        for _ in range(g.num_instances):
            vec_bytes += per_rhs * (1 + 3 * infos[inst]["iters"])
            inst += 1
    peak, peak_kind = _peaks()
    rounds_gbs = vec_bytes / (batched_ms * 1e-3) / 1e9
    # the plain single-instance path on every instance: one handle per group, the instance's
    # disturbances uploaded and the factor redone (set-up, untimed), one warm-up solve, then the
    # timed solve; the plain time is the sum of the 512 timed solves
    plain_ms, sample = 0.0, 0
    for gi, g in enumerate(groups):
        st = StoTree(g.instance(0), precision="fp32", device=dev)
        for k in range(g.num_instances):
            if k > 0:
                st.set_dynamics(None, None, g.c[k])
            st.factor()
            x0 = st.to_dev(g.x0[k])
            st.solve("nama", lams[gi], x0=x0, tol=TOL, max_iter=500, outputs=False)  # warm-up
            torch.cuda.synchronize()
            a, bb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            st.solve("nama", lams[gi], x0=x0, tol=TOL, max_iter=500, outputs=False)
            bb.record(stream)
            torch.cuda.synchronize()
            plain_ms += a.elapsed_time(bb)
            sample += 1
        st.close()
    # the same groups with a binding input box (|u| <= 0.3 instead of the configured |u| <= 1), so
    # that the instances iterate: labelled as a variant, beside the literal workload
    import dataclasses
    bgroups = [dataclasses.replace(g, ulo=-0.3 * np.ones(g.nu), uhi=0.3 * np.ones(g.nu)) for g in groups]
    sbb = StoBatch(bgroups, device=dev)
    sbb.factor()
    blams = sbb.group_lambdas()
    sbb.nama(blams, tol=TOL, max_iter=1000)  # warm-up (graph capture)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    bres = sbb.nama(blams, tol=TOL, max_iter=1000, outputs=False)
    e1.record(stream)
    torch.cuda.synchronize()
    binfos = bres["infos"]
    binding = {"workload": "the same 512 instances with the input box |u| <= 0.3 (a variant: the configured box is "
                           "|u| <= 1, under which most instances do not iterate)",
               "batched_ms": round(e0.elapsed_time(e1), 3),
               "all_converged": all(i["status"] == 0 and i["res_inf"] <= TOL for i in binfos),
               "mean_iters": round(float(np.mean([i["iters"] for i in binfos])), 3),
               "max_iters": int(max(i["iters"] for i in binfos)),
               "instances_needing_iterations": int(sum(i["iters"] > 0 for i in binfos))}
    sbb.close()
    # solve rounds alone: the literal workload (tile kernel: groups up to nx = 64) and the
    # learned-warm-start evaluation batch, a family that iterates (column kernel)
    rounds_uneven = time_batched_rounds(groups, dev)
    rounds_warm = time_batched_rounds([W.warm_start_draws(W.warm_start_system(4), W.WARM_EVAL_SEED, 5000,
                                                          dtype=np.float32)], dev)
    return {"workload": "16 shape groups x 32 instances (512): horizon U{10..30}, branching 2 or 3 for the first "
                        "stages with 64-1024 scenarios, nx in {16, 32, 64}, nu = nx/2, shared A, B, costs and box per "
                        "group, own x0 ~ U[-3,3] and w ~ N(0, 0.05^2) per instance, seed 3; NAMA to 1e-4",
            "binding_box_variant": binding,
            "rounds": {"uneven_512": rounds_uneven,
                       "warm_start_eval_5000": dict(rounds_warm, workload="the learned-warm-start family (horizon 15, "
                                                    "branching 4 for 4 stages, nx=20, nu=10), 5,000 evaluation draws")},
            "instances": sb.ninst, "dual_variables": sb.M, "batched_ms": round(batched_ms, 3),
            "max_iters": int(max(i["iters"] for i in infos)),
            "mean_iters": round(float(np.mean([i["iters"] for i in infos])), 3),
            "instances_needing_iterations": int(sum(i["iters"] > 0 for i in infos)),
            "plain_sequential_ms": round(plain_ms, 1),
            "plain_sample": f"all {sample} instances timed with the single-instance path, one after another (the sum of their solve times)",
            "speedup": round(plain_ms / batched_ms, 2),
            "solve_vector_rate": {"achieved": round(rounds_gbs, 1), "unit": "GB/s", "algorithmic_bytes": vec_bytes,
                                  "note": "vector bytes of the solve rounds over the whole batched NAMA time "
                                          "(elementwise passes and host round trips in the time, not in the bytes); "
                                          "the per-round roofline is under rounds"},
            "roofline": rounds_warm["roofline"]}


def cpu_baseline(p, lam, gpu_iters):
    """The FP64 oracle, as it stands, on the host cores: one full NAMA solve of the same instance
    (factor not timed), capped at 60 iterations."""
    from oracle import oracle as O
    o = O.LQOracle(p)
    t0 = time.perf_counter()
    res = O.nama(o, lam, tol=TOL, max_iter=60)
    sec = time.perf_counter() - t0
    return {"value": round(sec * 1e3, 1), "unit": "ms", "cores": O.num_threads(), "kind": "oracle",
            "sample": f"one full cold-started NAMA solve of the same instance with the same lambda "
                      f"(FP64 C + numpy, {res['iters']} iterations, status {res['status']}, residual "
                      f"{res['res_inf']:.2e}; factor not timed)"}


# wall-time budget of the reference arm's timed steps: every measured step is one full solve
# (tens of seconds on the host cores), so a run with many steps stops measuring after this
REF_BUDGET_S = 300.0


def run_reference(args, problem=None):
    """The oracle as the reference arm: same workload, config, metric and unit, on the host cores.
    Each timed step is one full cold-started NAMA solve to the tolerance; warm-up steps run one
    iteration each (the oracle has no caches or compilation to warm).  Steps stop being measured
    once REF_BUDGET_S of measured time is spent (at least one full solve): the line then says
    how many were measured and why."""
    world, rank, _ = _dist()
    if rank != 0:
        return None
    from oracle import oracle as O
    from paper_2107_01745_b300 import workloads as W
    p = W.paper_scale(2) if problem is None else problem
    o = O.LQOracle(p)
    lam, _ = O.power_lambda(o, np.random.default_rng(7).standard_normal(o.m))
    for _ in range(args.warmup):
        O.nama(o, lam, tol=TOL, max_iter=1)
    times, iters, spent = [], [], 0.0
    for _ in range(args.steps):
        t0 = time.perf_counter()
        r = O.nama(o, lam, tol=TOL, max_iter=500)
        dt = time.perf_counter() - t0
        if r["status"] != "converged":
            raise RuntimeError(f"oracle NAMA stopped at residual {r['res_inf']}")
        times.append(dt)
        iters.append(r["iters"])
        spent += dt
        if spent >= REF_BUDGET_S:
            break
    ms = 1e3 * statistics.mean(times)
    measured = len(times)
    note = (f"{measured} of {args.steps} steps measured: the measured steps reached the "
            f"{REF_BUDGET_S:.0f} s budget of the reference arm") if measured < args.steps else \
        f"all {measured} steps measured"
    n_primal = p.tree.num_nonleaf * p.nu + (p.tree.num_nodes - 1) * p.nx
    return {"impl": "reference", "metric": METRIC, "value": round(ms, 1), "unit": "ms", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 1), "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": _config(world, o.m, n_primal),
            "steps_measured": measured, "steps_note": note,
            "cpu_baseline": {"value": round(ms, 1), "unit": "ms", "cores": O.num_threads(), "kind": "oracle",
                             "sample": f"each timed step: one full cold-started NAMA solve of the instance by the "
                                       f"FP64 oracle (C + numpy), {iters[0]} iterations to tolerance; mean over "
                                       f"{measured} solves (factor and step-size estimate not timed)"},
            "e2e": {"value": round(ms, 1), "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def run_profile(method):
    """Set-up and one warm solve outside the profiler range, then exactly one solve inside
    cudaProfilerStart/Stop (for ncu --profile-from-start off)."""
    import torch
    from paper_2107_01745_b300 import workloads as W
    from paper_2107_01745_b300.stotree import StoBatch, StoTree
    if method == "warm":
        from paper_2107_01745_b300 import warmstart as WS
        system = W.warm_start_system(4)
        lam = WS.batch_lambda(system)
        data = WS.make_dataset(system, W.WARM_TRAIN_SEED, 64, lam)
        starter = WS.WarmStarter(system, hidden=256, batch=8192, seed=0)
        starter.net.set_draws(data["x0"], data["c"], data["y"])
        starter.net.train(5)
        torch.cuda.synchronize()
        torch.cuda.cudart().cudaProfilerStart()
        hist = starter.net.train(3)
        torch.cuda.synchronize()
        torch.cuda.cudart().cudaProfilerStop()
        print(json.dumps({"profiled": method, "train_steps": 3, "loss": float(hist[-1])}))
        return
    if method == "infer":
        from paper_2107_01745_b300 import warmstart as WS
        system = W.warm_start_system(4)
        ev = W.warm_start_draws(system, W.WARM_EVAL_SEED, 500, dtype=np.float32)
        x0 = torch.as_tensor(ev.x0, dtype=torch.float32, device="cuda")
        c = torch.as_tensor(ev.c, dtype=torch.float32, device="cuda")
        starter = WS.WarmStarter(system, hidden=256, batch=8192, seed=0)
        starter.predict(x0, c)
        torch.cuda.synchronize()
        torch.cuda.cudart().cudaProfilerStart()
        y = starter.predict(x0, c)
        torch.cuda.synchronize()
        torch.cuda.cudart().cudaProfilerStop()
        print(json.dumps({"profiled": method, "draws": 500, "rows": 500 * system.tree().num_nodes,
                          "outputs": int(y.numel())}))
        return
    if method in ("warm_round", "warm_round_full", "uneven_round"):
        # one batched solve round (Algorithm 3): 300 draws of the learned-warm-start family (the
        # column kernel; a few GB on the device), the 5,000 evaluation draws (for single-pass
        # counters only: about 50 GB on the device), or the 512-instance workload's 16 shape groups
        # with 8 instances each (the tile kernel; a few GB)
        if method == "warm_round":
            groups = [W.warm_start_draws(W.warm_start_system(4), W.WARM_EVAL_SEED, 300, dtype=np.float32)]
        elif method == "warm_round_full":
            groups = [W.warm_start_draws(W.warm_start_system(4), W.WARM_EVAL_SEED, 5000, dtype=np.float32)]
        else:
            groups = W.batched_uneven(3, instances=8)
        sb = StoBatch(groups)
        sb.factor()
        y = torch.randn(sb.M, device="cuda", generator=torch.Generator(device="cuda").manual_seed(1)) * 0.01
        for _ in range(3):
            sb.solve_step(y)
        torch.cuda.synchronize()
        torch.cuda.cudart().cudaProfilerStart()
        sb.solve_step(y)
        torch.cuda.synchronize()
        torch.cuda.cudart().cudaProfilerStop()
        sb.round_status()
        print(json.dumps({"profiled": method, "round_kernel": sb.round_config(1),
                          "algorithmic_bytes": batched_round_bytes(groups)}))
        return
    if method == "batched":
        sb = StoBatch(W.batched_uneven(3))
        sb.factor()
        lams = sb.group_lambdas()
        sb.nama(lams, tol=TOL, max_iter=500)
        torch.cuda.synchronize()
        torch.cuda.cudart().cudaProfilerStart()
        res = sb.nama(lams, tol=TOL, max_iter=500, outputs=False)
        torch.cuda.synchronize()
        torch.cuda.cudart().cudaProfilerStop()
        print(json.dumps({"profiled": method, "max_iters": int(max(i["iters"] for i in res["infos"]))}))
        return
    p = W.paper_scale(2)
    st = StoTree(p, precision="fp32")
    st.factor()
    r0 = torch.as_tensor(np.random.default_rng(7).standard_normal(st.m), dtype=torch.float32, device="cuda")
    lam, _ = st.estimate_lambda(r0, iters=50)
    st.solve(method, lam, tol=TOL)
    torch.cuda.synchronize()
    torch.cuda.cudart().cudaProfilerStart()
    res = st.solve(method, lam, tol=TOL)
    torch.cuda.synchronize()
    torch.cuda.cudart().cudaProfilerStop()
    print(json.dumps({"profiled": method, **res["info"]}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--warm-train-draws", type=int, default=50000,
                    help="training draws of the learned warm start (0 skips it)")
    ap.add_argument("--warm-eval-draws", type=int, default=5000,
                    help="held-out draws the learned warm start is evaluated on")
    ap.add_argument("--largest", type=int, default=1,
                    help="1: also solve the largest single instance (about a minute of set-up)")
    ap.add_argument("--spring-mass", type=int, default=1,
                    help="run the 300-problem spring-mass experiment of Section IV-A (0 skips it)")
    ap.add_argument("--profile", choices=["nama", "minfbe", "batched", "warm", "infer", "warm_round", "warm_round_full",
                                          "uneven_round"],
                    default=None,
                    help="run one solve inside a profiler range (no JSON benchmark line)")
    args = ap.parse_args()
    if args.profile:
        run_profile(args.profile)
        return
    if args.warmup < 3:
        raise SystemExit("at least 3 warm-up steps")
    line = run_reference(args) if args.impl == "reference" else run_ours(args)
    if line is not None:
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
