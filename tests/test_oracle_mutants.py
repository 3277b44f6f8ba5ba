"""Mutation check of the oracle's pins (CPU only).

The pins in test_oracle_pins.py, test_gpad_oracle.py, test_backtrack_oracle.py,
test_penalty_oracle.py, test_mlp_oracle.py, test_stream_kkt.py, test_kkt_oracle.py and
test_spring_mass.py tie
the oracle and the spring-mass inputs to facts outside them (dense KKT solves, closed forms,
brute force, Riccati, PyTorch's autograd, Adam and BF16 cast, scipy's hold discretisation,
Newton's law).  This file plants one plausible mistake at a time in a private copy -- a
dropped probability weight or factor 1/2, a flipped sign, a transposed operand, an
overwritten child sum, the paper's garbled signs and extrapolation taken literally -- and
checks that the unchanged pins reject every copy.  A mistake they let through is a gap in
the pins.

C mistakes go into a copy of stotree_oracle.c compiled into its own library, which the
oracle module then calls; Python mistakes go into a copy of oracle.py, mlp.py,
stream_kkt.py, kkt_check.py or workloads.py executed as a separate module, which the pin modules then use
in place of the real one.  Nothing here touches the installed oracle or the CUDA path, and
each planted text must occur exactly once in its source, so an edit that moves a line makes
this file fail loudly instead of silently testing nothing.
"""
import ctypes
import inspect
import itertools
import subprocess
import sys
import types

import numpy as np
import pytest

from oracle import mlp as M
from oracle import oracle as O
from oracle import kkt_check as KC
from oracle import stream_kkt as SK
from paper_2107_01745_b300 import workloads as W
from tests import (test_backtrack_oracle, test_fg_oracle, test_gpad_oracle, test_kkt_oracle, test_mlp_oracle,
                   test_oracle_pins, test_penalty_oracle, test_spring_mass, test_stream_kkt)

PIN_MODULES = [test_oracle_pins, test_gpad_oracle, test_backtrack_oracle, test_penalty_oracle, test_fg_oracle]
# Python parts of the oracle: (module, the name the pin modules import it under, pin modules)
TARGETS = {
    "oracle": (O, "O", PIN_MODULES),
    "mlp": (M, "M", [test_mlp_oracle]),
    "stream": (SK, "SK", [test_stream_kkt]),
    # the optimality residuals that the library's FP64 check is compared with
    "kkt": (KC, "KC", [test_kkt_oracle]),
    # the spring-mass generator of the shared input module, pinned by physics and probability
    "inputs": (W, "W", [test_spring_mass]),
}

# (id, mistake, text in the source, planted text)
C_MUTANTS = [
    ("leaf_P_no_pi", "leaf P^l without the probability pi^l",
     "Pl[k * nx + k] = p->prob[l] * p->PN[k];", "Pl[k * nx + k] = p->PN[k];"),
    ("Rbar_no_pi", "pi^i dropped from Rbar = pi R + sum B'PB",
     "Rb[a * nu + a] = pi * p->R[a];", "Rb[a * nu + a] = p->R[a];"),
    ("gu_no_half", "factor 1/2 dropped from the linear input cost in gu",
     "gui[a] = 0.5 * pi * p->r[a];", "gui[a] = pi * p->r[a];"),
    ("gx_no_pi", "pi^i dropped from the linear state cost in gx",
     "gxi[a] = 0.5 * pi * p->q[a];", "gxi[a] = 0.5 * p->q[a];"),
    ("M_transposed_PA", "M = sum B'(PA)' instead of B'PA",
     "s += Bj[k * nu + a] * PA[k * nx + b];", "s += Bj[k * nu + a] * PA[b * nx + k];"),
    ("K_sign", "K = +Rbar^-1 M",
     "Ki[a * nx + b] = -sol[a];", "Ki[a * nx + b] = sol[a];"),
    ("P_minus_MK", "P = pi Q + sum A'PA - M'K",
     "s += M[k * nx + a] * Ki[k * nx + b];", "s -= M[k * nx + a] * Ki[k * nx + b];"),
    ("chol_back_sub", "back substitution reads the (zero) upper triangle of L",
     "for (int k = i + 1; k < n; ++k) s -= L[k * n + i] * x[k];",
     "for (int k = i + 1; k < n; ++k) s -= L[i * n + k] * x[k];"),
    ("leaf_s_no_half", "leaf s^l = y^l instead of y^l / 2",
     "s[(size_t)l * nx + a] = 0.5 * yl[a] +", "s[(size_t)l * nx + a] = yl[a] +"),
    ("leaf_s_pN_no_half", "leaf s^l with pi^l p_N instead of pi^l p_N / 2",
     "0.5 * p->prob[l] * p->pN[a]", "p->prob[l] * p->pN[a]"),
    ("v_no_half", "v^i = y_u^i + ... instead of y_u^i / 2 + ...",
     "v[a] = 0.5 * yi[nx + a]", "v[a] = yi[nx + a]"),
    ("child_sum_overwrites", "child sum assigned, not accumulated (Algorithm 3 read literally)",
     "v[a] += acc;", "v[a] = acc;"),
    ("backward_A_not_transposed", "backward child sum with A^j instead of A^j'",
     "acc += Aj[k * nx + a] * sj[k];", "acc += Aj[a * nx + k] * sj[k];"),
    ("backward_minus_Kv", "s^i with -K'v instead of +K'v",
     "for (int k = 0; k < nu; ++k) acc += Ki[k * nx + a] * v[k];",
     "for (int k = 0; k < nu; ++k) acc -= Ki[k * nx + a] * v[k];"),
    ("ubar_sign", "ubar = +Rbar^-1 v",
     "for (int a = 0; a < nu; ++a) ub[a] = -ub[a];", "for (int a = 0; a < nu; ++a) ub[a] = ub[a];"),
    ("backward_skips_root", "backward loop stops before the root stage",
     "for (int t = p->N - 1; t >= 0; --t) {\n        const int first = p->soff[t], last = p->soff[t + 1];\n"
     "#pragma omp parallel for schedule(static)",
     "for (int t = p->N - 1; t >= 1; --t) {\n        const int first = p->soff[t], last = p->soff[t + 1];\n"
     "#pragma omp parallel for schedule(static)"),
    ("forward_no_c", "disturbance c^j dropped from the rollout",
     "double acc = homogeneous ? 0.0 : p->c[(size_t)j * nx + a];", "double acc = 0.0;"),
    ("forward_open_loop_u", "rollout with ubar^i in place of u^i = K x + ubar",
     "for (int k = 0; k < nu; ++k) acc += Bj[a * nu + k] * ui[k];",
     "for (int k = 0; k < nu; ++k) acc += Bj[a * nu + k] * ubar[(size_t)i * nu + k];"),
    ("forward_root_zero", "x^0 = 0 instead of p in Algorithm 3",
     "for (int a = 0; a < nx; ++a) x[a] = homogeneous ? 0.0 : x0[a];",
     "for (int a = 0; a < nx; ++a) x[a] = 0.0;"),
    ("dual_offset_nonleaf", "nonleaf dual blocks at i nx instead of i (nx + nu) (reads stay inside y)",
     "return i < p->Np ? (size_t)i * (p->nx + p->nu)", "return i < p->Np ? (size_t)i * p->nx"),
    ("forward_skips_last_stage", "rollout stops one stage early (leaves never set)",
     "for (int t = 0; t < p->N; ++t) {", "for (int t = 0; t < p->N - 1; ++t) {"),
]

PY_MUTANTS = [
    ("proj_unscaled", "box projection on Y instead of the scaled box S Y",
     "return np.minimum(np.maximum(v, o.sq * o.lo), o.sq * o.hi)",
     "return np.minimum(np.maximum(v, o.lo), o.hi)"),
    ("prox_unscaled", "z_lambda clamps v instead of v / sqrt(pi)",
     "t = v / s\n", "t = v\n"),
    ("residual_sign", "R = Hx - z instead of z - Hx",
     "r = z - h\n", "r = h - z\n"),
    ("T_sign", "T(y) = y + lam R (the sign of the forward-backward map taken literally)",
     "T=yb - lam * r", "T=yb + lam * r"),
    ("fbe_no_half", "FBE with lam ||Hx - z||^2 instead of lam / 2",
     "0.5 * lam * float(np.dot(h - z, h - z))", "lam * float(np.dot(h - z, h - z))"),
    ("fbe_no_g", "FBE without the g(z) term (matters for soft terms)",
     "phi = -(f + g_val(o, z) +", "phi = -(f +"),
    ("fbe_grad_sign", "grad phi = R - lam Hbar x_lin(R)",
     'return pt["r"] + lam * hbar_lin(o, pt["r"])', 'return pt["r"] - lam * hbar_lin(o, pt["r"])'),
    ("sigma_swapped", "support function with lo and hi swapped",
     "out[pos] = hi[pos] * y[pos]\n    out[neg] = lo[neg] * y[neg]",
     "out[pos] = lo[pos] * y[pos]\n    out[neg] = hi[neg] * y[neg]"),
    ("huber_prox_threshold", "Huber prox switching at delta instead of delta (1 + a rho)",
     "np.where(e <= o.delta * (1.0 + ar), e / (1.0 + ar), e - ar * o.delta)",
     "np.where(e <= o.delta, e / (1.0 + ar), e - ar * o.delta)"),
    ("soft_prox_unscaled_step", "soft-constraint prox moves by rho instead of rho / (lam pi)",
     "np.maximum(e_up - ar, 0.0)", "np.maximum(e_up - o.rho, 0.0)"),
    ("huber_conj_no_quadratic", "conjugate of the Huber term without y^2 / (2 rho)",
     "tot[k2] += y[k2] ** 2 / (2.0 * o.rho[k2])", "tot[k2] += 0.0 * y[k2]"),
    ("l1_conj_prox_unclipped", "closed-form prox of the l1 conjugate not clipped to [-rho, rho]",
     "eta[k1] = np.clip(eta[k1], -o.rho[k1], o.rho[k1])", "eta[k1] = eta[k1]"),
    ("huber_value_quadratic", "Huber value quadratic beyond delta",
     "np.where(d <= delta, 0.5 * d * d, delta * (d - 0.5 * delta))", "0.5 * d * d"),
    ("lbfgs_gamma", "L-BFGS H0 = <s,q>/<s,s> I instead of <s,q>/<q,q> I",
     "gamma = float(np.dot(s_new, y_new)) / float(np.dot(y_new, y_new))",
     "gamma = float(np.dot(s_new, y_new)) / float(np.dot(s_new, s_new))"),
    ("lbfgs_keeps_oldest", "L-BFGS memory drops the newest pair instead of the oldest",
     "self.S.pop(0)\n            self.Y.pop(0)", "self.S.pop()\n            self.Y.pop()"),
    ("lbfgs_alpha_order", "second loop of the two-loop recursion pairs the alphas in push order",
     "zip(zip(self.S, self.Y, rhos), reversed(alphas))", "zip(zip(self.S, self.Y, rhos), alphas)"),
    ("power_lambda_inverted", "step size lam = 0.9 L instead of 0.9 / L",
     "return safety / L, L", "return safety * L, L"),
    ("nama_literal_extrapolation", "NAMA's w = y + tau d + (1 - tau) R (Algorithm 2 read literally)",
     'pt["y"] + tau * d + (1.0 - tau) * fb_dir', 'pt["y"] + tau * d + (1.0 - tau) * pt["r"]'),
    ("minfbe_no_fb_step", "MINFBE's update y+ = w instead of T(w)",
     'new = fb_point(o, wp["T"], lam)\n        if backtrack == "original" and original_backtrack_fails(o, wp, new, lam, bt_beta):'
     '\n            halve()\n            continue\n        g_new',
     'new = fb_point(o, wp["y"], lam)\n        if backtrack == "original" and original_backtrack_fails(o, wp, new, lam, bt_beta):'
     '\n            halve()\n            continue\n        g_new'),
    ("gpad_theta_sign", "GPAD's theta recurrence with + theta^2",
     "th_prev, th = th, 0.5 * (np.sqrt(th ** 4 + 4.0 * th * th) - th * th)",
     "th_prev, th = th, 0.5 * (np.sqrt(th ** 4 + 4.0 * th * th) + th * th)"),
    ("gpad_extrapolation_sign", "GPAD extrapolates backwards",
     "(yb - y_prev)", "(y_prev - yb)"),
    ("original_rule_no_beta", "original backtracking test without the factor (1 - beta)",
     "> (1.0 - beta) * float(np.dot(R, R))", "> float(np.dot(R, R))"),
    ("original_rule_half_curvature", "original backtracking test with lam / 2 <R, grad^2 fhat R>",
     "return lam * float(np.dot(R, HR)) >", "return 0.5 * lam * float(np.dot(R, HR)) >"),
    ("simple_rule_no_lambda", "simple backtracking test without lam on the gradient difference",
     'lhs = lam * float(np.linalg.norm(-hT + pt["h"]))', 'lhs = float(np.linalg.norm(-hT + pt["h"]))'),
    ("halving_doubles", "NAMA's backtracking doubles lambda",
     "nonlocal lam, pt\n        lam *= 0.5", "nonlocal lam, pt\n        lam *= 2.0"),
    # general constraint maps z = F x + G u
    ("fg_ht_drops_G", "H'y without the G'y part (the inputs never see the dual)",
     "blk[:, nx:] = Yn @ p.G", "blk[:, nx:] = 0.0"),
    ("fg_hx_drops_Gu", "Hx without the G u part",
     "h[:npl * nc] = (x[:npl] @ p.F.T + u @ p.G.T).reshape(-1)", "h[:npl * nc] = (x[:npl] @ p.F.T).reshape(-1)"),
    ("fg_leaf_dual_dropped", "the leaves' dual left out of H'y",
     "out[npl * (nx + self.nu):] = (Yl @ p.FN).reshape(-1)", "out[npl * (nx + self.nu):] = 0.0"),
]

# the warm-start network (oracle/mlp.py) and the streamed optimality check (oracle/stream_kkt.py)
MLP_MUTANTS = [
    ("gelu_cubic_coefficient", "tanh-GELU cubic coefficient 0.0447 instead of 0.044715",
     "GELU_A = 0.044715", "GELU_A = 0.0447"),
    ("gelu_grad_chain", "GELU derivative without the factor 3 of the cubic term",
     "(1.0 + 3.0 * GELU_A * z * z)", "(1.0 + GELU_A * z * z)"),
    ("bf16_truncates", "BF16 storage by truncation instead of rounding",
     "r = ((u + 0x7FFF + lsb) >> 16) << 16", "r = (u >> 16) << 16"),
    ("bf16_ties_up", "BF16 ties rounded up instead of to even",
     "r = ((u + 0x7FFF + lsb) >> 16) << 16", "r = ((u + 0x8000) >> 16) << 16"),
    ("loss_unmasked", "loss over the padded outputs too",
     'diff = (f["Y"] - T) * mask', 'diff = (f["Y"] - T)'),
    ("loss_mean_over_all", "loss averaged over every output instead of the valid ones",
     "count = mask.sum()", "count = float(mask.size)"),
    ("grad_W2_transposed", "weight gradient of the hidden layer transposed",
     'g["W2"] = dZ2.T @ f["A1"]', 'g["W2"] = f["A1"].T @ dZ2'),
    ("backprop_W2_transposed", "data gradient through the hidden layer with W2' instead of W2",
     'dA1 = dZ2 @ f["W2"]', 'dA1 = dZ2 @ f["W2"].T'),
    ("adam_no_bias_correction", "Adam without the first moment's bias correction",
     "mh = m / (1.0 - beta1 ** t)", "mh = m"),
    ("adam_eps_inside_sqrt", "Adam with eps under the square root",
     "(np.sqrt(vh) + eps)", "np.sqrt(vh + eps)"),
    ("feature_stage_unscaled", "stage feature t instead of t / N",
     "out[r, nx] = stage[i] / horizon", "out[r, nx] = stage[i]"),
]

STREAM_MUTANTS = [
    ("leaf_multiplier_no_2", "leaf multiplier without the factor 2 of the quadratic cost",
     "mu[j] = 2.0 * prob[j] * PN * x[j]", "mu[j] = prob[j] * PN * x[j]"),
    ("child_A_not_transposed", "parents collect A^c mu^c instead of A^c' mu^c",
     'np.add.at(accA, pp, np.einsum("nij,ni->nj", A, mu[b0:b1]))',
     'np.add.at(accA, pp, np.einsum("nij,nj->ni", A, mu[b0:b1]))'),
    ("dynamics_no_c", "dynamics residual without the disturbance",
     "res = x[b0:b1] - ax - bu - hom * c", "res = x[b0:b1] - ax - bu"),
    ("u_equation_no_r", "u equations without the linear input cost",
     "+ prob[:npn, None] * r[None, :] + yu + accB", "+ yu + accB"),
    ("root_not_checked", "the root state is not compared with the parameter",
     "return {\"dynamics\": max(dyn_res, root_res)", "return {\"dynamics\": dyn_res"),
]

KKT_MUTANTS = [
    ("kkt_leaf_costate_no_2", "leaf costate without the factor 2 of the quadratic cost",
     "mu[j] = 2.0 * prob[j] * PN * x[j]", "mu[j] = prob[j] * PN * x[j]"),
    ("kkt_child_A_not_transposed", "parents collect A^c mu^c instead of A^c' mu^c",
     "sumA[parent[j]] += p.A[j].T @ mu[j]", "sumA[parent[j]] += p.A[j] @ mu[j]"),
    ("kkt_no_dual_in_u_equation", "u equation without the dual's input part",
     "+ prob[j] * r + y[o + nx:o + nx + nu] + sumB[j]", "+ prob[j] * r + sumB[j]"),
    ("kkt_dynamics_no_c", "dynamics residual without the disturbance",
     "p.B[j] @ u[i] + p.c[j])", "p.B[j] @ u[i])"),
    ("kkt_sign_at_upper_bound", "multiplier at an upper bound required to be <= 0",
     "elif at_hi and not at_lo:\n                    sign = max(sign, -yk)",
     "elif at_hi and not at_lo:\n                    sign = max(sign, yk)"),
    ("kkt_soft_kink_one_sided", "soft term's subdifferential at the upper bound taken as {0}",
     "rho[k] if hk >= hi[k] - tol_active else 0.0", "0.0"),
    ("kkt_huber_unsaturated", "Huber derivative rho d without the cap at delta",
     "gd = rho[k] * min(d, delta[k])", "gd = rho[k] * d"),
    ("kkt_fg_no_G_in_u_equation", "general maps: the u equations without G'y",
     "= p.G.T @ yi", "= 0.0 * (p.G.T @ yi)"),
    ("kkt_fg_leaf_dual_dropped", "general maps: the leaves' FN'y left out of the costates",
     "= p.FN.T @ y[o:o + ncn]", "= 0.0 * (p.FN.T @ y[o:o + ncn])"),
    ("kkt_gap_support_bound", "gap: the support function takes lo for a positive multiplier",
     "t = y * (hi - h)", "t = y * (lo - h)"),
    ("kkt_gap_huber_conjugate", "gap: Huber's conjugate without y^2 / (2 rho)",
     "+ y * y / (2.0 * rho)", ""),
    ("kkt_fg_sign_at_upper_bound", "general maps: multiplier of z at its upper bound required to be <= 0",
     "elif at_hi and not at_lo:\n                sign = max(sign, -yk)",
     "elif at_hi and not at_lo:\n                sign = max(sign, yk)"),
]

INPUT_MUTANTS = [
    ("actuator_sign", "actuator pushes both masses forward",
     "Bc[M + j, j] = -1.0 / mass", "Bc[M + j, j] = 1.0 / mass"),
    ("dampers_to_ground", "dampers tie each mass to the ground instead of its neighbours",
     "Ac[M:, M:] = -(b_d / mass) * Lap", "Ac[M:, M:] = -(b_d / mass) * np.eye(M)"),
    ("euler_input_matrix", "input matrix by Euler (Bc Ts) instead of the exact hold",
     "return F[:n, :n].copy(), F[:n, n:].copy()", "return F[:n, :n].copy(), Bc * Ts"),
    ("markov_ignores_mode", "every node branches with the first mode's conditional probabilities",
     "cond.extend([list(P_c[b]) for b in nxt])", "cond.extend([list(P_c[0]) for b in nxt])"),
    ("disturbance_modes_swapped", "disturbance of mode 0 given to mode 1 and back",
     'c[1:] = np.asarray(S["c_mode"])[modes[1:]][:, None]', 'c[1:] = np.asarray(S["c_mode"])[1 - modes[1:]][:, None]'),
]

PY_ALL = ([("oracle",) + m for m in PY_MUTANTS] + [("mlp",) + m for m in MLP_MUTANTS]
          + [("stream",) + m for m in STREAM_MUTANTS] + [("kkt",) + m for m in KKT_MUTANTS]
          + [("inputs",) + m for m in INPUT_MUTANTS])


ParameterSet = type(pytest.param(None))  # what pytest.param returns


def _plant(src: str, old: str, new: str) -> str:
    assert src.count(old) == 1, f"planted text must occur exactly once in the oracle: {old!r}"
    return src.replace(old, new)


class _BacktrackCase:
    """Stands for the module fixture `case` of test_backtrack_oracle.py (problem, oracle, L of
    the dense Hessian), built when the pin runs so that its oracle is the copy under test."""
    dense_L = {}

    def __init__(self, idx):
        self.idx = idx
        self.name = test_backtrack_oracle.BOXED[idx].name

    def build(self):
        T = test_backtrack_oracle
        p = T.BOXED[self.idx]
        o = T.O.LQOracle(p)
        assert T.O.fb_point(o, np.zeros(o.m), 0.1)["res_inf"] > 0.1
        if self.idx not in self.dense_L:
            self.dense_L[self.idx] = T._dense_L(p)
        return p, o, self.dense_L[self.idx]


class _SolvedCase:
    """Stands for the module fixture `solved` of test_kkt_oracle.py: a problem and its certified
    QP solution, which come from the oracle's solver and the dense KKT system, not from the
    module under test, so they are computed once."""
    cache = {}

    def __init__(self, idx):
        self.idx = idx
        self.name = test_kkt_oracle.PROBS[idx].name

    def build(self):
        if self.idx not in self.cache:
            p = test_kkt_oracle.PROBS[self.idx]
            self.cache[self.idx] = (p,) + test_kkt_oracle._solution(p)
        return self.cache[self.idx]


FIXTURES = {(test_backtrack_oracle, "case"): [_BacktrackCase(i) for i in range(len(test_backtrack_oracle.BOXED))],
            (test_kkt_oracle, "solved"): [_SolvedCase(i) for i in range(len(test_kkt_oracle.PROBS))]}


def _cases(mod):
    """(name, function, kwargs) for every pin of a module whose arguments all come from its
    parametrize marks or from FIXTURES (other fixtures are left out)."""
    for name, fn in vars(mod).items():
        if not name.startswith("test_") or not inspect.isfunction(fn):
            continue
        if any(m.name == "slow" for m in getattr(fn, "pytestmark", [])):
            continue
        axes = []
        for m in getattr(fn, "pytestmark", []):
            if m.name != "parametrize":
                continue
            names = m.args[0]
            names = [a.strip() for a in names.split(",")] if isinstance(names, str) else list(names)
            axes.append((names, list(m.args[1])))
        for arg in inspect.signature(fn).parameters:
            if (mod, arg) in FIXTURES:
                axes.append(([arg], FIXTURES[(mod, arg)]))
        covered = {a for names, _ in axes for a in names}
        if set(inspect.signature(fn).parameters) - covered:
            continue
        for combo in itertools.product(*[vals for _, vals in axes]):
            kw = {}
            for (names, _), v in zip(axes, combo):
                vals = v.values if isinstance(v, ParameterSet) else (v if len(names) > 1 else (v,))
                kw.update(zip(names, vals))
            yield f"{mod.__name__.split('.')[-1]}::{name}", fn, kw


ALL_CASES = [c for mod in PIN_MODULES for c in _cases(mod)]
TARGET_CASES = {k: [c for mod in mods for c in _cases(mod)] for k, (_, _, mods) in TARGETS.items()}
# slips in the general nonsmooth terms: their pins first (the order only saves time)
PENALTY_SLIPS = {"fbe_no_g", "huber_prox_threshold", "soft_prox_unscaled_step", "huber_conj_no_quadratic",
                 "l1_conj_prox_unclipped", "huber_value_quadratic"}


def _first_failing_pin(cases=ALL_CASES):
    """Run the pins in order; return the first that fails (or None).  Overflow in a diverging
    copy is expected and not reported as a warning."""
    for name, fn, kw in cases:
        try:
            with np.errstate(over="ignore", invalid="ignore", divide="ignore"):
                fn(**{k: v.build() if isinstance(v, (_BacktrackCase, _SolvedCase)) else v for k, v in kw.items()})
        except pytest.skip.Exception:
            continue
        except Exception as e:  # an assertion, a refused factor, a non-finite value ...
            return f"{name}({', '.join(f'{k}={getattr(v, 'name', v)}' for k, v in kw.items())}): {type(e).__name__}"
    return None


def _load_c(src: str, tmp_path) -> ctypes.CDLL:
    c_file, so_file = tmp_path / "mutant.c", tmp_path / "libmutant.so"
    c_file.write_text(src)
    subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
                           str(c_file), "-o", str(so_file), "-lm"])
    lib = ctypes.CDLL(str(so_file))
    lib.orc_factor.restype = ctypes.c_int
    lib.orc_solve.restype = ctypes.c_int
    lib.orc_num_threads.restype = ctypes.c_int
    return lib


def _load_py(src: str, like: types.ModuleType = O) -> types.ModuleType:
    mod = types.ModuleType(like.__name__ + "_mutant")
    mod.__file__ = like.__file__
    sys.modules[mod.__name__] = mod  # dataclasses look their module up while the class is built
    try:
        exec(compile(src, like.__file__, "exec"), mod.__dict__)
    finally:
        del sys.modules[mod.__name__]
    return mod


def test_harness_collects_the_pins():
    names = {n for n, _, _ in ALL_CASES}
    assert len(ALL_CASES) >= 60 and len(names) >= 25


def test_unmodified_copies_pass_every_pin(tmp_path, monkeypatch):
    """The harness itself: a compiled copy of the C oracle and an executed copy of oracle.py,
    both unmodified, pass every pin, so a failure below comes from the planted mistake."""
    with open(O._SRC) as f:
        lib = _load_c(f.read(), tmp_path)
    with open(O.__file__) as f:
        copy = _load_py(f.read())
    copy._lib_handle = lib
    for mod in PIN_MODULES:
        monkeypatch.setattr(mod, "O", copy)
    assert _first_failing_pin() is None
    for key in ("mlp", "stream", "kkt", "inputs"):
        target, attr, mods = TARGETS[key]
        with open(target.__file__) as f:
            other = _load_py(f.read(), target)
        for mod in mods:
            monkeypatch.setattr(mod, attr, other)
        assert _first_failing_pin(TARGET_CASES[key]) is None


@pytest.mark.parametrize("mid,what,old,new", C_MUTANTS, ids=[m[0] for m in C_MUTANTS])
def test_pins_reject_planted_c_mistake(mid, what, old, new, tmp_path, monkeypatch):
    with open(O._SRC) as f:
        src = _plant(f.read(), old, new)
    monkeypatch.setattr(O, "_lib_handle", _load_c(src, tmp_path))
    caught = _first_failing_pin()
    assert caught is not None, f"no pin rejects: {what}"


@pytest.mark.parametrize("key,mid,what,old,new", PY_ALL, ids=[f"{m[0]}-{m[1]}" for m in PY_ALL])
def test_pins_reject_planted_python_mistake(key, mid, what, old, new, monkeypatch):
    target, attr, mods = TARGETS[key]
    with open(target.__file__) as f:
        mutant = _load_py(_plant(f.read(), old, new), target)
    for mod in mods:
        monkeypatch.setattr(mod, attr, mutant)
    cases = TARGET_CASES[key]
    if mid in PENALTY_SLIPS:
        cases = sorted(cases, key=lambda c: not c[0].startswith("test_penalty_oracle"))
    caught = _first_failing_pin(cases)
    assert caught is not None, f"no pin rejects: {what}"
