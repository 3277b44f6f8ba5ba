"""FP64 CPU oracle for dual MINFBE / NAMA on scenario trees.

TEST INFRASTRUCTURE ONLY: imported by the tests, by the smoke check and by the
benchmark's CPU-baseline leg, never by the library.  It shares no code with
the CUDA path; both take their inputs from ``paper_2107_01745_b300.workloads``.

The heavy lifting (offline factor, Algorithms 3 and 4) is in
``stotree_oracle.c``; everything else here is plain numpy in FP64 and follows
the paper's definitions directly:

* Section II-D: prox, forward-backward map T_lambda, residual R_lambda = z - Hx,
  x(y) = grad f*(-H'y), z_lambda(y) = prox_{g/lambda}(y/lambda + Hx(y)).  g is separable
  (Section II-B): per component the indicator of a box, rho times the distance to it (a soft
  constraint; l1 when the box is a point) or rho times the Huber function of that distance.
  The sign of T_lambda follows the algorithms' own update, T(y) = y + lambda(Hx - z).
* Section III-A: the forward-backward envelope (FBE) phi_lambda, evaluated both
  by its definition and by the equivalent augmented-Lagrangian expression
  -[f(x) + <y, Hx - z> + lambda/2 ||Hx - z||^2].
* Section III-B, Algorithm 1: dual MINFBE with L-BFGS directions.
* Section III-C, Algorithm 2: NAMA.  The extrapolation is read as
  w = y + tau d + (1 - tau)(T(y) - y), so tau = 0 is the plain forward-backward step,
  and the dual update as y+ = T(w).
* Section III-E: diagonal preconditioning ybar^i = y^i / sqrt(pi^i); the solvers
  iterate on ybar (equivalently on S H and the box S Y with S = diag(sqrt(pi))).
  The termination test uses the unscaled residual ||z - Hx||_inf.
* Section III-B, step-size backtracking when L is unknown: eq. (original-backtracking)
  [TheStePat16], read as the descent-lemma test of the forward-backward step taken from the
  accepted line-search point w (its three terms at w are the ones the line search evaluated
  in phi(w)), evaluated through the exact second-order expansion of the quadratic fhat; on
  failure lambda is halved, the L-BFGS memory emptied and the iteration repeated from ybar.  Eq. (simple-backtracking) [BelloCruz 2016, Linesearch 1] at ybar:
  lambda ||grad fhat(T(ybar)) - grad fhat(ybar)|| > eps'' ||T(ybar) - ybar|| halves lambda,
  empties the memory and is tested again.
* Section III-F (warm start) and Section IV (comparison method): GPAD, the accelerated
  dual projected gradient, here in the theta form of Patrinos and Bemporad (2014):
  w = ybar + theta_k (1/theta_{k-1} - 1)(ybar - ybar_prev), ybar+ = T(w).

Line searches evaluate phi_lambda(w) with a full solve at every trial point
(no affine shortcut), so the oracle is slow but obviously follows the text.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import time

import numpy as np

from paper_2107_01745_b300.workloads import Problem, dual_offsets, problem_offsets

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "stotree_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")


def build_oracle(force: bool = False) -> str:
    """Compile the C oracle (gcc, -O2, OpenMP) into oracle/_build/liboracle.so."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
                               _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _SO)
    return _SO


class _OrcProblem(ctypes.Structure):
    _fields_ = [("Nn", ctypes.c_int), ("Np", ctypes.c_int), ("N", ctypes.c_int),
                ("nx", ctypes.c_int), ("nu", ctypes.c_int),
                ("parent", ctypes.c_void_p), ("cbeg", ctypes.c_void_p), ("ccnt", ctypes.c_void_p),
                ("soff", ctypes.c_void_p), ("prob", ctypes.c_void_p),
                ("A", ctypes.c_void_p), ("B", ctypes.c_void_p), ("c", ctypes.c_void_p),
                ("Q", ctypes.c_void_p), ("R", ctypes.c_void_p), ("PN", ctypes.c_void_p),
                ("q", ctypes.c_void_p), ("r", ctypes.c_void_p), ("pN", ctypes.c_void_p)]


_lib_handle = None


def _lib():
    global _lib_handle
    if _lib_handle is None:
        lib = ctypes.CDLL(build_oracle())
        lib.orc_factor.restype = ctypes.c_int
        lib.orc_solve.restype = ctypes.c_int
        lib.orc_num_threads.restype = ctypes.c_int
        _lib_handle = lib
    return _lib_handle


def num_threads() -> int:
    return int(_lib().orc_num_threads())


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


class LQOracle:
    """Factor once, then evaluate x(y) (Algorithm 3) and x_lin(r) (Algorithm 4)."""

    def __init__(self, p: Problem):
        self.p = p
        t = p.tree
        self.nx, self.nu = p.nx, p.nu
        self.Nn, self.Np, self.N = t.num_nodes, t.num_nonleaf, t.horizon
        self._keep = {}
        self._keep["parent"] = np.ascontiguousarray(t.parent, dtype=np.int32)
        self._keep["cbeg"] = np.ascontiguousarray(t.child_begin, dtype=np.int32)
        self._keep["ccnt"] = np.ascontiguousarray(t.child_count, dtype=np.int32)
        soff = np.zeros(self.N + 2, dtype=np.int32)
        for s in range(self.N + 1):
            soff[s] = int(np.searchsorted(t.stage, s))
        soff[self.N + 1] = self.Nn
        self._keep["soff"] = soff
        for name in ("A", "B", "c", "Q", "R", "PN", "q", "r", "pN"):
            self._keep[name] = np.ascontiguousarray(getattr(p, name), dtype=np.float64)
        self._keep["prob"] = np.ascontiguousarray(t.prob, dtype=np.float64)
        k = self._keep
        self._cp = _OrcProblem(self.Nn, self.Np, self.N, self.nx, self.nu,
                               _ptr(k["parent"]), _ptr(k["cbeg"]), _ptr(k["ccnt"]), _ptr(k["soff"]),
                               _ptr(k["prob"]), _ptr(k["A"]), _ptr(k["B"]), _ptr(k["c"]),
                               _ptr(k["Q"]), _ptr(k["R"]), _ptr(k["PN"]),
                               _ptr(k["q"]), _ptr(k["r"]), _ptr(k["pN"]))
        nx, nu = self.nx, self.nu
        self.P = np.zeros((self.Nn, nx, nx))
        self.K = np.zeros((self.Np, nu, nx))
        self.Lc = np.zeros((self.Np, nu, nu))
        self.gu = np.zeros((self.Np, nu))
        self.gx = np.zeros((self.Np, nx))
        st = _lib().orc_factor(ctypes.byref(self._cp), _ptr(self.P), _ptr(self.K), _ptr(self.Lc),
                               _ptr(self.gu), _ptr(self.gx))
        if st != 0:
            raise np.linalg.LinAlgError(f"Rbar not positive definite at node {-st - 1}")
        self._s = np.zeros((self.Nn, nx))
        self._ubar = np.zeros((self.Np, nu))
        # the [x; u] layout of Algorithms 3 and 4, and the dual layout (the same unless the problem
        # has general constraint maps z = F x + G u, Section II-C)
        self.sel_off = dual_offsets(t, nx, nu)
        self.sel_m = int(self.sel_off[-1])
        self.general = p.general
        self.off = problem_offsets(p)
        self.m = int(self.off[-1])
        self.solve_calls = 0
        # per dual element: sqrt(pi) of its node, unscaled box (selection: root state unbounded)
        node_of = np.repeat(np.arange(self.Nn), np.diff(self.off))
        self.node_of = node_of
        self.sq = np.sqrt(t.prob[node_of])
        lo = np.empty(self.m)
        hi = np.empty(self.m)
        for i in range(self.Nn):
            o, o1 = self.off[i], self.off[i + 1]
            if self.general:
                lo[o:o1], hi[o:o1] = (p.zlo, p.zhi) if i < self.Np else (p.zNlo, p.zNhi)
                continue
            lo[o:o + nx], hi[o:o + nx] = p.xlo, p.xhi
            if i < self.Np:
                lo[o + nx:o + nx + nu], hi[o + nx:o + nx + nu] = p.ulo, p.uhi
        if not self.general:
            lo[:nx], hi[:nx] = -np.inf, np.inf
        self.lo, self.hi = lo, hi
        # the nonsmooth term per element (Section II-B): kind, rho, delta of its component
        kind, rho, dl = np.zeros(self.m, dtype=np.int32), np.zeros(self.m), np.ones(self.m)
        if p.pen_kind is not None and self.general:
            raise ValueError("soft terms are per component of [x; u]: not with general constraint maps")
        if p.pen_kind is not None:
            comp = np.empty(self.m, dtype=np.int64)
            for i in range(self.Nn):
                o = self.off[i]
                comp[o:o + nx] = np.arange(nx)
                if i < self.Np:
                    comp[o + nx:o + nx + nu] = nx + np.arange(nu)
            kind, rho, dl = p.pen_kind[comp].astype(np.int32), p.pen_rho[comp].astype(float), p.pen_delta[comp].astype(float)
            kind[:nx] = 0  # the root state is the parameter: no term
        self.kind, self.rho, self.delta = kind, rho, dl

    @property
    def Rbar(self) -> np.ndarray:
        return np.einsum("iab,icb->iac", self.Lc, self.Lc)

    def ht(self, y: np.ndarray) -> np.ndarray:
        """H'y in the [x; u] layout: per nonleaf node [F'y^i; G'y^i], per leaf FN'y^l (the
        selection: y itself)."""
        if not self.general:
            return y
        p, npl, nx = self.p, self.Np, self.nx
        nc, ncn = p.F.shape[0], p.FN.shape[0]
        Yn = y[:npl * nc].reshape(npl, nc)
        Yl = y[npl * nc:].reshape(self.Nn - npl, ncn)
        out = np.empty(self.sel_m)
        blk = out[:npl * (nx + self.nu)].reshape(npl, nx + self.nu)
        blk[:, :nx] = Yn @ p.F
        blk[:, nx:] = Yn @ p.G
        out[npl * (nx + self.nu):] = (Yl @ p.FN).reshape(-1)
        return out

    def solve(self, y: np.ndarray, homogeneous: bool = False):
        """x(y) by Algorithm 3 (or Algorithm 4 if homogeneous): the minimiser of f(x) + <y, Hx>,
        i.e. Algorithm 3 with H'y in the [x; u] layout.  y is unscaled, dual-sized."""
        y = np.ascontiguousarray(y, dtype=np.float64)
        assert y.shape == (self.m,)
        y = np.ascontiguousarray(self.ht(y))
        x = np.zeros((self.Nn, self.nx))
        u = np.zeros((self.Np, self.nu))
        x0 = np.ascontiguousarray(self.p.x0, dtype=np.float64)
        _lib().orc_solve(ctypes.byref(self._cp), _ptr(self.K), _ptr(self.Lc), _ptr(self.gu), _ptr(self.gx),
                         _ptr(y), _ptr(x0), ctypes.c_int(1 if homogeneous else 0),
                         _ptr(x), _ptr(u), _ptr(self._s), _ptr(self._ubar))
        self.solve_calls += 1
        return x, u

    def stack(self, x: np.ndarray, u: np.ndarray) -> np.ndarray:
        """Hx laid out like y: nonleaf [x^i; u^i], leaf x^l; with general constraint maps
        F x^i + G u^i and FN x^l (x[0] is the root state)."""
        npl, nx, nu = self.Np, self.nx, self.nu
        h = np.empty(self.m)
        if self.general:
            p = self.p
            nc = p.F.shape[0]
            h[:npl * nc] = (x[:npl] @ p.F.T + u @ p.G.T).reshape(-1)
            h[npl * nc:] = (x[npl:] @ p.FN.T).reshape(-1)
            return h
        h[:npl * (nx + nu)] = np.concatenate([x[:npl], u], axis=1).reshape(-1)
        h[npl * (nx + nu):] = x[npl:].reshape(-1)
        return h

    def unstack(self, h: np.ndarray):
        assert not self.general, "H is not invertible in general"
        npl, nx, nu = self.Np, self.nx, self.nu
        blk = h[:npl * (nx + nu)].reshape(npl, nx + nu)
        x = np.concatenate([blk[:, :nx], h[npl * (nx + nu):].reshape(-1, nx)], axis=0)
        return x, blk[:, nx:].copy()

    def hx(self, y: np.ndarray, homogeneous: bool = False) -> np.ndarray:
        return self.stack(*self.solve(y, homogeneous))

    def cost(self, x: np.ndarray, u: np.ndarray) -> float:
        """f(x) of eq. (f-definition) with the quadratic costs of Section II-B (no 1/2).
        The root's state term pi^0 (p'Qp + q'p) is a constant and is included."""
        p, pr = self.p, self.p.tree.prob
        npl = self.Np
        xn, xl = x[:npl], x[npl:]
        f = np.sum(pr[:npl] * (xn ** 2 @ p.Q + u ** 2 @ p.R + xn @ p.q + u @ p.r))
        f += np.sum(pr[npl:] * (xl ** 2 @ p.PN + xl @ p.pN))
        return float(f)


# --------------------------------------------------------------------------------------
# Scaled dual quantities (Sections II-D, III-A, III-E).  ybar is the scaled dual.
# --------------------------------------------------------------------------------------

def hbar(o: LQOracle, yb: np.ndarray):
    """S Hx(S ybar) and the primal (x, u)."""
    x, u = o.solve(o.sq * yb)
    return o.sq * o.stack(x, u), x, u


def hbar_lin(o: LQOracle, r: np.ndarray) -> np.ndarray:
    """S H x_lin(S r) = -grad^2 fhat(ybar) r (Algorithm 4)."""
    return o.sq * o.hx(o.sq * r, homogeneous=True)


def proj_box(o: LQOracle, v: np.ndarray) -> np.ndarray:
    """Projection on the scaled box S Y (prox of the indicator, Section II-D)."""
    return np.minimum(np.maximum(v, o.sq * o.lo), o.sq * o.hi)


def _huber(d: np.ndarray, delta: np.ndarray) -> np.ndarray:
    return np.where(d <= delta, 0.5 * d * d, delta * (d - 0.5 * delta))


def g_val(o: LQOracle, zb: np.ndarray) -> float:
    """The scaled nonsmooth term g~(zbar) = sum_k g_k(zbar_k / sqrt(pi_k)) (Section II-B):
    indicator of the box (kind 0), rho dist (kind 1), rho Huber_delta(dist) (kind 2), where
    dist is the distance of the element to [lo, hi]."""
    s = o.sq
    # distance measured on the scaled box (s lo, s hi are the exact bounds prox_g returns)
    d = (np.maximum(s * o.lo - zb, 0.0) + np.maximum(zb - s * o.hi, 0.0)) / s
    k0, k1, k2 = o.kind == 0, o.kind == 1, o.kind == 2
    if np.any(d[k0] > 0.0):
        return np.inf
    return float(np.sum(o.rho[k1] * d[k1])) + float(np.sum(o.rho[k2] * _huber(d[k2], o.delta[k2])))


def prox_g(o: LQOracle, v: np.ndarray, lam: float) -> np.ndarray:
    """z_lambda: argmin_zbar g~(zbar) + lam/2 ||zbar - v||^2, element by element.  With
    zbar = s z (s = sqrt(pi)) this is z = prox_{a g_k}(v / s), a = 1 / (lam s^2):
    kind 0: clamp to [lo, hi]; kind 1: move toward the box by at most a rho, not past it;
    kind 2: outside the box by e, e / (1 + a rho) if e <= delta (1 + a rho), else e - a rho delta
    (the proximal map of the Huber function applied to the excess)."""
    s = o.sq
    t = v / s
    a = 1.0 / (lam * s * s)
    z = np.minimum(np.maximum(t, o.lo), o.hi)
    e_up = np.where(t > o.hi, t - o.hi, 0.0)
    e_dn = np.where(t < o.lo, o.lo - t, 0.0)
    k1, k2 = o.kind == 1, o.kind == 2
    ar = a * o.rho
    z1 = np.where(t > o.hi, o.hi + np.maximum(e_up - ar, 0.0), np.where(t < o.lo, o.lo - np.maximum(e_dn - ar, 0.0), t))
    shrink = lambda e: np.where(e <= o.delta * (1.0 + ar), e / (1.0 + ar), e - ar * o.delta)
    z2 = np.where(t > o.hi, o.hi + shrink(e_up), np.where(t < o.lo, o.lo - shrink(e_dn), t))
    z = np.where(k1, z1, np.where(k2, z2, z))
    return s * z


def _sigma(lo: np.ndarray, hi: np.ndarray, y: np.ndarray) -> np.ndarray:
    """Support function of [lo, hi] per element (inf where unbounded in y's direction)."""
    out = np.zeros_like(y)
    pos, neg = y > 0, y < 0
    out[pos] = hi[pos] * y[pos]
    out[neg] = lo[neg] * y[neg]
    return out


def g_conj(o: LQOracle, v: np.ndarray) -> float:
    """Conjugate of the scaled term, g~*(v) = sum_k g_k*(s_k v_k), with
    kind 0: sigma_[lo,hi]; kind 1: sigma on |y| <= rho; kind 2: sigma + y^2 / (2 rho) on
    |y| <= rho delta (+inf off the domains)."""
    y = o.sq * v
    sig = _sigma(o.lo, o.hi, y)
    k1, k2 = o.kind == 1, o.kind == 2
    # (domains closed up to rounding: the prox puts multipliers exactly on their boundary)
    if np.any(np.abs(y[k1]) > o.rho[k1] * (1 + 1e-12)) or np.any(np.abs(y[k2]) > o.rho[k2] * o.delta[k2] * (1 + 1e-12)):
        return np.inf
    tot = sig.copy()
    tot[k2] += y[k2] ** 2 / (2.0 * o.rho[k2])
    if np.any(np.isinf(tot)):
        return np.inf
    return float(np.sum(tot))


def prox_g_conj(o: LQOracle, v: np.ndarray, lam: float) -> np.ndarray:
    """prox_{lam g*}(v) = v - lam z(v / lam) (Moreau decomposition)."""
    return v - lam * prox_g(o, v / lam, lam)


def prox_g_conj_closed(o: LQOracle, v: np.ndarray, lam: float) -> np.ndarray:
    """prox_{lam g~*}(v) from the conjugates' own closed forms: with y = s v and c = lam s^2,
    eta = argmin g_k*(eta) + (eta - y)^2 / (2 c), returned as eta / s.  Box: two-sided shrink
    (y - c hi if y > c hi, y - c lo if y < c lo, else 0); kind 1: that shrink clamped to
    [-rho, rho]; kind 2: (y - c hi) / (1 + c / rho) or (y - c lo) / (1 + c / rho) on the same
    sides, clamped to [-rho delta, rho delta]."""
    s = o.sq
    y = s * v
    c = lam * s * s
    eta = np.zeros_like(v)
    up, dn = y > c * o.hi, y < c * o.lo
    eta[up] = y[up] - c[up] * o.hi[up]
    eta[dn] = y[dn] - c[dn] * o.lo[dn]
    k1, k2 = o.kind == 1, o.kind == 2
    eta[k1] = np.clip(eta[k1], -o.rho[k1], o.rho[k1])
    e2 = eta[k2] / (1.0 + c[k2] / o.rho[k2])
    eta[k2] = np.clip(e2, -o.rho[k2] * o.delta[k2], o.rho[k2] * o.delta[k2])
    return eta / s


def fb_point(o: LQOracle, yb: np.ndarray, lam: float) -> dict:
    """Everything the algorithms need at one dual point (full solve).  The FBE is minus the
    augmented Lagrangian f(x) + g(z) + <y, Hx - z> + lam/2 ||Hx - z||^2 at z = z_lambda(y)."""
    h, x, u = hbar(o, yb)
    z = prox_g(o, h + yb / lam, lam)
    r = z - h
    f = o.cost(x, u)
    phi = -(f + g_val(o, z) + float(np.dot(yb, h - z)) + 0.5 * lam * float(np.dot(h - z, h - z)))
    return dict(y=yb, h=h, x=x, u=u, z=z, r=r, f=f, phi=phi, T=yb - lam * r,
                res_inf=float(np.max(np.abs(r / o.sq))) if r.size else 0.0)


def fhat_at(pt: dict) -> float:
    """fhat at a point returned by fb_point: -(f(x) + <ybar, Hbar x>)."""
    return -(pt["f"] + float(np.dot(pt["y"], pt["h"])))


def original_backtrack_excess(o: LQOracle, wp: dict, new: dict, lam: float, beta: float) -> float:
    """Eq. (original-backtracking) at the accepted point w (wp) and T(w) (new), literally:
    fhat(T(w)) - [fhat(w) - lam <grad fhat(w), R(w)> + (1 - beta) lam / 2 ||R(w)||^2], with
    grad fhat(w) = -Hbar x(w).  Positive means the test fails.  Evaluated from fhat values it
    is exact only far from the solution: its margin is of the order of lam ||R||^2 while the
    terms are of the order of ||R||, so near the solution rounding decides its sign."""
    grad = -wp["h"]
    rhs = fhat_at(wp) - lam * float(np.dot(grad, wp["r"])) + 0.5 * (1.0 - beta) * lam * float(np.dot(wp["r"], wp["r"]))
    return fhat_at(new) - rhs


def original_backtrack_fails(o: LQOracle, wp: dict, new: dict, lam: float, beta: float) -> bool:
    """Eq. (original-backtracking) at w, evaluated without cancellation.  fhat is quadratic, so
    fhat(T(w)) = fhat(w) + <grad fhat(w), T(w) - w> + 1/2 (T(w) - w)' grad^2 fhat (T(w) - w)
    exactly, with T(w) - w = -lam R(w); the test is therefore
    lam <R, grad^2 fhat R> > (1 - beta) ||R||^2, R = R(w), with the Hessian-vector product
    grad^2 fhat R = -Hbar x_lin(R) of Algorithm 4 (one extra homogeneous solve)."""
    R = wp["r"]
    HR = -hbar_lin(o, R)
    return lam * float(np.dot(R, HR)) > (1.0 - beta) * float(np.dot(R, R))


def simple_backtrack_fails(o: LQOracle, pt: dict, lam: float, eps: float) -> bool:
    """Eq. (simple-backtracking) at ybar (pt): lam ||grad fhat(T(ybar)) - grad fhat(ybar)||
    > eps'' ||T(ybar) - ybar||, with grad fhat(T(ybar)) from a full solve at T(ybar)."""
    hT, _, _ = hbar(o, pt["T"])
    lhs = lam * float(np.linalg.norm(-hT + pt["h"]))
    return lhs > eps * float(np.linalg.norm(pt["T"] - pt["y"]))


def fhat(o: LQOracle, yb: np.ndarray) -> float:
    """fhat(ybar) = f*(-Hbar' ybar) = -(f(x(ybar)) + <ybar, Hbar x(ybar)>)."""
    h, x, u = hbar(o, yb)
    return -(o.cost(x, u) + float(np.dot(yb, h)))


def fbe_literal(o: LQOracle, yb: np.ndarray, lam: float) -> float:
    """phi_lambda(y) = fhat(y) + g*(T(y)) - lam <grad fhat(y), R(y)> + lam/2 ||R(y)||^2 (Section III-A)."""
    pt = fb_point(o, yb, lam)
    grad = -pt["h"]
    fh = -(pt["f"] + float(np.dot(yb, pt["h"])))
    return fh + g_conj(o, pt["T"]) - lam * float(np.dot(grad, pt["r"])) + 0.5 * lam * float(np.dot(pt["r"], pt["r"]))


def fbe_grad(o: LQOracle, yb: np.ndarray, lam: float, pt: dict | None = None) -> np.ndarray:
    """grad phi = (I - lam grad^2 fhat) R = R + lam Hbar x_lin(R)."""
    if pt is None:
        pt = fb_point(o, yb, lam)
    return pt["r"] + lam * hbar_lin(o, pt["r"])


# --------------------------------------------------------------------------------------
# L-BFGS (two-loop recursion, Nocedal & Wright Alg. 7.4), FIFO memory.
# --------------------------------------------------------------------------------------

class LBFGS:
    """H0 = gamma I with gamma = <s,q>/<q,q> of the newest pair; lam I while empty."""

    def __init__(self, mem: int, lam: float):
        self.mem, self.lam = mem, lam
        self.S, self.Y = [], []

    def push(self, s: np.ndarray, q: np.ndarray):
        self.S.append(s.copy())
        self.Y.append(q.copy())
        if len(self.S) > self.mem:
            self.S.pop(0)
            self.Y.pop(0)

    def clear(self):
        self.S, self.Y = [], []

    def apply(self, g: np.ndarray) -> np.ndarray:
        """B g, with B the L-BFGS inverse-Hessian approximation."""
        if not self.S:
            return self.lam * g
        qv = g.copy()
        alphas = []
        rhos = [1.0 / float(np.dot(s, y)) for s, y in zip(self.S, self.Y)]
        for s, y, rho in zip(reversed(self.S), reversed(self.Y), reversed(rhos)):
            a = rho * float(np.dot(s, qv))
            alphas.append(a)
            qv -= a * y
        s_new, y_new = self.S[-1], self.Y[-1]
        gamma = float(np.dot(s_new, y_new)) / float(np.dot(y_new, y_new))
        rvec = gamma * qv
        for (s, y, rho), a in zip(zip(self.S, self.Y, rhos), reversed(alphas)):
            b = rho * float(np.dot(y, rvec))
            rvec += (a - b) * s
        return rvec


def power_lambda(o: LQOracle, r0: np.ndarray, iters: int = 50, safety: float = 0.9):
    """Estimate L = ||grad^2 fhat|| by power iteration on r -> -Hbar x_lin(r), lam = safety / L."""
    r = r0 / np.linalg.norm(r0)
    L = 0.0
    for _ in range(iters):
        v = -hbar_lin(o, r)
        L = float(np.dot(r, v))
        nv = np.linalg.norm(v)
        if nv == 0.0:
            break
        r = v / nv
    return safety / L, L


# --------------------------------------------------------------------------------------
# Algorithms 1 and 2, and GPAD.
# --------------------------------------------------------------------------------------

def _result(o, pt, k, hist, status, t0):
    return dict(y=o.sq * pt["y"], ybar=pt["y"], x=pt["x"], u=pt["u"], z=pt["z"] / o.sq,
                h=pt["h"] / o.sq, res_inf=pt["res_inf"], iters=k, status=status,
                solve_calls=o.solve_calls, phi=hist["phi"], tau=hist["tau"], res=hist["res"],
                lam=hist.get("lam"), halvings=hist.get("halvings", 0), seconds=time.perf_counter() - t0)


def _check_backtrack(backtrack, bt_beta, bt_eps):
    if backtrack not in (None, "original", "simple"):
        raise ValueError(f"unknown backtracking rule {backtrack!r}")
    if not 0.0 <= bt_beta < 1.0 or not 0.0 < bt_eps < 0.5:
        raise ValueError("need beta in [0, 1) and eps'' in (0, 1/2)")


def nama(o: LQOracle, lam: float, y0: np.ndarray | None = None, tol: float = 1e-8, mem: int = 5,
         max_iter: int = 1000, max_ls: int = 30, eps_curv: float = 1e-12, backtrack: str | None = None,
         bt_beta: float = 0.0, bt_eps: float = 0.25, max_halvings: int = 60) -> dict:
    """Algorithm 2 on the preconditioned dual.  y0 is unscaled.  backtrack: None (fixed lambda),
    "original" (eq. original-backtracking with beta = bt_beta) or "simple" (eq.
    simple-backtracking with eps'' = bt_eps)."""
    _check_backtrack(backtrack, bt_beta, bt_eps)
    t0 = time.perf_counter()
    o.solve_calls = 0
    yb = np.zeros(o.m) if y0 is None else np.asarray(y0, dtype=np.float64) / o.sq
    lb = LBFGS(mem, lam)
    pt = fb_point(o, yb, lam)
    hist = dict(phi=[pt["phi"]], tau=[], res=[pt["res_inf"]], lam=lam, halvings=0)

    def halve():
        nonlocal lam, pt
        lam *= 0.5
        lb.clear()
        lb.lam = lam
        hist["lam"], hist["halvings"] = lam, hist["halvings"] + 1
        pt = fb_point(o, pt["y"], lam)

    k = 0
    while pt["res_inf"] > tol:
        if k >= max_iter or hist["halvings"] > max_halvings:
            return _result(o, pt, k, hist, "not_converged", t0)
        if backtrack == "simple" and simple_backtrack_fails(o, pt, lam, bt_eps):
            halve()
            continue
        r = pt["r"]
        d = -lb.apply(r)
        fb_dir = pt["T"] - pt["y"]
        tau, wp = 1.0, None
        for _ in range(max_ls + 1):
            cand = fb_point(o, pt["y"] + tau * d + (1.0 - tau) * fb_dir, lam)
            if cand["phi"] <= pt["phi"]:
                wp = cand
                break
            tau *= 0.5
        if wp is None:
            tau, wp = 0.0, fb_point(o, pt["T"].copy(), lam)
        new = fb_point(o, wp["T"], lam)
        if backtrack == "original" and original_backtrack_fails(o, wp, new, lam, bt_beta):
            halve()
            continue
        s = new["y"] - pt["y"]
        qv = new["r"] - r
        if float(np.dot(s, qv)) > eps_curv * float(np.dot(s, s)) * float(np.dot(r, r)):
            lb.push(s, qv)
        pt = new
        k += 1
        hist["phi"].append(pt["phi"])
        hist["tau"].append(tau)
        hist["res"].append(pt["res_inf"])
    return _result(o, pt, k, hist, "converged", t0)


def minfbe(o: LQOracle, lam: float, y0: np.ndarray | None = None, tol: float = 1e-8, mem: int = 5,
           max_iter: int = 1000, max_ls: int = 30, eps_curv: float = 1e-12, backtrack: str | None = None,
           bt_beta: float = 0.0, bt_eps: float = 0.25, max_halvings: int = 60) -> dict:
    """Algorithm 1 on the preconditioned dual.  y0 is unscaled.  backtrack as for nama."""
    _check_backtrack(backtrack, bt_beta, bt_eps)
    t0 = time.perf_counter()
    o.solve_calls = 0
    yb = np.zeros(o.m) if y0 is None else np.asarray(y0, dtype=np.float64) / o.sq
    lb = LBFGS(mem, lam)
    pt = fb_point(o, yb, lam)
    g = fbe_grad(o, yb, lam, pt)
    hist = dict(phi=[pt["phi"]], tau=[], res=[pt["res_inf"]], lam=lam, halvings=0)

    def halve():
        nonlocal lam, pt, g
        lam *= 0.5
        lb.clear()
        lb.lam = lam
        hist["lam"], hist["halvings"] = lam, hist["halvings"] + 1
        pt = fb_point(o, pt["y"], lam)
        g = fbe_grad(o, pt["y"], lam, pt)

    k = 0
    while pt["res_inf"] > tol:
        if k >= max_iter or hist["halvings"] > max_halvings:
            return _result(o, pt, k, hist, "not_converged", t0)
        if backtrack == "simple" and simple_backtrack_fails(o, pt, lam, bt_eps):
            halve()
            continue
        d = -lb.apply(g)
        tau, wp = 1.0, None
        for _ in range(max_ls + 1):
            cand = fb_point(o, pt["y"] + tau * d, lam)
            if cand["phi"] <= pt["phi"]:
                wp = cand
                break
            tau *= 0.5
        if wp is None:
            tau, wp = 0.0, pt
        new = fb_point(o, wp["T"], lam)
        if backtrack == "original" and original_backtrack_fails(o, wp, new, lam, bt_beta):
            halve()
            continue
        g_new = fbe_grad(o, new["y"], lam, new)
        s = new["y"] - pt["y"]
        qv = g_new - g
        if float(np.dot(s, qv)) > eps_curv * float(np.dot(s, s)) * float(np.dot(g, g)):
            lb.push(s, qv)
        pt, g = new, g_new
        k += 1
        hist["phi"].append(pt["phi"])
        hist["tau"].append(tau)
        hist["res"].append(pt["res_inf"])
    return _result(o, pt, k, hist, "converged", t0)


def gpad_theta(k: int) -> float:
    """theta_k of the accelerated dual gradient projection: theta_{-1} = theta_0 = 1,
    theta_{k+1} = (sqrt(theta_k^4 + 4 theta_k^2) - theta_k^2) / 2."""
    th = 1.0
    for _ in range(max(0, k)):
        th = 0.5 * (np.sqrt(th ** 4 + 4.0 * th * th) - th * th)
    return th


def gpad(o: LQOracle, lam: float, y0: np.ndarray | None = None, tol: float = 1e-8,
         max_iter: int = 1000) -> dict:
    """GPAD on the preconditioned dual (the warm start of Section III-E and the comparison
    method of Section IV).  y0 is unscaled.

    Iteration k at the extrapolated point w_k = ybar_k + theta_k (1/theta_{k-1} - 1)
    (ybar_k - ybar_{k-1}) (w_0 = ybar_0): one full solve x(w_k), the stopping test
    ||z(w_k) - Hx(w_k)||_inf <= tol (unscaled), then ybar_{k+1} = T_lambda(w_k).  The result
    is the point of the last stopping test, w_k, with x(w_k) and z(w_k); `iters` counts the
    forward-backward steps taken before it."""
    t0 = time.perf_counter()
    o.solve_calls = 0
    yb = np.zeros(o.m) if y0 is None else np.asarray(y0, dtype=np.float64) / o.sq
    y_prev = yb.copy()
    th_prev, th = 1.0, 1.0
    hist = dict(phi=[], tau=[], res=[])
    k = 0
    while True:
        w = yb + th * (1.0 / th_prev - 1.0) * (yb - y_prev)
        pt = fb_point(o, w, lam)
        hist["phi"].append(pt["phi"])
        hist["res"].append(pt["res_inf"])
        if pt["res_inf"] <= tol:
            return _result(o, pt, k, hist, "converged", t0)
        if k >= max_iter:
            return _result(o, pt, k, hist, "not_converged", t0)
        y_prev, yb = yb, pt["T"]
        th_prev, th = th, 0.5 * (np.sqrt(th ** 4 + 4.0 * th * th) - th * th)
        k += 1
