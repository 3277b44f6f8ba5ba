"""Seeded synthetic scenario trees and problem data.

This module only draws inputs: tree shapes, probabilities, dynamics, costs,
boxes and initial states.  It holds none of the method's arithmetic (no
factorisation, no solve, no prox), so both the CPU oracle and the CUDA path
can take their inputs from it.

Tree conventions (Section II-A, scenario trees):
  * nodes are numbered stage by stage (breadth first), the root is node 0;
  * the children of a node occupy a contiguous index range;
  * every leaf sits at stage N, so nodes 0..Np-1 are the non-leaf nodes and
    Np..Nn-1 the leaves;
  * node probabilities satisfy pi^0 = 1, sum over a stage = 1 and
    sum over child(i) = pi^i.

Problem data (Section II-B/C, eq. system_dynamics_tree and the quadratic
stage cost): per node j >= 1 the edge data A^j (nx x nx), B^j (nx x nu) and
c^j (nx) lives on the child; the costs Q, R, P_N are diagonal and shared by
all nodes, the linear terms q, r, p_N are shared vectors, and the box
constraints on x and u are shared vectors.
"""
from __future__ import annotations

import dataclasses
import json
import os
from dataclasses import dataclass, field

import numpy as np

_DATA_DIR = os.path.join(os.path.dirname(os.path.abspath(__file__)), "data")


@dataclass
class Tree:
    horizon: int
    parent: np.ndarray      # int32 [Nn], parent[0] = -1
    stage: np.ndarray       # int32 [Nn]
    prob: np.ndarray        # float64 [Nn]
    child_begin: np.ndarray  # int32 [Nn]
    child_count: np.ndarray  # int32 [Nn]

    @property
    def num_nodes(self) -> int:
        return int(self.parent.shape[0])

    @property
    def num_nonleaf(self) -> int:
        return int(np.count_nonzero(self.child_count > 0))

    @property
    def num_leaves(self) -> int:
        return self.num_nodes - self.num_nonleaf

    def stage_nodes(self, t: int) -> np.ndarray:
        return np.nonzero(self.stage == t)[0]

    def stage_ranges(self):
        """(first, count) of every stage; stages are contiguous by construction."""
        out = []
        for t in range(self.horizon + 1):
            idx = self.stage_nodes(t)
            out.append((int(idx[0]), int(idx.size)))
        return out


def tree_from_branching(branching, cond_probs=None) -> Tree:
    """Build a tree from a per-node child count.

    ``branching`` is either a list with one entry per stage 0..N-1 (every node
    of that stage gets that many children) or a list of per-stage lists with
    one child count per node of the stage (ragged trees).  ``cond_probs``
    optionally gives, per non-leaf node in index order, the conditional
    probabilities pi^[i] of its children; the default is uniform.
    """
    parent = [-1]
    stage = [0]
    prob = [1.0]
    frontier = [0]
    child_begin = {}
    child_count = {}
    t = 0
    cp_iter = iter(cond_probs) if cond_probs is not None else None
    for spec in branching:
        nxt = []
        counts = spec if isinstance(spec, (list, tuple, np.ndarray)) else [spec] * len(frontier)
        if len(counts) != len(frontier):
            raise ValueError("per-stage branching list has the wrong length")
        for node, b in zip(frontier, counts):
            b = int(b)
            if b < 1:
                raise ValueError("every non-leaf node needs at least one child")
            child_begin[node] = len(parent)
            child_count[node] = b
            w = np.full(b, 1.0 / b) if cp_iter is None else np.asarray(next(cp_iter), dtype=np.float64)
            for k in range(b):
                parent.append(node)
                stage.append(t + 1)
                prob.append(prob[node] * float(w[k]))
                nxt.append(len(parent) - 1)
        frontier = nxt
        t += 1
    nn = len(parent)
    cb = np.array([child_begin.get(i, 0) for i in range(nn)], dtype=np.int32)
    cc = np.array([child_count.get(i, 0) for i in range(nn)], dtype=np.int32)
    return Tree(horizon=t, parent=np.array(parent, dtype=np.int32),
                stage=np.array(stage, dtype=np.int32), prob=np.array(prob, dtype=np.float64),
                child_begin=cb, child_count=cc)


def random_tree(rng: np.random.Generator, horizon: int, max_branch: int = 3,
                p_branch: float = 0.6, random_probs: bool = True) -> Tree:
    """Ragged tree: each node of each stage draws 1..max_branch children."""
    counts_per_stage = []
    width = 1
    for _ in range(horizon):
        counts = [int(rng.integers(1, max_branch + 1)) if rng.random() < p_branch else 1
                  for _ in range(width)]
        counts_per_stage.append(counts)
        width = sum(counts)
    cond = None
    if random_probs:
        cond = []
        for counts in counts_per_stage:
            for b in counts:
                w = rng.uniform(0.2, 1.0, size=b)
                cond.append(w / w.sum())
    return tree_from_branching(counts_per_stage, cond)


@dataclass
class Problem:
    """One scenario-tree LQ problem with box constraints (FP64 host arrays)."""
    tree: Tree
    nx: int
    nu: int
    A: np.ndarray       # [Nn, nx, nx]; row 0 unused (zeros)
    B: np.ndarray       # [Nn, nx, nu]
    c: np.ndarray       # [Nn, nx]
    Q: np.ndarray       # [nx] diagonal
    R: np.ndarray       # [nu] diagonal
    PN: np.ndarray      # [nx] diagonal
    q: np.ndarray       # [nx]
    r: np.ndarray       # [nu]
    pN: np.ndarray      # [nx]
    xlo: np.ndarray     # [nx]
    xhi: np.ndarray     # [nx]
    ulo: np.ndarray     # [nu]
    uhi: np.ndarray     # [nu]
    x0: np.ndarray      # [nx]
    name: str = "problem"
    meta: dict = field(default_factory=dict)
    # Nonsmooth term g per component of [x; u] (Section II-B): kind 0 = indicator of the box
    # [lo, hi] (hard constraint); 1 = rho * distance to the box (soft constraint; lo = hi = c
    # gives rho |z - c|); 2 = rho * Huber_delta(distance to the box).  None = all kind 0.
    pen_kind: np.ndarray | None = None   # [nx + nu] int
    pen_rho: np.ndarray | None = None    # [nx + nu]
    pen_delta: np.ndarray | None = None  # [nx + nu]
    # General constraint maps (Section II-C): z^i = F x^i + G u^i at every nonleaf node (the root
    # included, with x^0 = x0) and z^l = FN x^l at every leaf, shared by all nodes, with the box
    # zlo <= z <= zhi (zNlo, zNhi at the leaves).  None: the selection z^i = [x^i; u^i], z^l = x^l
    # with the x and u boxes above (the root's state unboxed).
    F: np.ndarray | None = None      # [nc, nx]
    G: np.ndarray | None = None      # [nc, nu]
    FN: np.ndarray | None = None     # [ncN, nx]
    zlo: np.ndarray | None = None    # [nc]
    zhi: np.ndarray | None = None
    zNlo: np.ndarray | None = None   # [ncN]
    zNhi: np.ndarray | None = None

    @property
    def general(self) -> bool:
        return self.F is not None

    @property
    def num_dual(self) -> int:
        t = self.tree
        if self.general:
            return t.num_nonleaf * self.F.shape[0] + t.num_leaves * self.FN.shape[0]
        return t.num_nonleaf * (self.nx + self.nu) + t.num_leaves * self.nx

    @property
    def num_primal(self) -> int:
        t = self.tree
        return t.num_nonleaf * self.nu + (t.num_nodes - 1) * self.nx


def problem_offsets(p: "Problem") -> np.ndarray:
    """Start of node i's block in p's dual vector: [x; u] / x (selection) or z = F x + G u / FN x."""
    if p.general:
        return block_offsets(p.tree, p.F.shape[0], p.FN.shape[0])
    return dual_offsets(p.tree, p.nx, p.nu)


def block_offsets(tree: Tree, nb: int, nbl: int) -> np.ndarray:
    """Start of node i's block when nonleaf blocks have nb entries and leaf blocks nbl."""
    nn, npl = tree.num_nodes, tree.num_nonleaf
    off = np.empty(nn + 1, dtype=np.int64)
    idx = np.arange(nn, dtype=np.int64)
    off[:nn] = np.where(idx < npl, idx * nb, npl * nb + (idx - npl) * nbl)
    off[nn] = npl * nb + (nn - npl) * nbl
    return off


def dual_offsets(tree: Tree, nx: int, nu: int) -> np.ndarray:
    """Start of node i's block in a dual-sized vector: nonleaf [x; u], leaf [x]."""
    nn, npl = tree.num_nodes, tree.num_nonleaf
    off = np.empty(nn + 1, dtype=np.int64)
    idx = np.arange(nn, dtype=np.int64)
    off[:nn] = np.where(idx < npl, idx * (nx + nu), npl * (nx + nu) + (idx - npl) * nx)
    off[nn] = npl * (nx + nu) + (nn - npl) * nx
    return off


def spectral_rescale(M: np.ndarray, rho: float) -> np.ndarray:
    ev = np.linalg.eigvals(M)
    return M * (rho / np.max(np.abs(ev)))


# --------------------------------------------------------------------------------------
# Workload recipes.  Draw order per recipe: A, per-node perturbations, B, Q, w (= c), x0.
# --------------------------------------------------------------------------------------

def tiny_fp64(seed: int = 0) -> Problem:
    """Horizon 3, binary tree (15 nodes), nx=4, nu=2, shared A (rho 0.95) and B."""
    rng = np.random.default_rng(seed)
    nx, nu = 4, 2
    tree = tree_from_branching([2, 2, 2])
    nn = tree.num_nodes
    A0 = spectral_rescale(rng.standard_normal((nx, nx)), 0.95)
    B0 = rng.standard_normal((nx, nu))
    A = np.broadcast_to(A0, (nn, nx, nx)).copy()
    B = np.broadcast_to(B0, (nn, nx, nu)).copy()
    c = 0.1 * rng.standard_normal((nn, nx))
    A[0] = 0.0
    B[0] = 0.0
    c[0] = 0.0
    x0 = rng.uniform(-3.0, 3.0, size=nx)
    return Problem(tree=tree, nx=nx, nu=nu, A=A, B=B, c=c,
                   Q=np.ones(nx), R=0.1 * np.ones(nu), PN=np.ones(nx),
                   q=np.zeros(nx), r=np.zeros(nu), pN=np.zeros(nx),
                   xlo=-5.0 * np.ones(nx), xhi=5.0 * np.ones(nx),
                   ulo=-np.ones(nu), uhi=np.ones(nu), x0=x0, name="tiny_fp64")


def paper_scale_tree() -> Tree:
    """Horizon 20: binary for the first 10 stages, then one child (1024 scenarios)."""
    return tree_from_branching([2] * 10 + [1] * 10)


def paper_scale_unboxed(seed: int = 2, nx: int = 100, nu: int = 50, tree: Tree | None = None) -> Problem:
    """Paper-scale instance before its box is set: per-node A_j = A + 0.05 N(0,1),
    A at spectral radius 0.98, B_j ~ N(0, 1/nx), w ~ N(0, 0.05^2), Q = diag(U[0.5, 2]),
    R = 0.1 I, P_N = I, x0 ~ U[-3, 3].  Boxes are infinite here."""
    rng = np.random.default_rng(seed)
    tree = paper_scale_tree() if tree is None else tree
    nn = tree.num_nodes
    A0 = spectral_rescale(rng.standard_normal((nx, nx)), 0.98)
    A = np.empty((nn, nx, nx))
    A[0] = 0.0
    A[1:] = A0[None] + 0.05 * rng.standard_normal((nn - 1, nx, nx))
    B = np.empty((nn, nx, nu))
    B[0] = 0.0
    B[1:] = rng.standard_normal((nn - 1, nx, nu)) * (1.0 / np.sqrt(nx))
    Qd = rng.uniform(0.5, 2.0, size=nx)
    c = np.empty((nn, nx))
    c[0] = 0.0
    c[1:] = 0.05 * rng.standard_normal((nn - 1, nx))
    x0 = rng.uniform(-3.0, 3.0, size=nx)
    inf = np.inf
    return Problem(tree=tree, nx=nx, nu=nu, A=A, B=B, c=c,
                   Q=Qd, R=0.1 * np.ones(nu), PN=np.ones(nx),
                   q=np.zeros(nx), r=np.zeros(nu), pN=np.zeros(nx),
                   xlo=-inf * np.ones(nx), xhi=inf * np.ones(nx),
                   ulo=-inf * np.ones(nu), uhi=inf * np.ones(nu), x0=x0, name="paper_scale")


def load_box(name: str):
    path = os.path.join(_DATA_DIR, "boxes.json")
    with open(path) as f:
        boxes = json.load(f)
    if name not in boxes:
        raise KeyError(f"no stored box for workload {name!r}; run oracle/make_boxes.py")
    b = boxes[name]
    umax = np.asarray(b["umax"], dtype=np.float64)
    xmax = np.full(LARGEST_SHAPE["nx"] if b["xmax"] is None else len(b["xmax"]), np.inf) if b["xmax"] is None \
        else np.asarray(b["xmax"], dtype=np.float64)
    return xmax, umax


def with_penalty(p: Problem, kind, rho, delta=None) -> Problem:
    """Set the per-component kinds of g (see Problem); rho, delta broadcast to nx + nu."""
    n = p.nx + p.nu
    p.pen_kind = np.broadcast_to(np.asarray(kind, dtype=np.int32), (n,)).copy()
    p.pen_rho = np.broadcast_to(np.asarray(rho, dtype=np.float64), (n,)).copy()
    p.pen_delta = np.broadcast_to(np.asarray(1.0 if delta is None else delta, dtype=np.float64), (n,)).copy()
    return p


def with_box(p: Problem, xmax: np.ndarray, umax: np.ndarray) -> Problem:
    p.xlo, p.xhi = -np.asarray(xmax, dtype=np.float64), np.asarray(xmax, dtype=np.float64)
    p.ulo, p.uhi = -np.asarray(umax, dtype=np.float64), np.asarray(umax, dtype=np.float64)
    return p


def paper_scale(seed: int = 2) -> Problem:
    """The paper-scale instance (N=20, 1024 scenarios, nx=100, nu=50) with its stored box:
    per component 80 % of the largest |x_k| (|u_k|) of the unconstrained solution x(0),
    but not below the unconstrained values of the first two stages (see oracle/make_boxes.py)."""
    p = paper_scale_unboxed(seed)
    xmax, umax = load_box("paper_scale")
    p.name = "paper_scale"
    return with_box(p, xmax, umax)


def random_problem(seed: int, horizon: int = 3, nx: int = 3, nu: int = 2, max_branch: int = 3,
                   box_scale: float = 1.0, linear_terms: bool = True, p_branch: float = 0.6,
                   tree: Tree | None = None) -> Problem:
    """Small ragged problem with per-node dynamics, for parity cases and pins.  With `tree`
    given, that tree is used and no tree is drawn (horizon, max_branch, p_branch unused)."""
    rng = np.random.default_rng(seed)
    if tree is None:
        tree = random_tree(rng, horizon, max_branch=max_branch, p_branch=p_branch)
    nn = tree.num_nodes
    A0 = spectral_rescale(rng.standard_normal((nx, nx)), 0.95)
    A = np.empty((nn, nx, nx))
    A[0] = 0.0
    A[1:] = A0[None] + 0.1 * rng.standard_normal((nn - 1, nx, nx))
    B = np.empty((nn, nx, nu))
    B[0] = 0.0
    B[1:] = rng.standard_normal((nn - 1, nx, nu))
    c = np.empty((nn, nx))
    c[0] = 0.0
    c[1:] = 0.1 * rng.standard_normal((nn - 1, nx))
    Qd = rng.uniform(0.5, 2.0, size=nx)
    Rd = rng.uniform(0.05, 0.5, size=nu)
    PNd = rng.uniform(0.5, 2.0, size=nx)
    if linear_terms:
        q, r, pN = (0.1 * rng.standard_normal(nx), 0.1 * rng.standard_normal(nu),
                    0.1 * rng.standard_normal(nx))
    else:
        q, r, pN = np.zeros(nx), np.zeros(nu), np.zeros(nx)
    x0 = rng.uniform(-3.0, 3.0, size=nx)
    xmax = box_scale * rng.uniform(1.0, 3.0, size=nx)
    umax = box_scale * rng.uniform(0.3, 1.0, size=nu)
    return Problem(tree=tree, nx=nx, nu=nu, A=A, B=B, c=c, Q=Qd, R=Rd, PN=PNd, q=q, r=r, pN=pN,
                   xlo=-xmax, xhi=xmax, ulo=-umax, uhi=umax, x0=x0, name=f"random{seed}")


def random_dual(p: Problem, seed: int, scale: float = 1.0) -> np.ndarray:
    """A seeded dual vector (unscaled), zero on the root's state block (selection constraints:
    the root's state is the parameter and carries no constraint)."""
    rng = np.random.default_rng(seed)
    y = scale * rng.standard_normal(p.num_dual)
    if not p.general:
        y[:p.nx] = 0.0
    return y


def with_constraints(p: Problem, F, G, FN, zlo, zhi, zNlo, zNhi) -> Problem:
    """Set general constraint maps and their boxes (see Problem)."""
    p.F, p.G, p.FN = (np.ascontiguousarray(a, dtype=np.float64) for a in (F, G, FN))
    p.zlo, p.zhi, p.zNlo, p.zNhi = (np.ascontiguousarray(a, dtype=np.float64) for a in (zlo, zhi, zNlo, zNhi))
    return p


def constrained_problem(seed: int, horizon: int = 3, nx: int = 3, nu: int = 2, nc: int = 4, ncN: int = 2,
                        max_branch: int = 3, p_branch: float = 0.6, tree: Tree | None = None) -> Problem:
    """A random problem of random_problem's recipe with general constraint maps: F ~ N(0,1) [nc, nx],
    G ~ N(0,1) [nc, nu], FN ~ N(0,1) [ncN, nx] (draw order after the problem's own draws: F, G, FN),
    boxes left unbounded (+-inf); the caller sets them (e.g. from the unconstrained solution)."""
    p = random_problem(seed, horizon=horizon, nx=nx, nu=nu, max_branch=max_branch, p_branch=p_branch,
                       box_scale=1e6, tree=tree)
    rng = np.random.default_rng([seed, 7])
    F = rng.standard_normal((nc, nx))
    G = rng.standard_normal((nc, nu))
    FN = rng.standard_normal((ncN, nx))
    inf = np.inf
    return with_constraints(p, F, G, FN, -inf * np.ones(nc), inf * np.ones(nc), -inf * np.ones(ncN),
                            inf * np.ones(ncN))


# --------------------------------------------------------------------------------------
# Batched uneven instances: shape groups that share the tree, A, B, costs and box, and
# instances that draw their own x0 and disturbances.
# --------------------------------------------------------------------------------------

@dataclass
class Group:
    """One shape group: a tree with `branching` children per node for the first
    `branch_stages` stages and one child after that, shared A, B, Q, R, P_N and box."""
    horizon: int
    branching: int
    branch_stages: int
    nx: int
    nu: int
    A: np.ndarray          # [nx, nx]
    B: np.ndarray          # [nx, nu]
    Q: np.ndarray
    R: np.ndarray
    PN: np.ndarray
    xlo: np.ndarray
    xhi: np.ndarray
    ulo: np.ndarray
    uhi: np.ndarray
    x0: np.ndarray         # [I, nx]
    c: np.ndarray          # [I, Nn, nx]; c[:, 0] unused

    @property
    def num_instances(self) -> int:
        return int(self.x0.shape[0])

    def tree(self) -> Tree:
        return tree_from_branching([self.branching] * self.branch_stages + [1] * (self.horizon - self.branch_stages))

    def instance(self, k: int) -> Problem:
        """Instance k as a stand-alone problem (per-node copies of the shared data)."""
        t = self.tree()
        nn = t.num_nodes
        A = np.broadcast_to(self.A, (nn, self.nx, self.nx)).copy()
        B = np.broadcast_to(self.B, (nn, self.nx, self.nu)).copy()
        A[0] = 0.0
        B[0] = 0.0
        return Problem(tree=t, nx=self.nx, nu=self.nu, A=A, B=B, c=self.c[k].copy(), Q=self.Q, R=self.R,
                       PN=self.PN, q=np.zeros(self.nx), r=np.zeros(self.nu), pN=np.zeros(self.nx),
                       xlo=self.xlo, xhi=self.xhi, ulo=self.ulo, uhi=self.uhi, x0=self.x0[k].copy(),
                       name=f"group_instance{k}")


# (branching, branch stages) pairs with b^s in [64, 1024]: the reading of "branching 2 or 3 for
# the first U{3..8} stages (64-1024 scenarios)" (other draws are redrawn).
_BATCH_SHAPES = [(2, 6), (2, 7), (2, 8), (3, 4), (3, 5), (3, 6)]


def make_group(rng: np.random.Generator, horizon: int, branching: int, branch_stages: int, nx: int, nu: int,
               instances: int, w_std: float = 0.05) -> Group:
    """A group with the tiny workload's costs and box: A Gaussian at spectral radius 0.95,
    B ~ N(0,1), Q = I, R = 0.1 I, P_N = I, |u| <= 1, |x| <= 5; per instance x0 ~ U[-3, 3] and
    c ~ N(0, w_std^2) per node.  Draw order: A, B, x0, c."""
    A = spectral_rescale(rng.standard_normal((nx, nx)), 0.95)
    B = rng.standard_normal((nx, nu))
    nn = tree_from_branching([branching] * branch_stages + [1] * (horizon - branch_stages)).num_nodes
    x0 = rng.uniform(-3.0, 3.0, size=(instances, nx))
    c = w_std * rng.standard_normal((instances, nn, nx))
    c[:, 0] = 0.0
    return Group(horizon=horizon, branching=branching, branch_stages=branch_stages, nx=nx, nu=nu, A=A, B=B,
                 Q=np.ones(nx), R=0.1 * np.ones(nu), PN=np.ones(nx),
                 xlo=-5.0 * np.ones(nx), xhi=5.0 * np.ones(nx), ulo=-np.ones(nu), uhi=np.ones(nu),
                 x0=x0, c=c)


def batched_uneven(seed: int = 3, groups: int = 16, instances: int = 32):
    """The batched workload: `groups` shape groups x `instances` instances (512 in total by
    default).  Each group draws horizon U{10..30}, (branching, branching stages) from the pairs
    with 64..1024 scenarios, nx from {16, 32, 64} and nu = nx / 2."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(groups):
        horizon = int(rng.integers(10, 31))
        b, s = _BATCH_SHAPES[int(rng.integers(0, len(_BATCH_SHAPES)))]
        nx = int(rng.choice([16, 32, 64]))
        out.append(make_group(rng, horizon, b, s, nx, nx // 2, instances))
    return out


def batched_small(seed: int = 30, instances: int = 3):
    """Small batched case for parity tests: three groups of different shapes."""
    rng = np.random.default_rng(seed)
    return [make_group(rng, 4, 2, 2, 3, 2, instances), make_group(rng, 6, 3, 1, 4, 2, instances),
            make_group(rng, 3, 2, 3, 5, 3, instances)]


# Warm-start workload: horizon 15, branching 4 for the first 4 stages (256 scenarios, 3157 nodes),
# nx = 20, nu = 10, the tiny workload's recipe for A, B and the costs.  The input box is
# |u| <= 0.3 (|x| <= 5 as in the tiny workload): with |u| <= 1 the box almost never binds at
# this size (B ~ N(0,1) with 10 inputs), NAMA stops after 0-2 iterations and there is nothing
# for a warm start to save.
WARM_SHAPE = dict(horizon=15, branching=4, branch_stages=4, nx=20, nu=10)
WARM_UMAX = 0.3
WARM_TRAIN_SEED = 40000
WARM_EVAL_SEED = 90000


def warm_start_system(seed: int = 4) -> Group:
    """Shared data of the warm-start workload (no instances yet).  Draw order: A, B."""
    rng = np.random.default_rng(seed)
    nx, nu = WARM_SHAPE["nx"], WARM_SHAPE["nu"]
    A = spectral_rescale(rng.standard_normal((nx, nx)), 0.95)
    B = rng.standard_normal((nx, nu))
    nn = tree_from_branching([WARM_SHAPE["branching"]] * WARM_SHAPE["branch_stages"] +
                             [1] * (WARM_SHAPE["horizon"] - WARM_SHAPE["branch_stages"])).num_nodes
    return Group(horizon=WARM_SHAPE["horizon"], branching=WARM_SHAPE["branching"],
                 branch_stages=WARM_SHAPE["branch_stages"], nx=nx, nu=nu, A=A, B=B,
                 Q=np.ones(nx), R=0.1 * np.ones(nu), PN=np.ones(nx),
                 xlo=-5.0 * np.ones(nx), xhi=5.0 * np.ones(nx), ulo=-WARM_UMAX * np.ones(nu),
                 uhi=WARM_UMAX * np.ones(nu), x0=np.zeros((0, nx)), c=np.zeros((0, nn, nx)))


def warm_start_draws(system: Group, first_seed: int, count: int, dtype=np.float64) -> Group:
    """`count` draws of the warm-start workload; draw k uses its own generator seeded
    first_seed + k (x0 ~ U[-3, 3], then c ~ N(0, 0.1^2) per node, c[0] = 0), so any single
    draw can be regenerated on its own."""
    from concurrent.futures import ThreadPoolExecutor
    nx = system.nx
    nn = system.c.shape[1]
    x0 = np.empty((count, nx), dtype=dtype)
    c = np.empty((count, nn, nx), dtype=dtype)

    def one(k):
        r = np.random.default_rng(first_seed + k)
        x0[k] = r.uniform(-3.0, 3.0, size=nx)
        c[k] = 0.1 * r.standard_normal((nn, nx))
        c[k, 0] = 0.0

    with ThreadPoolExecutor(min(16, os.cpu_count() or 1)) as ex:
        list(ex.map(one, range(count)))
    return dataclasses.replace(system, x0=x0, c=c)


# Largest single instance: horizon 24, binary for 12 stages then one child (4096 scenarios,
# 57,343 nodes), nx = 200, nu = 100 (16.8 M primal and dual variables).  Its per-node data would
# take 27.5 GB of FP64 host memory, so it is generated block by block on demand: node block b
# (512 nodes) comes from its own generator seeded (seed, b) and is identical however it is
# requested.
LARGEST_SHAPE = dict(horizon=24, branching=2, branch_stages=12, nx=200, nu=100)
LARGE_BLOCK = 512


class NodeBlocks:
    """Per-node A_j = A + pert N(0,1), B_j = N(0,1) / sqrt(nx), c_j = w_std N(0,1) (node 0: zeros),
    generated in blocks of LARGE_BLOCK nodes.  Draw order inside a block: A perturbations, B, c."""

    def __init__(self, seed: int, num_nodes: int, nx: int, nu: int, A0: np.ndarray, pert: float, w_std: float):
        self.seed, self.nn, self.nx, self.nu = seed, num_nodes, nx, nu
        self.A0, self.pert, self.w_std = A0, pert, w_std
        self._cache = {}

    def block(self, b: int):
        if b not in self._cache:
            f = b * LARGE_BLOCK
            n = min(LARGE_BLOCK, self.nn - f)
            r = np.random.default_rng([self.seed, b])
            A = self.A0[None] + self.pert * r.standard_normal((n, self.nx, self.nx))
            B = r.standard_normal((n, self.nx, self.nu)) * (1.0 / np.sqrt(self.nx))
            c = self.w_std * r.standard_normal((n, self.nx))
            if f == 0:
                A[0], B[0], c[0] = 0.0, 0.0, 0.0
            if len(self._cache) >= 8:
                self._cache.pop(next(iter(self._cache)))
            self._cache[b] = (A, B, c)
        return self._cache[b]

    def prefetch(self, first: int, stop: int):
        """Generate the blocks covering nodes [first, stop) in parallel (the generator releases the GIL)."""
        from concurrent.futures import ThreadPoolExecutor
        bs = [b for b in range(first // LARGE_BLOCK, (stop - 1) // LARGE_BLOCK + 1) if b not in self._cache]
        if len(bs) > 1:
            with ThreadPoolExecutor(min(8, len(bs))) as ex:
                out = list(ex.map(lambda b: (b, NodeBlocks.block(self, b)), bs))
            for b, v in out:
                self._cache[b] = v

    def rows(self, field: int, first: int, stop: int) -> np.ndarray:
        self.prefetch(first, stop)
        parts = []
        n = first
        while n < stop:
            b = n // LARGE_BLOCK
            lo = n - b * LARGE_BLOCK
            hi = min(stop - b * LARGE_BLOCK, LARGE_BLOCK)
            parts.append(self.block(b)[field][lo:hi])
            n = b * LARGE_BLOCK + hi
        return np.concatenate(parts, axis=0)


class NodeArray:
    """Sliceable view of one field (0: A, 1: B, 2: c) of NodeBlocks: x[f:s] generates on demand."""

    def __init__(self, blocks: NodeBlocks, field: int, shape):
        self.blocks, self.field, self.shape = blocks, field, shape

    def __len__(self):
        return self.shape[0]

    def __getitem__(self, key):
        if isinstance(key, slice):
            first, stop, step = key.indices(self.shape[0])
            assert step == 1
            return self.blocks.rows(self.field, first, stop)
        return self.blocks.rows(self.field, int(key), int(key) + 1)[0]


def largest_tree(horizon: int = LARGEST_SHAPE["horizon"], branch_stages: int = LARGEST_SHAPE["branch_stages"]) -> Tree:
    return tree_from_branching([LARGEST_SHAPE["branching"]] * branch_stages + [1] * (horizon - branch_stages))


def largest_unboxed(seed: int = 5, tree: Tree | None = None) -> Problem:
    """The largest instance before its box: A at spectral radius 0.98 with per-node perturbation
    0.02 N(0,1), B ~ N(0, 1/nx), w ~ N(0, 0.05^2), Q = I, R = 0.1 I, P_N = I, x0 ~ U[-3, 3].
    Draw order of the shared data: A, x0."""
    nx, nu = LARGEST_SHAPE["nx"], LARGEST_SHAPE["nu"]
    rng = np.random.default_rng(seed)
    A0 = spectral_rescale(rng.standard_normal((nx, nx)), 0.98)
    x0 = rng.uniform(-3.0, 3.0, size=nx)
    tree = largest_tree() if tree is None else tree
    nn = tree.num_nodes
    blocks = NodeBlocks(seed, nn, nx, nu, A0, 0.02, 0.05)
    inf = np.inf
    return Problem(tree=tree, nx=nx, nu=nu, A=NodeArray(blocks, 0, (nn, nx, nx)), B=NodeArray(blocks, 1, (nn, nx, nu)),
                   c=NodeArray(blocks, 2, (nn, nx)), Q=np.ones(nx), R=0.1 * np.ones(nu), PN=np.ones(nx),
                   q=np.zeros(nx), r=np.zeros(nu), pN=np.zeros(nx),
                   xlo=-inf * np.ones(nx), xhi=inf * np.ones(nx), ulo=-inf * np.ones(nu), uhi=inf * np.ones(nu),
                   x0=x0, name="largest")


def largest(seed: int = 5) -> Problem:
    """The largest instance with its stored input box (states unbounded, see oracle/make_boxes.py)."""
    p = largest_unboxed(seed)
    xmax, umax = load_box("largest")
    return with_box(p, xmax, umax)


def largest_truncated(seed: int = 5, horizon: int = 14) -> Problem:
    """The largest instance's recipe cut at a smaller horizon: the same generator, sizes, box and
    binary stages (the first `horizon` stages of the tree), small enough for an FP64 host solve.
    Node data comes in the same seeded 512-node blocks, so every full block equals the full
    instance's; the last, partial block is drawn for its own size."""
    p = largest_unboxed(seed, tree=largest_tree(horizon=horizon,
                                                branch_stages=min(horizon, LARGEST_SHAPE["branch_stages"])))
    xmax, umax = load_box("largest")
    p = with_box(p, xmax, umax)
    p.name = f"largest_h{horizon}"
    return p


# ------------------------------------------------------------------------------------------
# Spring-mass-damper array (Section IV-A): M = 5 masses of 5 kg between two walls, M + 1
# springs (1 N/m) and dampers (0.1 Ns/m), M - 1 actuators between neighbouring masses,
# zero-order hold at T_s = 0.5 s; a two-mode Markov disturbance (c = 0 in mode 1, c = 0.1 in
# mode 2) over a horizon of 11 stages.
# ------------------------------------------------------------------------------------------

SPRING_MASS = dict(masses=5, mass=5.0, k_s=1.0, b_d=0.1, u_max=2.0, v_max=5.0, p_max=5.0, Ts=0.5, horizon=11,
                   p_c=(0.5, 0.5), P_c=((0.1, 0.9), (0.9, 0.1)), c_mode=(0.0, 0.1), Q=5.0, R=2.0, QN=100.0)


def spring_mass_continuous(masses: int = 5, mass: float = 5.0, k_s: float = 1.0, b_d: float = 0.1):
    """Newton's second law for the array, state x = (p_1..p_M, v_1..v_M), input u_j = force of
    the actuator between masses j and j+1 (pushing j back by u_j and j+1 forward by u_j).
    Each mass is tied to its neighbours (walls at both ends) by a spring and a damper."""
    M = masses
    Lap = 2.0 * np.eye(M) - np.eye(M, k=1) - np.eye(M, k=-1)   # spring / damper coupling
    Ac = np.zeros((2 * M, 2 * M))
    Ac[:M, M:] = np.eye(M)
    Ac[M:, :M] = -(k_s / mass) * Lap
    Ac[M:, M:] = -(b_d / mass) * Lap
    Bc = np.zeros((2 * M, M - 1))
    for j in range(M - 1):
        Bc[M + j, j] = -1.0 / mass
        Bc[M + j + 1, j] = 1.0 / mass
    return Ac, Bc


def zoh(Ac: np.ndarray, Bc: np.ndarray, Ts: float):
    """Zero-order-hold discretisation: expm([[Ac, Bc], [0, 0]] Ts) = [[A, B], [0, I]]."""
    import scipy.linalg
    n, m = Bc.shape
    E = np.zeros((n + m, n + m))
    E[:n, :n], E[:n, n:] = Ac, Bc
    F = scipy.linalg.expm(E * Ts)
    return F[:n, :n].copy(), F[:n, n:].copy()


def markov_tree(horizon: int, p_c, P_c) -> tuple[Tree, np.ndarray]:
    """Scenario tree of a Markov chain with len(p_c) modes, branching at every stage: the root's
    children are the modes of w_0 with probabilities p_c, a node in mode a has one child per
    mode b with conditional probability P_c[a][b].  Returns the tree and each node's mode
    (the root's entry is -1)."""
    nm = len(p_c)
    cond = [list(p_c)]
    modes = [-1]
    frontier = [-1]
    for t in range(horizon):
        nxt = []
        for a in frontier:
            for b in range(nm):
                nxt.append(b)
        if t < horizon - 1:
            cond.extend([list(P_c[b]) for b in nxt])
        modes.extend(nxt)
        frontier = nxt
    tree = tree_from_branching([nm] * horizon, cond_probs=cond)
    return tree, np.asarray(modes, dtype=np.int64)


def spring_mass(x0: np.ndarray | None = None, p_max: float | None = None) -> Problem:
    """The spring-mass stochastic optimal control problem with initial state x0 (default 0).
    The cost is x'Qx + u'Ru per stage and x'Q_N x at the leaves (Section IV-A's weights);
    |u| <= u_max, |v| <= v_max, |p| <= p_max (the position bound is not stated in the paper)."""
    S = SPRING_MASS
    M = S["masses"]
    Ac, Bc = spring_mass_continuous(M, S["mass"], S["k_s"], S["b_d"])
    A, B = zoh(Ac, Bc, S["Ts"])
    tree, modes = markov_tree(S["horizon"], S["p_c"], S["P_c"])
    nn = tree.num_nodes
    nx, nu = 2 * M, M - 1
    An = np.broadcast_to(A, (nn, nx, nx)).copy()
    Bn = np.broadcast_to(B, (nn, nx, nu)).copy()
    An[0], Bn[0] = 0.0, 0.0
    c = np.zeros((nn, nx))
    c[1:] = np.asarray(S["c_mode"])[modes[1:]][:, None]
    pm = S["p_max"] if p_max is None else p_max
    xmax = np.concatenate([np.full(M, pm), np.full(M, S["v_max"])])
    p = Problem(tree=tree, nx=nx, nu=nu, A=An, B=Bn, c=c, Q=np.full(nx, S["Q"]), R=np.full(nu, S["R"]),
                PN=np.full(nx, S["QN"]), q=np.zeros(nx), r=np.zeros(nu), pN=np.zeros(nx),
                xlo=-xmax, xhi=xmax.copy(), ulo=np.full(nu, -S["u_max"]), uhi=np.full(nu, S["u_max"]),
                x0=np.zeros(nx) if x0 is None else np.asarray(x0, dtype=np.float64), name="spring_mass")
    return p


def spring_mass_x0s():
    """The stored initial states: uniform on the problem's domain (rejection from the state box
    with an LP feasibility test), written by oracle/make_spring_mass.py."""
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "data", "spring_mass_x0.json")
    with open(path) as f:
        d = json.load(f)
    return np.asarray(d["x0"], dtype=np.float64), d
