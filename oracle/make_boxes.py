"""Write the stored boxes of the synthetic workloads (paper_2107_01745_b300/data/boxes.json).

Reading of "box constraints on x and u at 80 % of the unconstrained-LQ range": for
every state (input) component k, the bound is 0.8 max |x_k^i| (0.8 max |u_k^i|) over
the nodes of the unconstrained solution x(0) of the instance, computed here by the
FP64 oracle (Algorithm 3 at y = 0), but never below 1.02 times the unconstrained
values of the first two stages after the root (inputs of stages 0 and 1).  Those
states are set by x0 through nu < nx inputs, and a plain 80 % box makes the
instance infeasible (the dual iterates diverge).  The box is symmetric; the root
state is fixed to x0 and is not boxed.

Usage: python oracle/make_boxes.py [workload ...]
"""
import json
import os
import sys

import numpy as np

_ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if _ROOT not in sys.path:
    sys.path.insert(0, _ROOT)

from paper_2107_01745_b300 import workloads as W  # noqa: E402
from oracle.oracle import LQOracle  # noqa: E402

RECIPES = {
    "paper_scale": lambda: W.paper_scale_unboxed(2),
}


def largest_box(frac=0.8):
    """The largest instance's box (its statement says only "box constraints"): inputs only, at
    80 % of the largest |u_k| of the unconstrained solution on a calibration tree built by the
    same recipe (horizon 24, binary for the first 4 stages: 351 nodes, small enough for the
    oracle); states unbounded, so every draw stays feasible."""
    p = W.largest_unboxed(5, tree=W.largest_tree(branch_stages=4))
    nn = p.tree.num_nodes
    dense = W.Problem(tree=p.tree, nx=p.nx, nu=p.nu, A=p.A[0:nn], B=p.B[0:nn], c=p.c[0:nn], Q=p.Q, R=p.R, PN=p.PN,
                      q=p.q, r=p.r, pN=p.pN, xlo=p.xlo, xhi=p.xhi, ulo=p.ulo, uhi=p.uhi, x0=p.x0)
    o = LQOracle(dense)
    _, u = o.solve(np.zeros(o.m))
    return np.full(p.nx, np.inf), frac * np.max(np.abs(u), axis=0)


def box_of(p, frac=0.8, protect=2, margin=1.02):
    o = LQOracle(p)
    x, u = o.solve(np.zeros(o.m))
    st = p.tree.stage
    early_x = (st >= 1) & (st <= protect)
    early_u = st[:o.Np] < protect
    xmax = np.maximum(frac * np.max(np.abs(x[1:]), axis=0), margin * np.max(np.abs(x[early_x]), axis=0))
    umax = np.maximum(frac * np.max(np.abs(u), axis=0), margin * np.max(np.abs(u[early_u]), axis=0))
    return xmax, umax


def main(names):
    path = os.path.join(_ROOT, "paper_2107_01745_b300", "data", "boxes.json")
    boxes = {}
    if os.path.exists(path):
        with open(path) as f:
            boxes = json.load(f)
    for name in names:
        if name == "largest":
            xmax, umax = largest_box()
            boxes[name] = {"xmax": None, "umax": [float(v) for v in umax],
                           "recipe": "inputs only: 0.8 * max over nodes of |u_k| of the oracle's x(0) on the "
                                     "calibration tree (horizon 24, binary for 4 stages); states unbounded"}
        else:
            xmax, umax = box_of(RECIPES[name]())
            boxes[name] = {"xmax": [float(v) for v in xmax], "umax": [float(v) for v in umax],
                           "recipe": "max(0.8 * max over nodes, 1.02 * max over stages 1-2 (inputs 0-1)) of |x_k|, "
                                     "|u_k| of the oracle's x(0)"}
        print(name, "xmax range", xmax.min(), xmax.max(), "umax range", umax.min(), umax.max())
    with open(path, "w") as f:
        json.dump(boxes, f, indent=1)


if __name__ == "__main__":
    main(sys.argv[1:] or list(RECIPES) + ["largest"])
