"""Write spring_mass_oracle_iters.json: the FP64 oracle's iteration counts of NAMA and MINFBE
(tolerance 5e-4, L-BFGS memory 5, at most 300 iterations) on the first 16 stored initial
states of the spring-mass experiment (Section IV-A), with the lambda they used.  Calls only
the oracle; the GPU tests compare their own iteration counts with these.

    python -m tests.golden.make_spring_mass_iters
"""
import json
import os

import numpy as np

from oracle import oracle as O
from paper_2107_01745_b300 import workloads as W

COUNT = 16
MAX_ITER = 300


def main():
    X, meta = W.spring_mass_x0s()
    p = W.spring_mass(X[0], p_max=meta["p_max"])
    o = O.LQOracle(p)
    lam, L = O.power_lambda(o, np.random.default_rng(0).standard_normal(o.m))
    out = {"lambda": lam, "L": L, "tol": 5e-4, "max_iter": MAX_ITER, "states": list(range(COUNT))}
    for name, fn in (("nama", O.nama), ("minfbe", O.minfbe)):
        its, conv = [], []
        for k in range(COUNT):
            o.p.x0 = X[k]
            r = fn(o, lam, tol=5e-4, max_iter=MAX_ITER)
            its.append(int(r["iters"]))
            conv.append(r["status"] == "converged")
            print(name, k, its[-1], conv[-1], flush=True)
        out[name] = {"iters": its, "converged": conv}
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "spring_mass_oracle_iters.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print("wrote", path)


if __name__ == "__main__":
    main()
