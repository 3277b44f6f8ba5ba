"""The subtree split of the solve (oracle/split.py) on CPU ranks: the multi-GPU layout of the method
checked on host processes (gloo, 127.0.0.1).

Each rank owns whole subtrees below a split stage and the dual entries of their nodes; the stages
above are replicated.  A solve exchanges only the subtree roots' s (one all-gather), the factor
only the roots' P (one all-gather), NAMA's inner products, residual norm and FBE terms are
all-reduced scalars.  The split must reproduce the unsplit oracle: the factor node by node, the
solve step entry by entry (Algorithms 3 and 4), and NAMA's iterates step by step."""
import multiprocessing as mp
import os
import socket

import numpy as np
import pytest

from oracle import oracle as O
from oracle import split as SP
from paper_2107_01745_b300 import workloads as W
from tests import dense_kkt as D


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _problems():
    # a ragged tree, a tree shaped like the paper-scale one (binary, then one child per node), and
    # a problem whose box binds (NAMA iterates)
    return [W.random_problem(71, horizon=4, nx=3, nu=2, max_branch=3, p_branch=0.7),
            W.random_problem(72, tree=W.tree_from_branching([2, 2, 2, 1, 1, 1]), nx=4, nu=2),
            D.boxed_problem(17, horizon=4, nx=4, nu=2, frac=0.9)]


class _GlooComm:
    def __init__(self, dist):
        self.dist = dist
        self.rank, self.world = dist.get_rank(), dist.get_world_size()

    def allgather(self, a):
        out = [None] * self.world
        self.dist.all_gather_object(out, np.asarray(a))
        return out

    def _reduce(self, v, op):
        import torch
        t = torch.tensor([float(v)], dtype=torch.float64)
        self.dist.all_reduce(t, op=op)
        return float(t.item())

    def allreduce_sum(self, v):
        return self._reduce(v, self.dist.ReduceOp.SUM)

    def allreduce_max(self, v):
        return self._reduce(v, self.dist.ReduceOp.MAX)


def _run_rank(comm, problems):
    """Everything one rank computes: its factor rows, solves of two duals, NAMA after 0, 3, 8
    iterations and to tolerance, and the exchange counts of one solve."""
    out = []
    for pi, p in enumerate(problems):
        comm.calls = {}  # counted per problem
        plan = SP.Plan(p.tree, comm.world)
        rk = SP.SplitRank(p, plan, comm)
        rows = np.concatenate([rk.mine, rk.top])
        rec = {"rows": rows, "P": rk.P[rows], "K": {i: rk.K[i] for i in rows if i < rk.Np}, "solves": []}
        for seed, hom in ((5, False), (6, True)):
            y = W.random_dual(p, seed)
            y = np.where(rk.present, y, 0.0)  # a rank holds only its own entries and the top's
            before = dict(getattr(comm, "calls", {}))
            x, u = rk.solve(y, homogeneous=hom)
            after = comm.calls
            rec["solves"].append((seed, hom, x[rows], u[[i for i in rows if i < rk.Np]],
                                  after["allgather_s"] - before.get("allgather_s", 0)))
        if pi == 2:
            lam = 0.05
            rec["nama"] = [(K, rk.nama(lam, tol=0.0, max_iter=K)) for K in (0, 3, 8)]
            rec["nama_tol"] = rk.nama(lam, tol=1e-6, max_iter=2000)
            rec["present"] = rk.present
        rec["calls"] = dict(comm.calls)
        out.append(rec)
    return out


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        q.put((rank, _run_rank(_GlooComm(dist), _problems())))
    finally:
        dist.barrier()
        dist.destroy_process_group()


def _check(recs_by_rank, problems):
    for pi, p in enumerate(problems):
        o = O.LQOracle(p)
        covered = np.zeros(p.tree.num_nodes, dtype=int)
        for recs in recs_by_rank:
            rec = recs[pi]
            rows = rec["rows"]
            covered[rows] += 1
            # factor: node by node equal to the unsplit recursion
            assert np.allclose(rec["P"], o.P[rows], rtol=1e-12, atol=1e-12 * np.max(np.abs(o.P)))
            for i, K in rec["K"].items():
                assert np.allclose(K, o.K[i], rtol=1e-11, atol=1e-12 * np.max(np.abs(o.K)))
            for seed, hom, x, u, n_s in rec["solves"]:
                xr, ur = o.solve(W.random_dual(p, seed), homogeneous=hom)
                scale = max(1.0, np.max(np.abs(xr)), np.max(np.abs(ur)))
                assert np.max(np.abs(x - xr[rows])) <= 1e-12 * scale
                assert np.max(np.abs(u - ur[[i for i in rows if i < o.Np]])) <= 1e-12 * scale
                assert n_s == 1  # one all-gather of the roots' s per solve
            assert rec["calls"]["allgather_P"] == 1
        assert np.all(covered >= 1)
        if pi == 2:
            for recs in recs_by_rank:
                rec = recs[pi]
                pres = rec["present"]
                for K, got in rec["nama"]:
                    ref = O.nama(o, 0.05, tol=0.0, max_iter=K)
                    assert got["iters"] == ref["iters"] == K
                    d = np.max(np.abs(got["ybar"][pres] - ref["ybar"][pres]))
                    assert d <= 1e-10 * max(1.0, np.max(np.abs(ref["ybar"]))), (K, d)
                    assert abs(got["res"][-1] - ref["res"][-1]) <= 1e-10 * max(1.0, ref["res"][-1])
                # to 1e-6, where every FBE comparison of the line search is decided far above
                # rounding (near 1e-10 the two sides' summation orders can flip one of them):
                # the same stopping iteration and iterate
                ref = O.nama(o, 0.05, tol=1e-6, max_iter=2000)
                got = rec["nama_tol"]
                assert got["res_inf"] <= 1e-6 and got["iters"] == ref["iters"]
                assert np.max(np.abs(got["ybar"][pres] - ref["ybar"][pres])) <= 1e-9 * max(1.0, np.max(np.abs(ref["ybar"])))


def test_plan_owns_every_subtree_once():
    t = W.tree_from_branching([2, 3, 2, 1, 1])
    for world in (1, 2, 3, 4, 5, 6):
        plan = SP.Plan(t, world)
        assert len(plan.roots) >= world and np.all(t.stage[plan.roots] == plan.ts)
        assert np.all(t.stage[:plan.roots[0]] < plan.ts)
        # every node below the split has exactly one owner, the owner of its root; ranks own
        # contiguous blocks of roots, every rank at least one
        for j in range(t.num_nodes):
            if t.stage[j] >= plan.ts:
                a = j
                while t.stage[a] > plan.ts:
                    a = t.parent[a]
                assert plan.owner[j] == plan.owner[a] >= 0
            else:
                assert plan.owner[j] == -1
        assert sorted(set(plan.root_owner)) == list(range(world))
        assert np.all(np.diff(plan.root_owner) >= 0)
    with pytest.raises(ValueError):
        SP.Plan(t, 13)


def test_one_rank_equals_the_unsplit_oracle():
    probs = _problems()
    _check([_run_rank(SP.LocalComm(), probs)], probs)


@pytest.mark.parametrize("world", [2, 3])
def test_gloo_ranks_equal_the_unsplit_oracle(world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for pr in procs:
        pr.start()
    out = dict(q.get(timeout=600) for _ in range(world))
    for pr in procs:
        pr.join(timeout=120)
        assert pr.exitcode == 0
    _check([out[r] for r in range(world)], _problems())
