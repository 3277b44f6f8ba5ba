"""Batched instances (shared dynamics per shape group) against the FP64 oracle, instance by
instance: the oracle solves every instance as a stand-alone tree problem."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2107_01745_b300 import workloads as W

pytestmark = pytest.mark.gpu


def _rel2(a, b):
    return float(np.linalg.norm(a - b) / max(1e-30, np.linalg.norm(b)))


def _relinf(a, b):
    return float(np.max(np.abs(a - b)) / max(1.0, np.max(np.abs(b))))


@pytest.fixture(scope="module")
def small():
    from paper_2107_01745_b300.stotree import StoBatch
    groups = W.batched_small(30, instances=3)
    sb = StoBatch(groups)
    sb.factor()
    oracles = [[O.LQOracle(g.instance(k)) for k in range(g.num_instances)] for g in groups]
    return groups, sb, oracles


VARIANTS = [0, 1, 2, 3]  # the round kernels the tuner chooses from (stobatch_round_config order)


@pytest.mark.parametrize("variant", VARIANTS)
def test_batched_solve_step_matches_oracle(cuda_device, small, variant):
    """One batched round of Algorithm 3 / 4 equals the oracle's solve of every instance, with
    every round kernel variant."""
    groups, sb, oracles = small
    sb.set_round_variant(1, variant)
    ys = [W.random_dual(g.instance(k), 50 + 10 * gi + k) for gi, g in enumerate(groups) for k in range(g.num_instances)]
    flat = [o for row in oracles for o in row]
    y = sb.pack(ys)
    for homog in (False, True):
        h = sb.solve_step(y, homogeneous=homog).cpu().numpy()
        for k, (o, yk) in enumerate(zip(flat, ys)):
            hk = h[sb.offsets[k]:sb.offsets[k] + sb.sizes[k]]
            assert _rel2(hk, o.hx(yk, homogeneous=homog)) < 1e-5, (homog, k)
    # scaled: ybar in, S Hx out
    yb = sb.pack([yk / o.sq for o, yk in zip(flat, ys)])
    hs = sb.solve_step(yb, scaled=True).cpu().numpy()
    for k, (o, yk) in enumerate(zip(flat, ys)):
        assert _rel2(hs[sb.offsets[k]:sb.offsets[k] + sb.sizes[k]], o.sq * o.hx(yk)) < 1e-5


@pytest.mark.parametrize("variant", VARIANTS)
def test_batched_nama_matches_oracle(cuda_device, small, variant):
    """Batched NAMA reaches the tolerance for every instance; each solution matches the
    oracle's NAMA on that instance at the same tolerance and step size (rounds of one and two
    right-hand sides with every round kernel variant)."""
    groups, sb, oracles = small
    sb.set_round_variant(1, variant)
    sb.set_round_variant(2, variant)
    lams = []
    for row in oracles:
        lam, _ = O.power_lambda(row[0], np.random.default_rng(0).standard_normal(row[0].m))
        lams.append(lam)
    res = sb.nama(np.array(lams), tol=1e-5, max_iter=400)
    y = res["y"].cpu().numpy()
    hx = res["hx"].cpu().numpy()
    k = 0
    for gi, row in enumerate(oracles):
        for o in row:
            info = res["infos"][k]
            assert info["status"] == 0 and info["res_inf"] <= 1e-5
            ref = O.nama(o, lams[gi], tol=1e-5, max_iter=400)
            sl = slice(sb.offsets[k], sb.offsets[k] + sb.sizes[k])
            assert _relinf(hx[sl], ref["h"]) < 1e-4
            assert _relinf(y[sl], ref["y"]) < 1e-4
            k += 1


@pytest.mark.parametrize("variant", VARIANTS)
def test_batched_round_at_the_column_kernel_limits(cuda_device, variant):
    """Shapes at the column kernel's padded widths (nx = 32, nu = 16; nx = 20, nu = 10, the
    learned-warm-start family's) with branching and chain stages: one round with each variant
    against the oracle, and the tuner's measurements reported."""
    from paper_2107_01745_b300.stotree import StoBatch
    rng = np.random.default_rng(33)
    groups = [W.make_group(rng, 5, 2, 3, 32, 16, 2), W.make_group(rng, 6, 4, 2, 20, 10, 3)]
    sb = StoBatch(groups)
    sb.factor()
    cfg = sb.round_config(1)
    assert cfg["tile_cols"] in (32, 64, 128) and all(v > 0 for v in cfg["tuned_ms"].values())
    sb.set_round_variant(1, variant)
    ys, flat = [], []
    for gi, g in enumerate(groups):
        for k in range(g.num_instances):
            ys.append(W.random_dual(g.instance(k), 70 + 10 * gi + k))
            flat.append(O.LQOracle(g.instance(k)))
    y = sb.pack(ys)
    for homog in (False, True):
        h = sb.solve_step(y, homogeneous=homog).cpu().numpy()
        sb.round_status()
        for k, (o, yk) in enumerate(zip(flat, ys)):
            hk = h[sb.offsets[k]:sb.offsets[k] + sb.sizes[k]]
            assert _rel2(hk, o.hx(yk, homogeneous=homog)) < 1e-5, (homog, k)


def test_column_kernel_refused_for_wide_shapes(cuda_device):
    from paper_2107_01745_b300.stotree import StoBatch, StoError
    rng = np.random.default_rng(34)
    sb = StoBatch([W.make_group(rng, 3, 2, 2, 40, 8, 2)])
    sb.factor()
    assert sb.round_config(1)["tuned_ms"]["column128"] == -1.0
    with pytest.raises(StoError) as ei:
        sb.set_round_variant(1, 3)
    assert ei.value.code == 1


@pytest.mark.slow
def test_batched_uneven_workload(cuda_device):
    """The 512-instance workload: every instance converges; sampled instances match the oracle."""
    from paper_2107_01745_b300.stotree import StoBatch
    groups = W.batched_uneven(3)
    sb = StoBatch(groups)
    sb.factor()
    lams = sb.group_lambdas()
    res = sb.nama(lams, tol=1e-4, max_iter=500)
    assert all(i["status"] == 0 and i["res_inf"] <= 1e-4 for i in res["infos"])
    hx = res["hx"].cpu().numpy()
    rng = np.random.default_rng(0)
    for gi in rng.choice(len(groups), size=4, replace=False):
        g = groups[gi]
        k_local = int(rng.integers(0, g.num_instances))
        k = sum(gg.num_instances for gg in groups[:gi]) + k_local
        o = O.LQOracle(g.instance(k_local))
        ref = O.nama(o, lams[gi], tol=1e-4, max_iter=500)
        sl = slice(sb.offsets[k], sb.offsets[k] + sb.sizes[k])
        assert _relinf(hx[sl], ref["h"]) < 1e-4
        assert _relinf(res["y"].cpu().numpy()[sl], ref["y"]) < 1e-4
