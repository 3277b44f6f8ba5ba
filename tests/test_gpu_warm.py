"""Learned warm start on the tensor cores against the FP64 oracle (oracle/mlp.py).

The GPU keeps inputs, weights, hidden activations and output gradients in BF16 and accumulates
in FP32; the oracle models the same storage rounding in FP64 (bf16=True).  Tolerances: the two
differ where an activation sits within the FP32 evaluation error of a BF16 rounding boundary
(one BF16 unit, 2^-8 relative, at a few entries) and by FP32 accumulation, so outputs agree to
2e-3 of their scale and gradients to 1e-2 of each block's norm; against the exact FP64 network
(no storage rounding) the bound is a few BF16 units, 3e-2 of the scale."""
import numpy as np
import pytest
import torch

from oracle import mlp as M
from oracle import oracle as O
from paper_2107_01745_b300 import workloads as W

pytestmark = pytest.mark.gpu

NX, NU, BATCH = 3, 2, 256
WIDTHS = [128, 256]  # both hidden widths the kernels tile (256 is the configured one)


def _tree():
    return W.tree_from_branching([2, 2, 1])


def _params(seed, H, d_in=4 * NX + 1, d_out=NX + NU):
    p = M.init_params(np.random.default_rng(seed), d_in, H, d_out)
    return {k: v.astype(np.float32).astype(np.float64) for k, v in p.items()}


@pytest.fixture(scope="module", params=WIDTHS, ids=lambda h: f"hidden{h}")
def net(cuda_device, request):
    from paper_2107_01745_b300.stotree import StoWarm
    return StoWarm(_tree(), NX, NU, hidden=request.param, batch=BATCH, seed=1)


def _rows(seed, rows, d_in=4 * NX + 1, d_out=NX + NU):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((rows, d_in)).astype(np.float32)
    T = rng.standard_normal((rows, d_out)).astype(np.float32)
    nv = rng.choice([NX, NX + NU], size=rows).astype(np.int32)
    return X, T, nv


def _dev(a):
    return torch.as_tensor(a, device="cuda")


@pytest.mark.parametrize("M_,N_,K_", [(128, 16, 16), (256, 256, 256), (300, 40, 104), (1000, 600, 520)])
def test_gemm_bf16_matches_fp64(cuda_device, M_, N_, K_):
    from paper_2107_01745_b300.stotree import gemm_bf16
    g = torch.Generator().manual_seed(M_ + N_ + K_)
    A = torch.randn(M_, K_, generator=g).to(torch.bfloat16)
    B = torch.randn(N_, K_, generator=g).to(torch.bfloat16)
    C = gemm_bf16(A.cuda(), B.cuda()).cpu().double()
    ref = A.double() @ B.double().T
    assert (C - ref).abs().max().item() <= 1e-5 * ref.abs().max().item()


@pytest.mark.parametrize("rows", [BATCH, 200])
def test_forward_matches_oracle(net, rows):
    p = _params(2, net.hidden)
    net.set_params(net.flatten(p))
    X, _, _ = _rows(3, rows)
    Y = net.forward(_dev(X)).cpu().numpy().astype(np.float64)
    ref_b = M.forward(p, X, bf16=True)["Y"]
    ref = M.forward(p, X)["Y"]
    assert np.max(np.abs(Y - ref_b)) <= 2e-3 * max(1.0, np.max(np.abs(ref_b)))
    assert np.max(np.abs(Y - ref)) <= 3e-2 * max(1.0, np.max(np.abs(ref)))


def test_params_round_trip(net):
    p = net.flatten(_params(4, net.hidden)).astype(np.float32)
    net.set_params(p)
    assert np.array_equal(net.params(), p)


@pytest.mark.parametrize("rows", [BATCH, 137])
def test_gradients_match_oracle(net, rows):
    p = _params(5, net.hidden)
    net.set_params(net.flatten(p))
    X, T, nv = _rows(6, rows)
    g, loss = net.gradients(_dev(X), _dev(T), _dev(nv))
    g = net.unflatten(g.cpu().numpy().astype(np.float64))
    loss_ref, g_ref, _ = M.loss_and_grads(p, X, T, nv, bf16=True)
    assert abs(loss - loss_ref) <= 1e-3 * loss_ref
    for k in g_ref:
        assert np.linalg.norm(g[k] - g_ref[k]) <= 1e-2 * np.linalg.norm(g_ref[k]), k


def test_adam_steps_match_oracle(net):
    """Three Adam steps on one batch.  An Adam step moves each weight by about lr times the sign
    of its gradient, so weights whose gradient is within the gradient tolerance of zero may move
    the other way; all others must agree closely."""
    p = _params(7, net.hidden)
    net.set_params(net.flatten(p))
    X, T, nv = _rows(8, BATCH)
    lr, steps = 1e-3, 3
    st = M.adam_init(p)
    ref = {k: v.copy() for k, v in p.items()}
    for _ in range(steps):
        net.train_batch(_dev(X), _dev(T), _dev(nv), lr=lr)
        _, g_ref, _ = M.loss_and_grads(ref, X, T, nv, bf16=True)
        M.adam_step(ref, g_ref, st, lr=lr)
    got = net.unflatten(net.params().astype(np.float64))
    for k in ref:
        d = np.abs(got[k] - ref[k]).ravel()
        assert np.max(d) <= 2 * steps * lr + 1e-6, k
        assert np.mean(d <= 0.05 * steps * lr) >= 0.97, k


def test_predict_matches_oracle_features(net):
    """Feature gather (x0, t/N, c of the node and two ancestors), forward pass and the scatter of
    sqrt(pi) ybar into the dual layout, for every node of three draws."""
    tree = _tree()
    p = _params(9, net.hidden)
    net.set_params(net.flatten(p))
    rng = np.random.default_rng(10)
    D = 3
    x0 = rng.uniform(-3, 3, (D, NX)).astype(np.float32)
    c = (0.1 * rng.standard_normal((D, tree.num_nodes, NX))).astype(np.float32)
    c[:, 0] = 0.0
    net.set_draws(_dev(x0), _dev(c))
    y = net.predict(0, D).cpu().numpy().astype(np.float64)
    offs = W.dual_offsets(tree, NX, NU)
    nonleaf = tree.child_count > 0
    for d in range(D):
        F = M.node_features(tree.parent, tree.stage, tree.horizon, x0[d].astype(np.float64),
                            c[d].astype(np.float64))
        Yr = M.forward(p, F, bf16=True)["Y"]
        ref = np.zeros(net.m)
        for i in range(tree.num_nodes):
            nv = NX + NU if nonleaf[i] else NX
            ref[offs[i]:offs[i] + nv] = np.sqrt(tree.prob[i]) * Yr[i, :nv]
        assert np.max(np.abs(y[d] - ref)) <= 2e-3 * max(1.0, np.max(np.abs(ref))), d


def test_training_reduces_loss(net):
    """Targets: the unconstrained trajectory Hx(0) of each draw (affine in x0 and c); training
    over many epochs must cut the loss several times."""
    tree = _tree()
    rng = np.random.default_rng(11)
    g = W.make_group(rng, 3, 2, 2, NX, NU, 64)
    y = np.stack([O.LQOracle(g.instance(k)).hx(np.zeros(net.m)) for k in range(64)])
    net.set_params(net.flatten(_params(12, net.hidden)))
    net.set_draws(_dev(g.x0.astype(np.float32)), _dev(g.c.astype(np.float32)), _dev(y.astype(np.float32)))
    assert g.tree().num_nodes == tree.num_nodes
    hist = net.train(300, lr=2e-3, seed=5).cpu().numpy()
    assert np.all(np.isfinite(hist))
    assert hist[-20:].mean() < 0.2 * hist[:20].mean()


def test_rejects_bad_sizes(cuda_device):
    from paper_2107_01745_b300.stotree import StoError, StoWarm
    with pytest.raises(StoError):
        StoWarm(_tree(), NX, NU, hidden=64, batch=BATCH)
    with pytest.raises(StoError):
        StoWarm(_tree(), NX, NU, hidden=128, batch=300)
