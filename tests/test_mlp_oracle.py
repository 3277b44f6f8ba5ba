"""Pins of the warm-start MLP oracle against things other than itself: PyTorch's FP64 autograd,
its tanh-form GELU, its Adam and its BF16 cast (independent library routines; the oracle does
not call PyTorch), exact central differences, and a feature row traced by hand."""
import numpy as np
import pytest
import torch

from oracle import mlp as M
from paper_2107_01745_b300 import workloads as W


def _torch_params(p):
    return {k: torch.tensor(v, dtype=torch.float64, requires_grad=True) for k, v in p.items()}


def _torch_loss(tp, X, T, nvalid):
    Xt = torch.tensor(X, dtype=torch.float64)
    a1 = torch.nn.functional.gelu(Xt @ tp["W1"].T + tp["b1"], approximate="tanh")
    a2 = torch.nn.functional.gelu(a1 @ tp["W2"].T + tp["b2"], approximate="tanh")
    y = a2 @ tp["W3"].T + tp["b3"]
    mask = torch.tensor((np.arange(T.shape[1])[None, :] < nvalid[:, None]).astype(np.float64))
    d = (y - torch.tensor(T)) * mask
    return (d * d).sum() / mask.sum()


def _case(seed=0, B=37, d_in=9, hidden=16, d_out=6):
    rng = np.random.default_rng(seed)
    p = M.init_params(rng, d_in, hidden, d_out)
    X = rng.standard_normal((B, d_in))
    T = rng.standard_normal((B, d_out))
    nvalid = rng.choice([d_out - 2, d_out], size=B)
    return p, X, T, nvalid


def test_gelu_matches_torch_tanh_gelu():
    z = np.linspace(-9.0, 9.0, 2001)
    ref = torch.nn.functional.gelu(torch.tensor(z), approximate="tanh").numpy()
    assert np.max(np.abs(M.gelu(z) - ref)) < 1e-14
    assert M.gelu(0.0) == 0.0
    # the derivative against exact central differences (error O(h^2) ~ 1e-10)
    h = 1e-5
    fd = (M.gelu(z + h) - M.gelu(z - h)) / (2 * h)
    assert np.max(np.abs(M.gelu_grad(z) - fd)) < 1e-8
    assert abs(M.gelu_grad(0.0) - 0.5) < 1e-15


def test_gelu_close_to_exact_erf_form():
    """The tanh form approximates x Phi(x) to within about 5e-4 (Hendrycks and Gimpel)."""
    from scipy.special import erf
    z = np.linspace(-6.0, 6.0, 1201)
    exact = 0.5 * z * (1.0 + erf(z / np.sqrt(2.0)))
    assert np.max(np.abs(M.gelu(z) - exact)) < 1e-3


def test_loss_and_gradients_match_torch_autograd():
    p, X, T, nvalid = _case()
    loss, g, _ = M.loss_and_grads(p, X, T, nvalid)
    tp = _torch_params(p)
    tl = _torch_loss(tp, X, T, nvalid)
    tl.backward()
    assert abs(loss - tl.item()) < 1e-13 * max(1.0, abs(loss))
    for k in p:
        ref = tp[k].grad.numpy()
        assert np.max(np.abs(g[k] - ref)) < 1e-12 * max(1.0, np.max(np.abs(ref))), k


def test_gradients_by_central_differences():
    p, X, T, nvalid = _case(seed=1, B=11, d_in=5, hidden=7, d_out=4)
    _, g, _ = M.loss_and_grads(p, X, T, nvalid)
    rng = np.random.default_rng(3)
    h = 1e-6
    for k in p:
        for _ in range(6):
            idx = tuple(int(rng.integers(0, s)) for s in p[k].shape)
            pp = {kk: v.copy() for kk, v in p.items()}
            pm = {kk: v.copy() for kk, v in p.items()}
            pp[k][idx] += h
            pm[k][idx] -= h
            fd = (M.loss_and_grads(pp, X, T, nvalid)[0] - M.loss_and_grads(pm, X, T, nvalid)[0]) / (2 * h)
            assert abs(fd - g[k][idx]) < 1e-7 * max(1.0, abs(fd)), (k, idx)


def test_adam_matches_torch_adam():
    p, X, T, nvalid = _case(seed=2)
    tp = _torch_params(p)
    opt = torch.optim.Adam(list(tp.values()), lr=1e-2, betas=(0.9, 0.999), eps=1e-8)
    st = M.adam_init(p)
    for _ in range(4):
        _, g, _ = M.loss_and_grads(p, X, T, nvalid)
        M.adam_step(p, g, st, lr=1e-2)
        opt.zero_grad()
        _torch_loss(tp, X, T, nvalid).backward()
        opt.step()
    for k in p:
        assert np.max(np.abs(p[k] - tp[k].detach().numpy())) < 1e-12, k


def test_bf16_round_matches_torch_cast():
    rng = np.random.default_rng(4)
    a = np.concatenate([rng.standard_normal(5000) * 10.0 ** rng.integers(-6, 6, 5000),
                        [0.0, -0.0, 1.0, 65504.0, 1e-40, 3.3895313892515355e38]])
    ref = torch.tensor(a, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(M.bf16_round(a), ref)
    # ties go to the even neighbour: 1 + 2^-8 lies halfway between 1 and 1 + 2^-7
    assert M.bf16_round(1.0 + 2.0 ** -8) == 1.0
    assert M.bf16_round(1.0 + 3 * 2.0 ** -8) == 1.0 + 2.0 ** -6


def test_bf16_forward_within_bf16_bound():
    """The BF16 storage model stays within a few BF16 units of the exact forward pass."""
    p, X, T, nvalid = _case(seed=5, B=64, d_in=30, hidden=64, d_out=8)
    y = M.forward(p, X)["Y"]
    yb = M.forward(p, X, bf16=True)["Y"]
    assert np.max(np.abs(y - yb)) < 16 * 2.0 ** -8 * max(1.0, np.max(np.abs(y)))
    assert np.max(np.abs(y - yb)) > 0.0


def test_node_features_by_hand():
    tree = W.tree_from_branching([2, 2, 1])
    stage = np.zeros(tree.num_nodes, dtype=int)
    for i in range(1, tree.num_nodes):
        stage[i] = stage[tree.parent[i]] + 1
    nx = 2
    x0 = np.array([0.5, -1.5])
    c = np.arange(tree.num_nodes * nx, dtype=float).reshape(tree.num_nodes, nx)
    c[0] = 0.0
    F = M.node_features(tree.parent, stage, 3, x0, c)
    assert F.shape == (tree.num_nodes, 4 * nx + 1)
    # root: x0, t/N = 0, no disturbance, no ancestors
    assert np.array_equal(F[0], [0.5, -1.5, 0.0] + [0.0] * 6)
    # node 8 is the only child of node 4 (stage 2), whose parent is node 1 (stage 1)
    leaf = 8
    assert tree.parent[leaf] == 4 and tree.parent[4] == 1
    assert np.array_equal(F[leaf], [0.5, -1.5, 1.0] + list(c[8]) + list(c[4]) + list(c[1]))
    # node 3: parent 1, grandparent the root (zeros)
    assert np.array_equal(F[3], [0.5, -1.5, 2 / 3] + list(c[3]) + list(c[1]) + [0.0, 0.0])
