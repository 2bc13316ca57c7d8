"""Learned projection (MLP features for the sign projection): forward,
gradient and optimiser parity with oracle/mlp.py, and what training buys.

Tolerances come from float accumulation over K terms: each output is
within K * 2^-24 * sum |a_k b_k| of the exact value (per GEMM); we allow
4x that plus the gelu evaluation error."""
import numpy as np
import pytest

import oracle
import workloads as W
from oracle import mlp as omlp

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def msm():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_0904_3151_gb300 import build as b
    b.build()
    import paper_0904_3151_gb300 as m
    m.lib()
    return m


def _t(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _net(msm, dim=128, hidden=512, dim_out=128, seed=3):
    net = msm.MLPProjection(dim, hidden, dim_out, seed=seed)
    # give the biases nonzero values so they are exercised
    h, d, o = hidden, dim, dim_out
    rng = np.random.default_rng(seed)
    p = net.params.cpu().numpy()
    p[h * d: h * d + h] = rng.normal(0, 0.1, h)
    p[h * d + h + o * h:] = rng.normal(0, 0.1, o)
    net.params.copy_(_t(p))
    return net


def _oracle_weights(net):
    h, d, o = net.hidden, net.dim, net.dim_out
    p = net.params.cpu().numpy().astype(np.float64)
    W1 = net.W1h.float().cpu().numpy().astype(np.float64)   # the bf16 values
    W2 = net.W2h.float().cpu().numpy().astype(np.float64)
    return W1, p[h * d: h * d + h], W2, p[h * d + h + o * h:]


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_mlp_forward_matches_oracle(msm, dtype):
    import torch
    net = _net(msm)
    X = W.clustered(3000, 128, 10, 0.1, 5)
    if dtype == "bf16":
        X = W.to_bf16_values(X)
    Xg = _t(X).to(torch.bfloat16) if dtype == "bf16" else _t(X)
    Y = net.features(Xg).cpu().numpy().astype(np.float64)
    W1, b1, W2, b2 = _oracle_weights(net)
    Yo, H, A = omlp.forward(X, W1, b1, W2, b2)
    # bound, valid for both the float CUDA-core path and the tensor-core path
    # (operands split into bf16 high and low parts: each carries 16
    # significant bits, 2^-16 relative, and twice the products accumulate):
    # per layer (2^-16 + 4 * 2 * terms * 2^-24) * |operand| @ |weights|, the
    # first layer's error carried through gelu (|gelu'| <= 1.13) and W2
    rep = 2.0 ** -16
    e1 = (rep + 4 * 2 * 128 * 2.0 ** -24) * (np.abs(X) @ np.abs(W1).T)
    bound = (rep + 4 * 2 * 512 * 2.0 ** -24) * (np.abs(A) @ np.abs(W2).T) + \
        1.2 * (e1 + 1e-6) @ np.abs(W2).T
    assert np.all(np.abs(Y - Yo) <= bound + 1e-6)
    # and far tighter in practice than the worst case
    assert np.max(np.abs(Y - Yo)) < 1e-3 * np.max(np.abs(Yo))


def test_mlp_grad_matches_oracle(msm):
    import torch
    net = _net(msm, seed=4)
    X = W.clustered(2000, 128, 8, 0.1, 6)
    rng = np.random.default_rng(1)
    B = 512
    pi = rng.integers(0, 2000, B).astype(np.uint32)
    pj = rng.integers(0, 2000, B).astype(np.uint32)
    label = rng.integers(0, 2, B).astype(np.uint8)
    W1, b1, W2, b2 = _oracle_weights(net)
    mp, mn = 0.98, 0.3
    Yo, _, _ = omlp.forward(X, W1, b1, W2, b2)
    cos = np.einsum("ij,ij->i", Yo[pi], Yo[pj]) / (
        np.linalg.norm(Yo[pi], axis=1) * np.linalg.norm(Yo[pj], axis=1))
    viol = np.where(label == 1, mp - cos, cos - mn)
    keep = np.abs(viol) > 1e-4              # away from the hinge's kink
    pi, pj, label = pi[keep], pj[keep], label[keep]
    loss_o, grads_o = omlp.loss_and_grads(X, W1, b1, W2, b2, pi.astype(np.int64),
                                          pj.astype(np.int64), label, mp, mn)
    loss, g = net.grad(_t(X), _t(pi.view(np.int32)), _t(pj.view(np.int32)), _t(label), mp, mn)
    g = g.cpu().numpy().astype(np.float64)
    assert loss == pytest.approx(loss_o, rel=1e-4)
    off = 0
    for go in grads_o:
        gg = g[off: off + go.size].reshape(go.shape)
        off += go.size
        assert np.linalg.norm(gg - go) <= 1e-3 * np.linalg.norm(go) + 1e-7


def test_mlp_adam_matches_oracle(msm):
    import torch
    net = _net(msm, dim=32, hidden=64, dim_out=16, seed=5)
    rng = np.random.default_rng(2)
    p0 = net.params.cpu().numpy().astype(np.float64)
    g = rng.normal(size=p0.size).astype(np.float32)
    m = np.zeros(p0.size)
    v = np.zeros(p0.size)
    gt = _t(g)
    want = p0
    for t in (1, 2, 3):
        net.adam(gt, lr=1e-2)
        want, m, v = omlp.adam_step(want, g.astype(np.float64), m, v, t, 1e-2)
    got = net.params.cpu().numpy().astype(np.float64)
    assert np.allclose(got, want, rtol=1e-5, atol=1e-6)
    h, d, o = 64, 32, 16
    assert np.array_equal(net.W1h.float().cpu().numpy(),
                          W.to_bf16_values(got[:h * d].astype(np.float32)).reshape(h, d))


def test_learned_projection_lowers_missing_ratio(msm):
    """Train on pairs the plain method finds (neighbours) and random pairs
    (non-neighbours); at equal ell, k, d and a single replicate the learned
    features miss fewer true pairs than the random projection of x, and the
    result still has no false pair (the recheck uses x)."""
    import torch
    wl = W.WORKLOADS["small"]
    n, eps = 6000, wl.eps
    X = W.clustered(n, 128, 24, wl.sigma, 77)
    Xg = _t(X)
    truth = msm.eps_count_exhaustive(Xg, "cosine", eps)
    # training pairs: the plain method's output (Q = 3) + random pairs
    pos, _, _ = msm.eps_graph(Xg, "cosine", eps, wl.ell, wl.k, wl.d, Q=3, seed=11)
    rng = np.random.default_rng(3)
    P = pos.cpu().numpy().view(np.uint64)
    P = P[rng.choice(len(P), min(len(P), 200000), replace=False)]
    # non-neighbours: random pairs outside eps
    ri = rng.integers(0, n, 3 * len(P))
    rj = rng.integers(0, n, 3 * len(P))
    Xn = X / np.linalg.norm(X, axis=1, keepdims=True)
    far = (ri != rj) & (1.0 - np.einsum("ij,ij->i", Xn[ri], Xn[rj]) > eps)
    ri, rj = ri[far][:len(P)].astype(np.uint32), rj[far][:len(P)].astype(np.uint32)
    pi = np.concatenate([(P >> np.uint64(32)).astype(np.uint32), ri])
    pj = np.concatenate([(P & np.uint64(0xFFFFFFFF)).astype(np.uint32), rj])
    lab = np.concatenate([np.ones(len(P), np.uint8), np.zeros(len(ri), np.uint8)])
    net = msm.MLPProjection(128, 512, 128, seed=1)
    # neighbours sit at cos ~0.99 in x: m_pos above that pulls them tighter
    hist = net.train(Xg, _t(pi.view(np.int32)), _t(pj.view(np.int32)), _t(lab), steps=1000,
                     batch=4096, lr=1e-2, m_pos=0.999, m_neg=0.2)
    assert np.mean(hist[-20:]) < np.mean(hist[:5])
    Y = net.features(Xg)
    miss = {}
    for name, kw in [("random", {}), ("learned", {"Y": Y})]:
        ratios = []
        for seed in (21, 22, 23):
            p, _, _ = msm.eps_graph(Xg, "cosine", eps, wl.ell, wl.k, wl.d, Q=1, seed=seed, **kw)
            ratios.append((truth - p.numel()) / truth)
        miss[name] = float(np.mean(ratios))
    assert miss["random"] > 0.01
    assert miss["learned"] < 0.1 * miss["random"], miss
    # no false pairs with learned strings either
    p, d, _ = msm.eps_graph(Xg, "cosine", eps, wl.ell, wl.k, wl.d, Q=1, seed=21, Y=Y)
    assert p.numel() <= truth
    dv = oracle.dist(X, p.cpu().numpy().view(np.uint64)[:2000], oracle.COSINE)
    assert np.all(dv <= np.float32(eps))
