"""E2LSH symbol strings on the GPU against the oracle: offsets, symbols
(bit for bit, including values that land exactly on bucket boundaries), the
symbol MSM, and the whole epsilon graph."""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

COS, EUC = 0, 1


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


def _u64(t):
    return t.cpu().numpy().view(np.uint64)


def test_offsets_match_oracle(msm):
    for seed, Q, ell in [(3, 2, 37), (99, 5, 64)]:
        got = msm.e2lsh_offsets(seed, Q * ell).cpu().numpy()
        assert np.array_equal(got, oracle.e2lsh_offsets(seed, Q, ell).ravel())


@pytest.mark.parametrize("sw,ell,dtype", [(4, 40, "f32"), (2, 100, "f32"), (4, 64, "bf16"),
                                          (2, 128, "bf16"), (1, 70, "f32")])
def test_projection_bit_exact(msm, sw, ell, dtype):
    import torch
    n, D, Q = 3000, 96, 2
    X = W.clustered(n, D, 12, 0.05, 31 + sw)
    if dtype == "bf16":
        X = W.to_bf16_values(X)
    R = W.gaussian_R(Q, D, ell, 5 + ell)
    u = oracle.e2lsh_offsets(17, Q, ell)
    width = np.float32(0.37)
    Xg = _t(X).to(torch.bfloat16) if dtype == "bf16" else _t(X)
    S, rec = msm.project_e2lsh(Xg, _t(R), _t(u), float(width), sw, return_recomputed=True)
    want = oracle.project_e2lsh(X, R, u, float(width), sw)
    assert np.array_equal(_u64(S), want.view(np.uint64))
    assert 0 <= rec < Q * n * ell


def test_projection_on_bucket_boundaries(msm):
    """t / width + u lands exactly on integers: R holds multiples of the
    width, rows are basis vectors and u = 0, so every float value is a tie
    that only the double evaluation settles."""
    D, ell, Q, sw = 16, 32, 1, 4
    width = 0.5
    rng = np.random.default_rng(1)
    R = (rng.integers(-20, 21, size=(Q, D, ell)) * width).astype(np.float32)
    X = np.eye(D, dtype=np.float32)
    u = np.zeros((Q, ell), dtype=np.float32)
    S, rec = msm.project_e2lsh(_t(X), _t(R), _t(u), width, sw, return_recomputed=True)
    assert np.array_equal(_u64(S), oracle.project_e2lsh(X, R, u, width, sw).view(np.uint64))
    assert rec == Q * D * ell


def _sym_pool(n, ell, sw, Q, seed):
    rng = np.random.default_rng(seed)
    C = rng.integers(0, 1 << sw, size=(20, ell))
    lab = rng.integers(0, 20, size=(Q, n))
    sym = np.where(rng.random((Q, n, ell)) < 0.05, rng.integers(0, 1 << sw, size=(Q, n, ell)),
                   C[lab])
    Wd = (ell * sw + 63) // 64
    S = np.zeros((Q, n, Wd), dtype=np.uint64)
    for c in range(ell):
        S[:, :, (c * sw) // 64] |= sym[:, :, c].astype(np.uint64) << np.uint64((c * sw) % 64)
    return S


@pytest.mark.parametrize("n,ell,sw,k,d,Q", [(3000, 32, 2, 8, 4, 2), (2500, 30, 4, 10, 5, 1),
                                            (2000, 64, 4, 8, 3, 2), (4500, 24, 2, 6, 0, 3)])
def test_enumerate_symbols_bit_exact(msm, n, ell, sw, k, d, Q):
    S = _sym_pool(n, ell, sw, Q, n + ell + sw)
    pairs, st = msm.enumerate_symbols(_t(S.view(np.int64)), ell, sw, k, d, canonical=True)
    want, ost = oracle.msm_sym(S, ell, sw, k, d)
    assert np.array_equal(_u64(pairs), want)
    assert st["masks"] == ost["masks"]


@pytest.mark.parametrize("metric,eps,sw", [(EUC, 0.45, 2), (COS, 0.1, 4)])
def test_eps_graph_e2lsh_matches_oracle(msm, metric, eps, sw):
    n, D = 5000, 64
    X = W.clustered(n, D, 10, 0.05, 77)
    ell, k, d, Q = 24, 6, 3, 2
    R = W.gaussian_R(Q, D, ell, 8)
    radius = eps if metric == EUC else float(np.sqrt(2 * np.float32(eps)))
    width = float(np.float32(4.0 * radius))
    seed = 12
    pairs, dist, st = msm.eps_graph(_t(X), metric, eps, ell, k, d, Q=Q, R=_t(R), seed=seed,
                                    canonical=True, e2lsh={"symbol_bits": sw, "width": width})
    u = oracle.e2lsh_offsets(seed, Q, ell)
    want, wd, info = oracle.eps_graph_e2lsh(X, R, u, width, sw, ell, k, d, metric, eps)
    assert np.array_equal(_u64(pairs), want)
    assert np.allclose(dist.cpu().numpy().astype(np.float64), wd, rtol=1e-5,
                       atol=(D + 8) * 2.0 ** -51)
    assert st["cand"] == info["cand"] and st["count"] > 0
