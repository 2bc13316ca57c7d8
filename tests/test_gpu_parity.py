"""Parity of the CUDA path (through the C ABI) against the CPU oracle.

Integer and index results (strings, pair lists, counts) must match bit for
bit; distances within 1e-5 relative of the oracle's double-precision value
(plus that value's own cancellation error, (dim + 8) 2^-51 for Eq. 2).
"""
import itertools
import math

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


def _sorted_u64(t):
    return np.sort(_u64(t))


def _ham_q(Sa, Sb):
    """Hamming distance per replicate: [Q][m] from two [Q][m][W] pools."""
    x = np.ascontiguousarray(Sa ^ Sb)
    return np.unpackbits(x.view(np.uint8), axis=-1).reshape(x.shape[0], x.shape[1], -1).sum(-1)


def _dist_tol(dim):
    return dict(rtol=1e-5, atol=(dim + 8) * 2.0 ** -51)


# ----------------------------------------------------------------- A0'

def test_gaussian_matches_oracle(msm):
    for seed, count in [(0, 1), (3, 4097), (2002, 300_001)]:
        g = msm.gaussian(seed, count).cpu().numpy()
        o = oracle.gaussian(seed, count)
        diff_ulp = np.abs(g.view(np.int32).astype(np.int64) - o.view(np.int32).astype(np.int64))
        assert diff_ulp.max() <= 1
        assert (diff_ulp == 0).mean() >= 0.9999


# ------------------------------------------------------------------ A1

@pytest.mark.parametrize("n,dim,ell,Q", [(1, 7, 16, 1), (130, 33, 64, 2), (1000, 64, 96, 3),
                                         (777, 128, 128, 2), (300, 256, 200, 1),
                                         (65, 5, 256, 2), (4097, 128, 128, 1),
                                         (20000, 128, 128, 3), (3000, 32, 64, 5)])
@pytest.mark.parametrize("dtype", ["f32", "bf16"])
@pytest.mark.parametrize("simt", [False, True])
def test_project_bit_exact(msm, n, dim, ell, Q, dtype, simt):
    """Rows of 128..512 bytes take the tcgen05 path unless simt is forced."""
    import torch
    X = W.clustered(n, dim, 7, 0.2, n + dim, normalise=False)
    if dtype == "bf16":
        X = W.to_bf16_values(X)
    R = W.gaussian_R(Q, dim, ell, ell + Q)
    Xg = _t(X).to(torch.bfloat16) if dtype == "bf16" else _t(X)
    S, rec = msm.project(Xg, ell, Q, R=_t(R), simt=simt, return_recomputed=True)
    assert np.array_equal(_u64(S).reshape(Q, n, -1), oracle.project(X, R))


def test_project_ties_and_zero_rows(msm):
    # x orthogonal to some columns exactly: t == 0 must give '0' (Eq. 3)
    dim, ell = 4, 64
    R = np.zeros((1, dim, ell), dtype=np.float32)
    R[0, 0, :] = 1.0
    R[0, 1, :] = -1.0
    R[0, 2, ::2] = 0.5
    X = np.array([[1, 1, 0, 0], [0, 0, 0, 0], [1, 1, 2, 0], [2, 1, 0, 3]], dtype=np.float32)
    S, rec = msm.project(_t(X), ell, 1, R=_t(R), return_recomputed=True)
    assert np.array_equal(_u64(S).reshape(1, 4, -1), oracle.project(X, R))
    assert rec > 0


def test_project_device_R_from_seed(msm):
    X = W.clustered(500, 32, 5, 0.1, 3)
    S = msm.project(_t(X), 64, 2, seed=77)
    R = oracle.gaussian(77, 2 * 32 * 64).reshape(2, 32, 64)
    want = oracle.project(X, R)
    # R agrees with the oracle's generator to 1 ulp; bits may differ only
    # where |t| is of the order of that ulp difference
    assert (np.unpackbits(_u64(S).reshape(2, 500, 1).view(np.uint8)) !=
            np.unpackbits(want.view(np.uint8))).sum() <= 2


# --------------------------------------------------------------- A3-A7

ENUM_CASES = [  # n, ell, k, d, Q, centres, flip
    (2, 16, 4, 2, 1, 1, 0.0),
    (200, 16, 4, 2, 1, 8, 0.1),
    (5000, 64, 8, 4, 2, 40, 0.04),
    (4097, 64, 8, 0, 3, 300, 0.0),
    (3000, 96, 8, 4, 2, 25, 0.03),
    (3000, 128, 10, 6, 2, 20, 0.03),
    (2000, 130, 7, 3, 2, 30, 0.02),
    (1500, 200, 12, 8, 1, 10, 0.03),
    (1000, 256, 9, 4, 2, 10, 0.01),
    (1200, 32, 32, 3, 2, 40, 0.03),
    (3000, 40, 5, 1, 2, 200, 0.02),
    (2500, 128, 12, 8, 1, 15, 0.03),
]


@pytest.mark.parametrize("n,ell,k,d,Q,nc,flip", ENUM_CASES)
def test_enumerate_bit_exact(msm, n, ell, k, d, Q, nc, flip):
    S = W.random_strings(n, ell, Q, n + ell + k + d, n_centres=nc, flip=flip)
    pairs, st = msm.enumerate_pairs(_t(S.view(np.int64)), ell, k, d, canonical=True)
    want, ost = oracle.msm(S, ell, k, d)
    got = _u64(pairs)
    assert np.array_equal(got, want)          # canonical order: identical arrays
    assert st["cand"] == len(want)
    assert st["masks"] == ost["masks"]
    if _keys_exact(ell, k, d):
        assert st["checks"] == ost["checks"]
    else:
        assert st["checks"] >= ost["checks"]


def _keys_exact(ell, k, d):
    """Whether the library's automatic grouping key holds every kept block
    set exactly (then the in-group pair count equals the oracle's): with a
    first-gap sub-key (some grouping has gap blocks, blocks <= 16 bits) the
    key is 32 bits and the kept bits plus the first gap block must fit;
    otherwise the kept bits must fit 24."""
    widths = [(b + 1) * ell // k - b * ell // k for b in range(k)]
    masks = list(itertools.combinations(range(k), k - d))
    gaps = [[b for b in range(max(K)) if b not in K] for K in masks]
    if any(gaps) and max(widths) <= 16:
        return all(sum(widths[b] for b in K) + (widths[g[0]] if g else 0) <= 32
                   for K, g in zip(masks, gaps))
    return max(sum(widths[b] for b in K) for K in masks) <= 24


def test_enumerate_one_large_group(msm):
    """All strings equal: one run of n items -> every pair (tiled path)."""
    n, ell = 300, 64
    S = np.tile(W.random_strings(1, ell, 1, 5), (1, n, 1))
    for d in [0, 3]:
        pairs, st = msm.enumerate_pairs(_t(S.view(np.int64)), ell, 8, d, canonical=True)
        i, j = np.triu_indices(n, 1)
        want = (i.astype(np.uint64) << np.uint64(32)) | j.astype(np.uint64)
        assert np.array_equal(_u64(pairs), np.sort(want))


@pytest.mark.parametrize("seed,ell,k,d,probs", [
    (1, 64, 8, 4, [0.02, 0.1, 0.3, 0.5, 0.5, 0.3, 0.1, 0.02]),
    (2, 64, 8, 4, [0.5, 0.05, 0.2, 0.02, 0.4, 0.1, 0.3, 0.5]),
    (3, 40, 10, 6, [0.15] * 10),
    (4, 40, 10, 6, [0.4, 0.03, 0.25, 0.1, 0.5, 0.05, 0.2, 0.3, 0.02, 0.45]),
])
def test_enumerate_subkey_groups(msm, seed, ell, k, d, probs):
    """Long runs split into first-gap-block groups of every size: block b of
    a string is a fixed value with its lowest bit flipped with probability
    probs[b], so the Hamming distance is the number of differing blocks and
    runs of equal kept blocks hold hundreds of members whose first gap block
    takes two values in sorted order -- tiles with uniform rows, uniform
    columns, two groups on the diagonal and mixed groups all occur."""
    n = 1200
    rng = np.random.default_rng(seed)
    lo = [b * ell // k for b in range(k)]
    S = np.zeros((1, n, 1), dtype=np.uint64)
    for b in range(k):
        width = (b + 1) * ell // k - lo[b]
        v = np.uint64(rng.integers(0, 1 << width))
        flip = (rng.random(n) < probs[b]).astype(np.uint64)
        S[0, :, 0] |= (v ^ flip) << np.uint64(lo[b])
    pairs, st = msm.enumerate_pairs(_t(S.view(np.int64)), ell, k, d, canonical=True)
    want, ost = oracle.msm(S, ell, k, d)
    assert len(want) > 10000
    assert np.array_equal(_u64(pairs), want)
    if _keys_exact(ell, k, d):
        assert st["checks"] == ost["checks"]
    else:
        assert st["checks"] >= ost["checks"]


def test_enumerate_unordered_matches(msm):
    S = W.random_strings(3000, 64, 2, 9, n_centres=30, flip=0.05)
    pairs, _ = msm.enumerate_pairs(_t(S.view(np.int64)), 64, 8, 4, canonical=False)
    want, _ = oracle.msm(S, 64, 8, 4)
    got = _u64(pairs)
    assert len(np.unique(got)) == len(got)
    assert np.array_equal(np.sort(got), want)


# ------------------------------------------------------------------ A8

def _pairs_from(i, j):
    lo, hi = np.minimum(i, j), np.maximum(i, j)
    keep = lo < hi
    return np.unique((lo[keep].astype(np.uint64) << np.uint64(32)) | hi[keep].astype(np.uint64))


@pytest.mark.parametrize("metric,eps,dtype", [(COS, 0.05, "f32"), (EUC, 0.3, "f32"),
                                              (COS, 0.1, "bf16"), (EUC, 0.45, "bf16")])
def test_recheck_exact_decisions(msm, metric, eps, dtype):
    import torch
    n, dim = 3000, 96
    X = W.clustered(n, dim, 10, 0.04, 21)
    # boundary stress: pairs built at distance ~eps
    rng = np.random.default_rng(5)
    if dtype == "bf16":
        X = W.to_bf16_values(X)
    cand = _pairs_from(rng.integers(0, n, 40000), rng.integers(0, n, 40000))
    dv = oracle.dist(X, cand, metric)
    # add the 2000 candidate pairs closest to eps from a wider sample
    wide = _pairs_from(rng.integers(0, n, 400000), rng.integers(0, n, 400000))
    wd = oracle.dist(X, wide, metric)
    near = wide[np.argsort(np.abs(wd - eps))[:2000]]
    cand = np.unique(np.concatenate([cand, near]))
    dv = oracle.dist(X, cand, metric)
    Xg = _t(X).to(torch.bfloat16) if dtype == "bf16" else _t(X)
    p, dist, rec = msm.recheck(Xg, _t(cand.view(np.int64)), metric, eps)
    got = _u64(p)
    order = np.argsort(got)
    got, gd = got[order], dist.cpu().numpy()[order].astype(np.float64)
    keep = dv <= float(np.float32(eps))
    assert np.array_equal(got, cand[keep])
    assert np.allclose(gd, dv[keep], **_dist_tol(dim))


def test_recheck_exact_ties(msm):
    # Euclidean distance exactly eps (3-4-5) and cosine exactly 1 (orthogonal)
    X = np.array([[0, 0, 0, 0], [3, 4, 0, 0], [6, 8, 0, 0], [0, 0, 5, 0]], dtype=np.float32)
    cand = _pairs_from(np.array([0, 0, 1, 0, 1, 2]), np.array([1, 2, 2, 3, 3, 3]))
    p, dist, _ = msm.recheck(_t(X), _t(cand.view(np.int64)), EUC, 5.0)
    assert set(_u64(p).tolist()) == set(cand[oracle.dist(X, cand, EUC) <= 5.0].tolist())
    Xc = X[1:] + np.float32(1.0)
    cand = _pairs_from(np.array([0, 0, 1]), np.array([1, 2, 2]))
    p, dist, _ = msm.recheck(_t(Xc), _t(cand.view(np.int64)), COS, 1.0)
    assert set(_u64(p).tolist()) == set(cand[oracle.dist(Xc, cand, COS) <= 1.0].tolist())


@pytest.mark.parametrize("bad", [(7, 300), (9, 9), (12, 5), (1 << 31, 2)])
def test_recheck_rejects_out_of_range_pairs(msm, bad):
    """A candidate that is not i < j < n (j = n, i = j, i > j, huge i) is
    never read: the call returns MSM_E_INVAL, and the next call is clean."""
    n, dim = 300, 16
    X = W.clustered(n, dim, 4, 0.05, 3)
    good = _pairs_from(np.arange(0, 40), np.arange(1, 41))
    cand = np.append(good, np.uint64((bad[0] << 32) | bad[1]))
    with pytest.raises(msm.MSMError) as e:
        msm.recheck(_t(X), _t(cand.view(np.int64)), COS, 0.5)
    assert e.value.status == -1 and "i < j < n" in str(e.value)
    p, _, _ = msm.recheck(_t(X), _t(good.view(np.int64)), COS, 0.5)
    assert np.array_equal(np.sort(_u64(p)), good[oracle.dist(X, good, COS) <= 0.5])


# ------------------------------------------------------------ whole path

def _eps_graph_case(msm, wl, Q, n=None, dtype="f32", **kw):
    import torch
    n = n or wl.n
    X = W.clustered(n, wl.dim, max(2, wl.n_clusters * n // wl.n), wl.sigma, wl.data_seed)
    if dtype == "bf16":
        X = W.to_bf16_values(X)
    R = W.gaussian_R(Q, wl.dim, wl.ell, wl.r_seed)
    Xg = _t(X).to(torch.bfloat16) if dtype == "bf16" else _t(X)
    metric = COS if wl.metric == "cosine" else EUC
    pairs, dist, st = msm.eps_graph(Xg, metric, wl.eps, wl.ell, wl.k, wl.d, Q=Q,
                                    R=_t(R), canonical=True, **kw)
    want, wd, info = oracle.eps_graph(X, R, wl.ell, wl.k, wl.d, metric, wl.eps)
    return X, pairs, dist, st, want, wd, info


def test_eps_graph_small_workload(msm):
    """The 20,000 x 64 workload (l=64, k=8, d=4, cosine eps=0.15)."""
    wl = W.WORKLOADS["small"]
    # 32-bit exact grouping keys, so the inspected-pair count is the oracle's
    X, pairs, dist, st, want, wd, info = _eps_graph_case(msm, wl, Q=7, group_bits=32)
    assert np.array_equal(_u64(pairs), want)
    assert np.allclose(dist.cpu().numpy().astype(np.float64), wd, **_dist_tol(wl.dim))
    assert st["cand"] == info["cand"]
    assert st["checks"] == info["checks"]      # 32 kept bits: exact keys
    assert st["type1"] == info["type1"]
    assert st["masks"] == 7 * 70


@pytest.mark.parametrize("group_bits", [8, 16])
def test_eps_graph_hashed_grouping_keys(msm, group_bits):
    """Grouping keys narrower than the kept bits collide; the pair list
    must not change (the in-group check requires equal kept blocks)."""
    wl = W.WORKLOADS["small"]
    X, pairs, dist, st, want, wd, info = _eps_graph_case(msm, wl, Q=2, n=4000,
                                                         group_bits=group_bits)
    assert np.array_equal(_u64(pairs), want)
    assert st["checks"] >= info["checks"]


def test_eps_graph_precision_geometry_bf16(msm):
    """bf16 storage, Euclidean eps=0.3, l=128, k=12, d=8 (495 groupings)."""
    wl = W.WORKLOADS["precision"]
    X, pairs, dist, st, want, wd, info = _eps_graph_case(msm, wl, Q=2, n=3000, dtype="bf16")
    assert np.array_equal(_u64(pairs), want)
    assert np.allclose(dist.cpu().numpy().astype(np.float64), wd, **_dist_tol(wl.dim))


def test_eps_graph_scale_geometry_small_n(msm):
    """l=128, k=10, d=6 (210 groupings, ~51 kept bits -> hashed keys)."""
    wl = W.WORKLOADS["scale"]
    X, pairs, dist, st, want, wd, info = _eps_graph_case(msm, wl, Q=3, n=6000)
    assert np.array_equal(_u64(pairs), want)
    assert st["cand"] == info["cand"]


def test_eps_graph_host_input_and_overflow_retry(msm):
    import torch
    wl = W.WORKLOADS["small"]
    X = W.clustered(5000, wl.dim, 12, wl.sigma, 3)
    R = W.gaussian_R(3, wl.dim, wl.ell, 4)
    want, _, _ = oracle.eps_graph(X, R, wl.ell, wl.k, wl.d, COS, wl.eps)
    for host in [torch.from_numpy(X), torch.from_numpy(X).pin_memory()]:
        pairs, dist, st = msm.eps_graph(host, COS, wl.eps, wl.ell, wl.k, wl.d, Q=3,
                                        R=_t(R), canonical=True, cand_capacity=1000)
        assert np.array_equal(_u64(pairs), want)
        assert st["overflow_retries"] > 0


def test_eps_graph_output_modes(msm):
    wl = W.WORKLOADS["small"]
    X = W.clustered(3000, wl.dim, 10, wl.sigma, 8)
    Xg = _t(X)
    p0, d0, s0 = msm.eps_graph(Xg, COS, wl.eps, wl.ell, wl.k, wl.d, Q=2, seed=5, canonical=True)
    p1, d1, s1 = msm.eps_graph(Xg, COS, wl.eps, wl.ell, wl.k, wl.d, Q=2, seed=5, out_mode=1,
                               canonical=True)
    p2, d2, s2 = msm.eps_graph(Xg, COS, wl.eps, wl.ell, wl.k, wl.d, Q=2, seed=5, out_mode=2)
    assert np.array_equal(_u64(p0), _u64(p1)) and d1 is None
    assert p2 is None and s2["count"] == s0["count"] == len(p0)


def test_eps_graph_Q_from_bound(msm):
    wl = W.WORKLOADS["small"]
    X = W.clustered(2000, wl.dim, 10, wl.sigma, 9)
    _, _, st = msm.eps_graph(_t(X), COS, wl.eps, wl.ell, wl.k, wl.d, Q=0, miss_ratio=1e-3)
    assert st["Q"] == oracle.solve_Q(wl.ell, wl.d, oracle.p_cosine(float(np.float32(wl.eps))), 1e-3)


def test_errors_are_reported(msm):
    wl = W.WORKLOADS["small"]
    X = W.clustered(500, wl.dim, 5, wl.sigma, 1)
    Z = X.copy()
    Z[17] = 0
    with pytest.raises(msm.MSMError) as e:
        msm.eps_graph(_t(Z), COS, 0.1, 64, 8, 4, Q=1)
    assert e.value.status == -6
    N = X.copy()
    N[3, 2] = np.nan
    with pytest.raises(msm.MSMError) as e:
        msm.eps_graph(_t(N), COS, 0.1, 64, 8, 4, Q=1)
    assert e.value.status == -7
    for ell, k, d in [(64, 8, 8), (300, 8, 4), (64, 40, 4), (16, 20, 2)]:
        with pytest.raises(msm.MSMError) as e:
            msm.eps_graph(_t(X), COS, 0.1, ell, k, d, Q=1)
        assert e.value.status == -1
    # Euclidean accepts zero rows
    msm.eps_graph(_t(Z), EUC, 0.1, 64, 8, 4, Q=1)


@pytest.mark.parametrize("metric,eps", [(COS, 0.15), (EUC, 0.4)])
def test_exhaustive_count(msm, metric, eps):
    X = W.clustered(2500, 48, 10, 0.06, 4)
    got = msm.eps_count_exhaustive(_t(X), metric, eps)
    want, _ = oracle.eps_bruteforce(X, metric, float(np.float32(eps)))
    assert got == len(want)


# ------------------------------------------------- full-size, sampled

def test_scale_workload_sampled(msm):
    """The 1,000,000 x 128 workload in the benchmark's launch configuration
    (device-generated R, Q = 11): no false positives, no duplicates, and a
    two-way sampled check against strings and distances the oracle
    computes one point at a time."""
    import torch
    wl = W.WORKLOADS["scale"]
    Q, seed = 11, wl.r_seed
    X = W.clustered(wl.n, wl.dim, wl.n_clusters, wl.sigma, wl.data_seed)
    lab = W.cluster_labels(wl.n, wl.n_clusters, wl.data_seed, wl.dim)
    Xg = _t(X)
    pairs, dist, st = msm.eps_graph(Xg, COS, wl.eps, wl.ell, wl.k, wl.d, Q=Q, seed=seed,
                                    canonical=True)
    m = pairs.numel()
    assert m > 0 and st["count"] == m
    # canonical order from the library's own sort: strictly increasing means
    # every pair once (checked on the device: the list is ~5e8 long)
    assert bool((pairs[1:] > pairs[:-1]).all())
    assert bool((pairs >> 32 < (pairs & 0xFFFFFFFF)).all())
    R = oracle.gaussian(seed, Q * wl.dim * wl.ell).reshape(Q, wl.dim, wl.ell)
    rng = np.random.default_rng(0)
    # (1) sampled output pairs: distance <= eps, some replicate within d
    pos = torch.from_numpy(np.sort(rng.choice(m, 400, replace=False))).cuda()
    smp = _u64(pairs[pos])
    gd = dist[pos].cpu().numpy().astype(np.float64)
    i, j = oracle.unpack_pairs(smp)
    dv = oracle.dist(X, smp, COS)
    assert np.all(dv <= float(np.float32(wl.eps)))
    assert np.allclose(gd, dv, **_dist_tol(wl.dim))
    ham = _ham_q(oracle.project(X[i], R), oracle.project(X[j], R))
    assert np.all(ham.min(axis=0) <= wl.d)
    # (2) sampled same-cluster pairs: in the output iff some replicate finds
    # them within d and their distance is <= eps
    a = rng.integers(0, wl.n, 3000)
    b = np.array([rng.choice(np.flatnonzero(lab == lab[x])[:64]) for x in a[:600]])
    cand = _pairs_from(a[:600], b)
    ci, cj = oracle.unpack_pairs(cand)
    hm = _ham_q(oracle.project(X[ci], R), oracle.project(X[cj], R))
    found = hm.min(axis=0) <= wl.d
    within = oracle.dist(X, cand, COS) <= float(np.float32(wl.eps))
    ct = torch.from_numpy(cand.view(np.int64)).cuda()
    at = torch.searchsorted(pairs, ct).clamp(max=m - 1)
    in_out = (pairs[at] == ct).cpu().numpy()
    assert np.array_equal(in_out, found & within)
    assert found.sum() > 100        # the sample does exercise the path
