"""Batched form: many independent point sets in one call.

The batched result is defined as the union of the per-set results of the
single-pool method, with each set's indices shifted by its offset; no pair
may join two sets.  The oracle runs set by set, so a set boundary that the
GPU path failed to respect shows up as an extra pair."""
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


def _shift(pairs, o):
    return pairs + ((np.uint64(o) << np.uint64(32)) | np.uint64(o))


# sizes chosen to cover empty and one-point sets, sets that end exactly on a
# radix tile (4096 items) and one item past it, and a set spanning tiles
SIZES = [0, 1, 700, 2, 4096, 0, 37, 4097, 300, 1, 2500]


@pytest.mark.parametrize("ell,k,d,Q", [(64, 8, 4, 2), (128, 10, 6, 1), (200, 12, 8, 1)])
def test_enumerate_sets_bit_exact(msm, ell, k, d, Q):
    off = np.concatenate([[0], np.cumsum(SIZES)]).astype(np.int64)
    n = int(off[-1])
    # one shared centre pool: many close strings lie in different sets
    S = W.random_strings(n, ell, Q, 31 + ell, n_centres=25, flip=0.02)
    pairs, st = msm.enumerate_sets(_t(S.view(np.int64)), off, ell, k, d, canonical=True)
    want = []
    for s in range(len(SIZES)):
        a, b = int(off[s]), int(off[s + 1])
        if b - a >= 2:
            p, _ = oracle.msm(np.ascontiguousarray(S[:, a:b]), ell, k, d)
            want.append(_shift(p, a))
    want = np.sort(np.concatenate(want))
    assert np.array_equal(_u64(pairs), want)
    # the same strings as one pool do have pairs across the sets
    whole, _ = msm.enumerate_pairs(_t(S.view(np.int64)), ell, k, d)
    assert whole.numel() > len(want)


def _sets_case(sizes, dim=64, seed=5):
    X, off = W.clustered_sets(sizes, dim, 6, 0.05, seed)
    return X, off


@pytest.mark.parametrize("metric,eps", [(COS, 0.12), (EUC, 0.45)])
def test_eps_graph_sets_matches_per_set_oracle(msm, metric, eps):
    X, off = _sets_case([900, 0, 1, 2000, 3, 1500, 4097])
    ell, k, d, Q = 64, 8, 4, 2
    R = W.gaussian_R(Q, X.shape[1], ell, 77)
    Xg = _t(X)
    pairs, dist, counts, st = msm.eps_graph_sets(Xg, off, metric, eps, ell, k, d, Q=Q, R=_t(R),
                                                 out_mode=0, canonical=True)
    want, wd, wc = [], [], []
    for s in range(len(off) - 1):
        a, b = int(off[s]), int(off[s + 1])
        if b - a < 2:
            wc.append(0)
            continue
        p, dd, _ = oracle.eps_graph(X[a:b], R, ell, k, d, metric, eps)
        want.append(_shift(p, a))
        wd.append(dd)
        wc.append(len(p))
    want = np.concatenate(want)
    order = np.argsort(want)
    assert np.array_equal(_u64(pairs), want[order])
    assert np.allclose(dist.cpu().numpy().astype(np.float64), np.concatenate(wd)[order],
                       rtol=1e-5, atol=(X.shape[1] + 8) * 2.0 ** -51)
    assert np.array_equal(counts, np.array(wc))
    # count-only (recheck fused into the pair check): same per-set counts
    _, _, c2, s2 = msm.eps_graph_sets(Xg, off, metric, eps, ell, k, d, Q=Q, R=_t(R),
                                      out_mode=2)
    assert np.array_equal(c2, counts)
    assert s2["count"] == len(want)
    assert s2["cand"] == st["cand"]


def test_eps_graph_sets_degenerate(msm):
    X, off = _sets_case([1, 1, 1, 1, 0, 1], dim=32)
    _, _, counts, st = msm.eps_graph_sets(_t(X), off, COS, 0.5, 32, 4, 2, Q=1, seed=1)
    assert st["count"] == 0 and not counts.any()
    # one set holding everything equals the single-pool call
    X, off = _sets_case([3000], dim=32)
    p1, _, c1, _ = msm.eps_graph_sets(_t(X), off, COS, 0.1, 32, 4, 2, Q=2, seed=3, out_mode=1,
                                      canonical=True)
    p0, _, _ = msm.eps_graph(_t(X), COS, 0.1, 32, 4, 2, Q=2, seed=3, out_mode=1, canonical=True)
    assert np.array_equal(_u64(p1), _u64(p0)) and c1[0] == p0.numel()


def test_eps_graph_sets_rejects_bad_offsets(msm):
    X, off = _sets_case([100, 200], dim=32)
    for bad in ([1, 100, 300], [0, 200, 100, 300], [0, 100, 299]):
        with pytest.raises((msm.MSMError, AssertionError)):
            msm.eps_graph_sets(_t(X), np.array(bad), COS, 0.1, 32, 4, 2, Q=1)


@pytest.mark.parametrize("wl_name,Q,n", [("small", 3, 6000), ("scale", 2, 8000),
                                          ("precision", 1, 3000)])
def test_fused_count_equals_pair_list(msm, wl_name, Q, n):
    """Count-only output rechecks candidates inside the pair check; its
    count, candidate and type-I figures equal those of the pair-list path."""
    import torch
    wl = W.WORKLOADS[wl_name]
    X = W.clustered(n, wl.dim, max(4, n // 500), wl.sigma, 11, normalise=wl.normalise)
    Xg = _t(X)
    if wl.dtype == "bf16":
        Xg = Xg.to(torch.bfloat16)
    metric = COS if wl.metric == "cosine" else EUC
    p, _, s0 = msm.eps_graph(Xg, metric, wl.eps, wl.ell, wl.k, wl.d, Q=Q, seed=2, out_mode=1)
    _, _, s1 = msm.eps_graph(Xg, metric, wl.eps, wl.ell, wl.k, wl.d, Q=Q, seed=2, out_mode=2)
    assert s1["count"] == p.numel() == s0["count"]
    assert s1["cand"] == s0["cand"] and s1["type1"] == s0["type1"]
    assert s1["checks"] == s0["checks"]


# ------------------------------------------------- plans and the autotuner

def test_plan_runs_direct_then_graph(msm):
    import torch
    X, off = _sets_case([900, 0, 1, 2000, 3, 1500, 4097], seed=21)
    ell, k, d, Q = 64, 8, 4, 2
    _, _, want, st = msm.eps_graph_sets(_t(X), off, COS, 0.12, ell, k, d, Q=Q, seed=4)
    plan = msm.Plan(off, X.shape[1], torch.float32, COS, 0.12, ell, k, d, Q=Q, seed=4)
    graphs = []
    for _ in range(3):
        c, counts, s = plan.run(_t(X))
        assert c == st["count"] and np.array_equal(counts, want)
        assert s["cand"] == st["cand"] and s["checks"] == st["checks"]
        graphs.append(plan.is_graph)
    assert graphs == [False, True, True]
    # other data of the same shape through the input buffer (no copy)
    Y, _ = _sets_case([900, 0, 1, 2000, 3, 1500, 4097], seed=22)
    plan.input.copy_(_t(Y))
    c, counts, _ = plan.run()
    _, _, want2, st2 = msm.eps_graph_sets(_t(Y), off, COS, 0.12, ell, k, d, Q=Q, seed=4)
    assert c == st2["count"] and np.array_equal(counts, want2)
    plan.close()


def test_plan_reports_deferred_input_errors(msm):
    import torch
    X, off = _sets_case([500, 700], dim=32, seed=3)
    plan = msm.Plan(off, 32, torch.float32, COS, 0.1, 32, 4, 2, Q=1, seed=1)
    plan.run(_t(X))
    plan.run(_t(X))                     # now a graph
    Z = X.copy()
    Z[600] = 0
    with pytest.raises(msm.MSMError) as e:
        plan.run(_t(Z))
    assert e.value.status == -6
    Z[600, 3] = np.nan
    with pytest.raises(msm.MSMError) as e:
        plan.run(_t(Z))
    assert e.value.status == -7
    c, _, _ = plan.run(_t(X))           # the plan stays usable
    _, _, _, st = msm.eps_graph_sets(_t(X), off, COS, 0.1, 32, 4, 2, Q=1, seed=1)
    assert c == st["count"]
    plan.close()


def test_autotune_picks_valid_knobs_and_caches(msm, tmp_path):
    X, off = _sets_case([3000, 2000, 5000], dim=64, seed=8)
    cache = str(tmp_path / "tune.txt")
    tu = msm.autotune(_t(X), off, COS, 0.12, 64, 8, 4, Q=3, seed=2, cache_path=cache)
    assert tu["check_min_blocks"] in (2, 4, 5) and tu["check_ctas_per_sm"] in (6, 8)
    assert tu["masks_per_batch"] in (0, 18, 35)
    lines = open(cache).read().splitlines()
    assert len(lines) == 1
    assert msm.autotune(_t(X), off, COS, 0.12, 64, 8, 4, Q=3, seed=2, cache_path=cache) == tu
    assert open(cache).read().splitlines() == lines   # served from the cache
    _, _, c0, _ = msm.eps_graph_sets(_t(X), off, COS, 0.12, 64, 8, 4, Q=3, seed=2)
    _, _, c1, _ = msm.eps_graph_sets(_t(X), off, COS, 0.12, 64, 8, 4, Q=3, seed=2, tuning=tu)
    assert np.array_equal(c0, c1)


@pytest.mark.parametrize("tuning", [dict(check_min_blocks=2), dict(check_min_blocks=5,
                                    check_ctas_per_sm=8), dict(masks_per_batch=7)])
def test_tuning_knobs_do_not_change_results(msm, tuning):
    X, off = _sets_case([2500, 4000, 10], dim=64, seed=12)
    _, _, c0, s0 = msm.eps_graph_sets(_t(X), off, COS, 0.12, 64, 8, 4, Q=2, seed=6)
    _, _, c1, s1 = msm.eps_graph_sets(_t(X), off, COS, 0.12, 64, 8, 4, Q=2, seed=6, tuning=tuning)
    assert np.array_equal(c0, c1) and s0["cand"] == s1["cand"]
