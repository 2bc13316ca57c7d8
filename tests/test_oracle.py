"""Pins for the CPU oracle: each test ties one oracle function to something
other than itself -- a value the paper prints, a closed form, a library
routine, an independent brute force, or a statistical law the paper states.
"""
import itertools
import math
import os

import numpy as np
import pytest
from scipy import stats

import oracle
import workloads as W

COS, EUC = oracle.COSINE, oracle.EUCLIDEAN


def _bits_to_words(bitstrings, ell):
    Wn = (ell + 63) // 64
    out = np.zeros((len(bitstrings), Wn), dtype=np.uint64)
    for i, s in enumerate(bitstrings):
        for c, ch in enumerate(s):
            if ch == "1":
                out[i, c >> 6] |= np.uint64(1) << np.uint64(c & 63)
    return out


def _read_golden(path):
    kv, strings, pairs = {}, [], []
    with open(path) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            tok = line.split()
            if tok[0] == "string":
                strings.append(tok[1])
            elif tok[0] == "pair":
                pairs.append((int(tok[1]), int(tok[2])))
            else:
                kv[tok[0]] = tok[1:]
    return kv, strings, pairs


def _pairs_set(p):
    i, j = oracle.unpack_pairs(p)
    return set(zip(i.tolist(), j.tolist()))


def _ham_numpy(Sq):
    """Pairwise Hamming distances through numpy's bit unpacking (a library
    primitive, independent of the oracle's popcount loop)."""
    bits = np.unpackbits(Sq.view(np.uint8), axis=1, bitorder="little").astype(np.int32)
    return (bits[:, None, :] != bits[None, :, :]).sum(axis=2)


# --------------------------------------------------------------- generator

def test_philox_known_answer(golden_dir):
    kv, _, _ = _read_golden(os.path.join(golden_dir, "philox4x64_10_kat.txt"))
    ctr = [int(x) for x in kv["ctr"]]
    key = [int(x) for x in kv["key"]]
    want = [int(x, 16) for x in kv["out"]]
    assert [int(v) for v in oracle.philox(ctr, key)] == want


@pytest.mark.parametrize("seed", [0, 7, 2**63 + 5])
def test_philox_matches_numpy(seed):
    # numpy's Philox (Philox4x64-10) increments its counter before each block.
    rng = np.random.default_rng(seed)
    for _ in range(20):
        key = rng.integers(0, 2**64, size=2, dtype=np.uint64)
        ctr = rng.integers(0, 2**64, size=4, dtype=np.uint64)
        prev = ctr.copy()
        # counter - 1 with borrow across the 256-bit counter
        for w in range(4):
            if prev[w] != 0:
                prev[w] -= np.uint64(1)
                break
            prev[w] = np.uint64(2**64 - 1)
        bg = np.random.Philox(key=key, counter=prev)
        assert list(bg.random_raw(4)) == list(oracle.philox(ctr, key))


def test_gaussian_distribution():
    z = oracle.gaussian(1234, 400_000).astype(np.float64)
    assert abs(z.mean()) < 5 / math.sqrt(z.size)
    assert abs(z.var() - 1.0) < 5 * math.sqrt(2 / z.size)
    assert stats.kstest(z, "norm").pvalue > 1e-3
    # the two outputs of one Box-Muller pair and neighbouring blocks are
    # uncorrelated
    zz = z.reshape(-1, 4)
    for a, b in [(0, 1), (2, 3), (0, 2)]:
        assert abs(np.corrcoef(zz[:, a], zz[:, b])[0, 1]) < 5 / math.sqrt(zz.shape[0])
    # a prefix of a longer draw is the shorter draw (counter-based)
    assert np.array_equal(oracle.gaussian(1234, 1001), oracle.gaussian(1234, 4000)[:1001])


# -------------------------------------------------------------- projection

@pytest.mark.parametrize("ell", [16, 64, 96, 130])
def test_project_basis_vectors(ell):
    """x = e_m gives t_c = R[m][c] exactly (Eq. 3), so bit c = R[m][c] > 0."""
    D, Q = 7, 2
    R = W.gaussian_R(Q, D, ell, 5)
    X = np.eye(D, dtype=np.float32)
    S = oracle.project(X, R)
    Wn = (ell + 63) // 64
    for q in range(Q):
        for m in range(D):
            want = np.zeros(Wn, dtype=np.uint64)
            for c in range(ell):
                if R[q, m, c] > 0:
                    want[c >> 6] |= np.uint64(1) << np.uint64(c & 63)
            assert np.array_equal(S[q, m], want), (q, m)


def test_project_sign_zero_and_bit_order():
    D, ell = 4, 70
    R = -np.ones((1, D, ell), dtype=np.float32)
    R[0, 0, 5] = 1.0
    R[0, 0, 66] = 2.0
    X = np.array([[1, 0, 0, 0], [0, 0, 0, 0], [-1, 0, 0, 0]], dtype=np.float32)
    S = oracle.project(X, R)
    assert S[0, 0, 0] == np.uint64(1 << 5) and S[0, 0, 1] == np.uint64(1 << 2)
    assert not S[0, 1].any()                      # t == 0 -> '0' (Eq. 3)
    full = np.uint64(2**64 - 1)
    assert S[0, 2, 0] == full ^ np.uint64(1 << 5)
    assert S[0, 2, 1] == np.uint64((1 << 6) - 1) ^ np.uint64(1 << 2)


def test_project_scale_invariance_and_numpy():
    X = W.clustered(200, 24, 5, 0.3, 11, normalise=False)
    R = W.gaussian_R(3, 24, 64, 12)
    S1 = oracle.project(X, R)
    S2 = oracle.project(X * np.float32(4.0), R)   # exact power-of-two scaling
    assert np.array_equal(S1, S2)
    T = np.einsum("nd,qdl->qnl", X.astype(np.float64), R.astype(np.float64))
    bits = (T > 0)
    ok = np.abs(T) > 1e-9                           # away from ties
    got = np.unpackbits(S1.view(np.uint8).reshape(3, 200, 8), axis=2,
                        bitorder="little").astype(bool)
    assert np.array_equal(got[ok], bits[ok])


@pytest.mark.parametrize("theta_over_pi", [0.03, 0.1, 0.25])
def test_eq4_flip_probability_and_binomial_hits(theta_over_pi):
    """Eq. 4: Pr(s_ik != s_jk) = theta/pi; then Ham ~ Binom(ell, theta/pi),
    so one replicate finds the pair with probability F_Binom(d; ell, p)."""
    th = theta_over_pi * math.pi
    X = np.array([[1, 0, 0], [math.cos(th), math.sin(th), 0]], dtype=np.float64)
    Qd, ell, d = 3000, 64, 4
    R = W.gaussian_R(Qd, 3, ell, 99)
    S = oracle.project(X, R)
    h = np.array([int(sum(bin(int(a ^ b)).count("1") for a, b in zip(S[q, 0], S[q, 1])))
                  for q in range(Qd)])
    rate = h.sum() / (Qd * ell)
    sd = math.sqrt(theta_over_pi * (1 - theta_over_pi) / (Qd * ell))
    assert abs(rate - theta_over_pi) < 5 * sd
    hit = (h <= d).mean()
    want = stats.binom.cdf(d, ell, theta_over_pi)
    assert abs(hit - want) < 5 * math.sqrt(want * (1 - want) / Qd) + 1e-12


# ----------------------------------------------------------------- Hamming

def test_golden_fig2c_pool(golden_dir):
    kv, strings, pairs = _read_golden(os.path.join(golden_dir, "fig2c_blockwise.txt"))
    ell, k, d = int(kv["ell"][0]), int(kv["k"][0]), int(kv["d"][0])
    S = _bits_to_words(strings, ell)
    assert _pairs_set(oracle.ham_pairs(S, ell, d)) == set(pairs)
    got, st = oracle.msm(S[None], ell, k, d)
    assert _pairs_set(got) == set(pairs)
    assert st["masks"] == int(kv["block_sorts"][0]) == math.comb(k, d)
    gp, sorts = oracle.msm_positions(S, ell, d)
    assert _pairs_set(gp) == set(pairs)
    assert sorts == int(kv["position_sorts"][0]) == math.comb(ell, d)


@pytest.mark.parametrize("ell,d", [(10, 2), (64, 5), (100, 20), (200, 60)])
def test_ham_pairs_vs_numpy(ell, d):
    S = W.random_strings(150, ell, 1, ell + d, n_centres=6, flip=0.08)[0]
    H = _ham_numpy(S)[:, :]
    n = S.shape[0]
    want = {(i, j) for i in range(n) for j in range(i + 1, n) if H[i, j] <= d}
    assert _pairs_set(oracle.ham_pairs(S, ell, d)) == want


# ---------------------------------------------------------------- blockwise

CASES = [  # ell, k, d, Q, n, centres, flip
    (16, 4, 2, 1, 200, 8, 0.1),
    (64, 8, 4, 2, 400, 12, 0.04),
    (64, 8, 0, 3, 300, 30, 0.0),
    (96, 8, 4, 2, 300, 10, 0.03),
    (128, 10, 6, 2, 300, 10, 0.03),
    (130, 7, 3, 2, 250, 10, 0.02),
    (200, 12, 8, 1, 200, 8, 0.03),
    (256, 9, 4, 1, 150, 8, 0.01),
    (33, 33, 3, 2, 200, 20, 0.05),
    (40, 5, 1, 2, 300, 40, 0.02),
    (32, 4, 3, 2, 300, 10, 0.1),    # d = k - 1: one kept block per grouping
    (64, 8, 4, 2, 2, 1, 0.0),       # two equal strings
    (64, 8, 4, 1, 1, 1, 0.0),       # a single string: no pairs
]


@pytest.mark.parametrize("ell,k,d,Q,n,nc,flip", CASES)
def test_msm_equals_union_of_bruteforce(ell, k, d, Q, n, nc, flip):
    """E = E_1 u ... u E_Q with E_q of Eq. 5 computed by definition; every
    pair reported exactly once (pigeonhole argument of Sec. 2.1 plus the
    Appendix de-duplication)."""
    S = W.random_strings(n, ell, Q, 17 * ell + k + d, n_centres=nc, flip=flip)
    got, st = oracle.msm(S, ell, k, d)
    want = set()
    for q in range(Q):
        want |= _pairs_set(oracle.ham_pairs(S[q], ell, d))
    assert len(got) == len(set(got.tolist()))          # each pair once
    assert _pairs_set(got) == want
    assert st["masks"] == Q * math.comb(k, d)
    assert np.all(np.diff(got.astype(np.int64)) > 0) or len(got) < 2


@pytest.mark.parametrize("ell,k,d,Q,n,nc,flip", CASES[:6])
def test_msm_group_checks_count(ell, k, d, Q, n, nc, flip):
    """The pairs inspected inside groups: sum over replicates and masks of
    sum over groups of equal kept blocks of C(size, 2), recounted with
    numpy.unique on the unpacked bits."""
    S = W.random_strings(n, ell, Q, 17 * ell + k + d, n_centres=nc, flip=flip)
    _, st = oracle.msm(S, ell, k, d)
    bounds = [(b * ell // k, (b + 1) * ell // k) for b in range(k)]
    total = 0
    for q in range(Q):
        bits = np.unpackbits(S[q].view(np.uint8), axis=1, bitorder="little")[:, :ell]
        for K in itertools.combinations(range(k), k - d):
            cols = np.concatenate([np.arange(*bounds[b]) for b in K])
            _, cnt = np.unique(bits[:, cols], axis=0, return_counts=True)
            total += int((cnt * (cnt - 1) // 2).sum())
    assert st["checks"] == total


@pytest.mark.parametrize("ell,k,d,Q,n,nc,flip", CASES[:6])
def test_msm_checks_equal_pairwise_block_agreements(ell, k, d, Q, n, nc, flip):
    """The same count seen pair by pair: a pair shares a group under kept set
    K iff all blocks of K agree, so it is inspected C(e, k - d) times in a
    replicate where e of its k blocks agree (Sec. 2.2); summed over pairs and
    replicates this must equal the oracle's count of in-group inspections."""
    S = W.random_strings(n, ell, Q, 17 * ell + k + d, n_centres=nc, flip=flip)
    _, st = oracle.msm(S, ell, k, d)
    bounds = [(b * ell // k, (b + 1) * ell // k) for b in range(k)]
    iu, ju = np.triu_indices(n, 1)
    total = 0
    for q in range(Q):
        bits = np.unpackbits(S[q].view(np.uint8), axis=1, bitorder="little")[:, :ell]
        e = np.zeros(len(iu), dtype=np.int64)
        for lo, hi in bounds:
            e += np.all(bits[iu, lo:hi] == bits[ju, lo:hi], axis=1)
        binom = np.array([math.comb(v, k - d) for v in range(k + 1)], dtype=np.int64)
        total += int(binom[e].sum())
    assert st["checks"] == total


def test_msm_d0_is_equivalence_classes():
    """d = 0 (Sec. 2.1, Fig. 1): pairs of identical strings."""
    S = W.random_strings(500, 48, 1, 3, n_centres=40, flip=0.0)
    got, _ = oracle.msm(S, 48, 6, 0)
    groups = {}
    for i, row in enumerate(S[0]):
        groups.setdefault(tuple(int(v) for v in row), []).append(i)
    want = {(a, b) for g in groups.values() for a, b in itertools.combinations(g, 2)}
    assert _pairs_set(got) == want


def test_msm_k_equals_ell_is_position_masking():
    ell, d = 12, 2
    S = W.random_strings(120, ell, 1, 8, n_centres=5, flip=0.15)
    a, st = oracle.msm(S, ell, ell, d)
    b, sorts = oracle.msm_positions(S[0], ell, d)
    assert np.array_equal(a, b)
    assert st["masks"] == sorts == math.comb(ell, d)


def test_msm_replicate_dedup_first_replicate_wins():
    """Appendix: a pair is added in replicate h only if no g < h has
    Hamming <= d; with identical pools every pair comes from replicate 0,
    so the result equals the single-pool result."""
    S1 = W.random_strings(300, 64, 1, 21, n_centres=10, flip=0.04)
    S3 = np.concatenate([S1, S1, S1], axis=0)
    a, sa = oracle.msm(S1, 64, 8, 4)
    b, sb = oracle.msm(S3, 64, 8, 4)
    assert np.array_equal(a, b)
    assert sb["checks"] == 3 * sa["checks"]


# ---------------------------------------------------------------- distances

def test_distance_closed_forms():
    x = np.array([3.0, 4.0, 0.0])
    y = np.array([0.0, 0.0, 2.0])
    assert oracle.distance(x, x, COS) == pytest.approx(0.0, abs=1e-15)
    assert oracle.distance(x, -x, COS) == pytest.approx(2.0, abs=1e-15)
    assert oracle.distance(x, y, COS) == pytest.approx(1.0, abs=1e-15)
    assert oracle.distance(x, 7.5 * x, COS) == pytest.approx(0.0, abs=1e-15)
    assert oracle.distance(x, np.zeros(3), EUC) == 5.0       # 3-4-5
    assert oracle.distance(x, y, EUC) == pytest.approx(math.sqrt(29.0), rel=1e-15)
    for th in [0.01, 0.3, 1.0, 2.5]:
        a = np.array([1.0, 0.0])
        b = np.array([math.cos(th), math.sin(th)])
        assert oracle.distance(a, b, COS) == pytest.approx(1 - math.cos(th), rel=1e-12, abs=1e-15)
        # unit vectors: |a-b|^2 = 2 * cosine distance (Sec. 5.1)
        assert oracle.distance(a, b, EUC) ** 2 == pytest.approx(2 * oracle.distance(a, b, COS), rel=1e-12)


def test_dist_vs_numpy():
    X = W.clustered(300, 40, 6, 0.2, 3, normalise=False).astype(np.float64)
    rng = np.random.default_rng(0)
    i = rng.integers(0, 300, 2000)
    j = rng.integers(0, 300, 2000)
    lo, hi = np.minimum(i, j), np.maximum(i, j)
    keep = lo < hi
    lo, hi = lo[keep], hi[keep]
    pairs = (lo.astype(np.uint64) << np.uint64(32)) | hi.astype(np.uint64)
    nrm = np.linalg.norm(X, axis=1)
    cos_np = 1 - np.einsum("ij,ij->i", X[lo], X[hi]) / (nrm[lo] * nrm[hi])
    euc_np = np.linalg.norm(X[lo] - X[hi], axis=1)
    assert np.allclose(oracle.dist(X, pairs, COS), cos_np, rtol=1e-12, atol=1e-14)
    assert np.allclose(oracle.dist(X, pairs, EUC), euc_np, rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("metric,eps", [(COS, 0.05), (EUC, 0.4)])
def test_eps_bruteforce_vs_numpy(metric, eps):
    X = W.clustered(400, 16, 8, 0.08, 4, normalise=True)
    Xd = X.astype(np.float64)
    if metric == COS:
        nrm = np.linalg.norm(Xd, axis=1)
        Dm = 1 - (Xd @ Xd.T) / np.outer(nrm, nrm)
    else:
        Dm = np.linalg.norm(Xd[:, None, :] - Xd[None, :, :], axis=2)
    iu = np.triu_indices(400, 1)
    vals = Dm[iu]
    safe = np.abs(vals - eps) > 1e-9
    want = {(a, b) for a, b, v, s in zip(iu[0], iu[1], vals, safe) if s and v <= eps}
    got, dv = oracle.eps_bruteforce(X, metric, eps)
    gs = _pairs_set(got)
    unsure = {(a, b) for a, b, s in zip(iu[0], iu[1], safe) if not s}
    assert gs - unsure == want
    assert np.all(dv <= eps)


# ------------------------------------------------------------------- bound

def test_eps_angle_golden(golden_dir):
    with open(os.path.join(golden_dir, "eps_angle.txt")) as f:
        rows = [l.split() for l in f if l.strip() and not l.startswith("#")]
    for eps, ang in rows:
        # printed radii have three significant digits
        assert oracle.p_cosine(float(eps)) == pytest.approx(float(ang), abs=2e-3)


def test_bound_matches_binomial_survival():
    for ell, d, p in [(50, 0, 0.1), (50, 3, 0.1), (128, 6, 0.04), (64, 4, 0.12)]:
        assert oracle.miss_bound(ell, d, p, 1) == pytest.approx(stats.binom.sf(d, ell, p), rel=1e-9)
        assert oracle.miss_bound(ell, d, p, 7) == pytest.approx(stats.binom.sf(d, ell, p) ** 7, rel=1e-9)
    # d = ell: every replicate finds the pair; 1 - sum rounds to ~1e-16
    assert oracle.miss_bound(20, 20, 0.3, 3) < 1e-40
    assert oracle.miss_bound(20, 0, 0.0, 3) == 0.0


def test_solve_Q_minimal_and_fig3_trend():
    p, ell, gamma = 0.1, 50, 1e-6
    prev = None
    for d in range(0, 8):
        Q = oracle.solve_Q(ell, d, p, gamma)
        assert oracle.miss_bound(ell, d, p, Q) <= gamma
        assert Q == 1 or oracle.miss_bound(ell, d, p, Q - 1) > gamma
        if prev is not None:
            assert Q < prev          # Sec. 4.2: Q falls quickly as d grows
        prev = Q
    assert oracle.solve_Q(ell, 0, p, gamma) > 1000   # "many replicates ... when d = 0"


def test_missing_ratio_statistics_planted_angle():
    """Per-pair miss probability over Q replicates is (1 - F_Binom(d))^Q."""
    th = 0.09 * math.pi
    X = np.array([[1, 0, 0], [math.cos(th), math.sin(th), 0]])
    ell, d, Q, trials = 32, 2, 2, 4000
    R = W.gaussian_R(Q * trials, 3, ell, 7)
    S = oracle.project(X, R)
    x = S[:, 0, 0] ^ S[:, 1, 0]
    h = np.array([bin(int(v)).count("1") for v in x]).reshape(trials, Q)
    missed = np.all(h > d, axis=1).mean()
    want = oracle.miss_bound(ell, d, 0.09, Q)
    assert abs(missed - want) < 5 * math.sqrt(want * (1 - want) / trials)


# --------------------------------------------------------------- end to end

def test_eps_graph_no_false_positives_and_recall():
    wl = W.Workload("t", 1500, 32, 15, 0.05, "cosine", 0.15, 64, 8, 4, "f32", 5, 6)
    X = W.clustered(wl.n, wl.dim, wl.n_clusters, wl.sigma, wl.data_seed)
    p = oracle.p_cosine(wl.eps)
    Q = oracle.solve_Q(wl.ell, wl.d, p, 1e-2)
    R = W.gaussian_R(Q, wl.dim, wl.ell, wl.r_seed)
    pairs, dv, info = oracle.eps_graph(X, R, wl.ell, wl.k, wl.d, COS, wl.eps)
    truth, tdv = oracle.eps_bruteforce(X, COS, float(np.float32(wl.eps)))
    got, tru = _pairs_set(pairs), _pairs_set(truth)
    assert got <= tru                                     # type-I removed
    missing = len(tru - got) / max(1, len(tru))
    assert missing <= 1e-2
    assert info["type1"] == info["cand"] - len(pairs)
    assert np.all(dv <= np.float32(wl.eps))


def test_eps_bruteforce_inclusive_boundary():
    """Def. 1.1 keeps pairs with distance exactly eps."""
    X = np.array([[0.0, 0.0], [3.0, 4.0], [6.0, 8.0], [1.0, 0.0]])
    got, dv = oracle.eps_bruteforce(X, EUC, 5.0)
    assert _pairs_set(got) == {(0, 1), (1, 2), (1, 3), (0, 3)}
    Xc = np.array([[1.0, 0.0], [0.0, 2.0], [-1.0, 0.0]])
    got, dv = oracle.eps_bruteforce(Xc, COS, 1.0)      # orthogonal: exactly 1
    assert _pairs_set(got) == {(0, 1), (1, 2)}


# ------------------------------------------------ Sec. 4.3 parameter rule

def test_choose_params_hand_worked():
    """n = 1024 -> l = 2 * 10 = 20; p = 0.1, gamma = 1e-6, S = 1e6 -> the
    replicate limit is 24.  P(Binom(20, 0.1) <= 1) = 0.9^20 + 2 * 0.9^19 =
    0.39175 -> Q = ceil(ln 1e-6 / ln 0.60825) = 28 > 24; P(<= 2) adds
    190 * 0.01 * 0.9^18 = 0.28518 -> 0.67693 -> Q = ceil(13.8155 / 1.1299)
    = 13.  So d = 2, k = 4, Q = 13."""
    assert oracle.choose_params(1024, 0.1, 1e-6, 1e6) == (20, 4, 2, 13)


def test_choose_params_halves_l_when_no_output():
    """S < 1: l = 10, limit 5.  P(Binom(10, 0.1) <= 2) = 0.92981 ->
    Q = ceil(13.8155 / 2.6565) = 6 > 5; P(<= 3) = 0.98720 -> Q = 4."""
    assert oracle.choose_params(1024, 0.1, 1e-6, 0.5) == (10, 6, 3, 4)


@pytest.mark.parametrize("n,p,S", [(5000, 0.12, 1e5), (1 << 20, 0.1436, 5e8),
                                   (123457, 0.05, 10.0), (3, 0.2, 2.0)])
def test_choose_params_is_minimal(n, p, S):
    ell, k, d, Q = oracle.choose_params(n, p, 1e-6, S)
    assert ell == min(256, 2 * math.ceil(math.log2(n)) // (1 if S >= 1 else 2))
    assert k == (2 * d if d else 1)
    limit = min(24, max(math.ceil(30 * S / n), 5))
    assert Q <= limit and Q == oracle.solve_Q(ell, d, p, 1e-6)
    if d > 0:  # one mismatch fewer needs more replicates than allowed
        assert oracle.solve_Q(ell, d - 1, p, 1e-6) > limit


def test_choose_params_replicate_budget_is_24():
    """n = 1024 (l = 20), p = 0.1434, large S: P(Binom(20, p) <= 2) =
    0.8566^20 + 20 p 0.8566^19 + 190 p^2 0.8566^18 = 0.0452 + 0.1514 + 0.2407
    = 0.4373, so d = 2 needs Q = ceil(13.8155 / 0.5750) = 25 -- one more than
    the budget (below 25) allows; the rule moves on to d = 3."""
    assert oracle.solve_Q(20, 2, 0.1434, 1e-6) == 25
    assert oracle.choose_params(1024, 0.1434, 1e-6, 1e9) == (20, 6, 3, 13)
