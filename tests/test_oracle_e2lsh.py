"""Pins of the oracle's E2LSH symbol strings (no GPU): the collision
probability against simulation, the projection against closed forms and
numpy, symbol mismatch counts against numpy, and the symbol MSM against
brute force and against the (separately pinned) bit-string MSM."""
import math

import numpy as np
import pytest

import oracle
import workloads as W


@pytest.mark.parametrize("w", [0.5, 1.0, 3.5, 12.0])
def test_e2lsh_collision_probability_matches_simulation(w):
    """Two points at Euclidean distance c = 1, bucket width W = w:
    symbols floor(r.x / W + u) with r ~ N(0, I), u ~ U[0, 1)."""
    rng = np.random.default_rng(int(w * 100))
    m = 400_000
    D = 8
    r = rng.standard_normal((m, D))
    u = rng.random(m)
    y = np.zeros(D)
    y[3] = 1.0                                  # |x - y| = 1 with x = 0
    same = np.floor(0.0 / w + u) == np.floor(r @ y / w + u)
    f = same.mean()
    want = 1.0 - oracle.e2lsh_p(w)
    assert abs(f - want) < 5 * math.sqrt(want * (1 - want) / m) + 1e-12


def test_e2lsh_probability_limits():
    assert oracle.e2lsh_p(1e6) < 1e-5            # wide buckets always collide
    assert oracle.e2lsh_p(1e-6) > 1 - 1e-5       # narrow ones never do
    ws = np.linspace(0.2, 20, 50)
    ps = [oracle.e2lsh_p(x) for x in ws]
    assert all(a > b for a, b in zip(ps, ps[1:]))  # monotone in w


def test_e2lsh_offsets_definition():
    u = oracle.e2lsh_offsets(17, 3, 5)
    assert u.shape == (3, 5) and np.all((u >= 0) & (u < 1))
    for q in range(3):
        for c in range(5):
            w0 = int(oracle.philox([q * 5 + c, 0, 0, 0], [17, 2])[0])
            assert u[q, c] == np.float32((w0 >> 40) * 2.0 ** -24)
    big = oracle.e2lsh_offsets(3, 1, 20000).ravel()
    assert abs(big.mean() - 0.5) < 0.01 and abs(big.var() - 1 / 12) < 0.005


def _unpack_symbols(S, ell, sw):
    """numpy unpacking: symbol c = bits [c sw, (c + 1) sw) of the string."""
    Q, n, Wd = S.shape
    bits = np.unpackbits(np.ascontiguousarray(S).view(np.uint8), axis=-1,
                         bitorder="little").reshape(Q, n, Wd * 64)[:, :, :ell * sw]
    bits = bits.reshape(Q, n, ell, sw).astype(np.int64)
    return (bits * (1 << np.arange(sw))).sum(-1)


@pytest.mark.parametrize("sw", [1, 2, 4])
def test_e2lsh_projection_closed_form_and_numpy(sw):
    rng = np.random.default_rng(sw)
    Q, D, ell = 2, 12, 40
    R = rng.standard_normal((Q, D, ell)).astype(np.float32)
    u = oracle.e2lsh_offsets(9, Q, ell)
    width = 0.75
    # basis vectors: t = R[q][m][c]
    X = np.eye(D, dtype=np.float32)
    S = oracle.project_e2lsh(X, R, u, width, sw)
    sym = _unpack_symbols(S, ell, sw)
    t = np.transpose(R.astype(np.float64), (0, 1, 2))          # [Q][m][c]
    want = np.floor(t / width + u[:, None, :].astype(np.float64)).astype(np.int64) & ((1 << sw) - 1)
    assert np.array_equal(sym, want)
    # random points, away from bucket boundaries
    X = rng.standard_normal((50, D)).astype(np.float32)
    S = oracle.project_e2lsh(X, R, u, width, sw)
    z = np.einsum("nd,qdc->qnc", X.astype(np.float64), R.astype(np.float64)) / width + u[:, None, :]
    ok = np.abs(z - np.round(z)) > 1e-9
    want = np.floor(z).astype(np.int64) & ((1 << sw) - 1)
    assert np.array_equal(_unpack_symbols(S, ell, sw)[ok], want[ok])


def _sym_strings(n, ell, sw, Q, seed, centres=8, flip=0.06):
    rng = np.random.default_rng(seed)
    C = rng.integers(0, 1 << sw, size=(centres, ell))
    lab = rng.integers(0, centres, size=(Q, n))
    sym = C[lab]
    change = rng.random((Q, n, ell)) < flip
    sym = np.where(change, rng.integers(0, 1 << sw, size=(Q, n, ell)), sym)
    Wd = (ell * sw + 63) // 64
    S = np.zeros((Q, n, Wd), dtype=np.uint64)
    for c in range(ell):
        bit = c * sw
        S[:, :, bit // 64] |= sym[:, :, c].astype(np.uint64) << np.uint64(bit % 64)
    return S, sym


@pytest.mark.parametrize("sw", [2, 4])
def test_sym_pairs_match_numpy(sw):
    ell, n = 20, 300
    S, sym = _sym_strings(n, ell, sw, 1, 40 + sw)
    d = 4
    got = oracle.sym_pairs(S[0], ell, sw, d)
    mism = (sym[0][:, None, :] != sym[0][None, :, :]).sum(-1)
    i, j = np.nonzero(np.triu(mism <= d, 1))
    want = (i.astype(np.uint64) << np.uint64(32)) | j.astype(np.uint64)
    assert np.array_equal(got, want)


@pytest.mark.parametrize("sw,ell,k,d,Q", [(2, 24, 6, 3, 2), (4, 16, 8, 4, 2), (4, 30, 10, 5, 1),
                                         (2, 40, 8, 0, 3)])
def test_msm_sym_equals_union_of_brute_force(sw, ell, k, d, Q):
    n = 400
    S, _ = _sym_strings(n, ell, sw, Q, 7 * ell + sw)
    got, st = oracle.msm_sym(S, ell, sw, k, d)
    assert len(np.unique(got)) == len(got)                  # each pair once
    want = np.unique(np.concatenate([oracle.sym_pairs(S[q], ell, sw, d) for q in range(Q)]))
    assert np.array_equal(got, want)
    assert st["masks"] == Q * math.comb(k, d)


def test_msm_sym_with_one_bit_symbols_is_the_bit_msm():
    S = W.random_strings(500, 64, 2, 11, n_centres=10, flip=0.05)
    a, sa = oracle.msm_sym(S, 64, 1, 8, 4)
    b, sb = oracle.msm(S, 64, 8, 4)
    assert np.array_equal(a, b) and sa == sb
