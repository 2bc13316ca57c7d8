"""The pair check's work decomposition, replayed on the CPU: within each group
of equal kept blocks (Sec. 2.2) the members are ordered by their first gap
block (the sub-key), runs of more than 32 members are cut into 32 x 32 tiles
of the upper triangle, and a tile (or a run of at most 32) whose first and
last member carry the same sub-key is skipped, since every pair in it is
equal on a gap block and the first-mask rule can never report it under this
kept set.  Inside an off-diagonal tile that is not skipped, the reference
prefilter picks for every gap block the most frequent value among the
tile's 32 column lanes (ties: the highest lane, as the warp reduction does;
lanes past the last column hold a value no block can have) and drops each
pair whose two members both carry that value on some gap block.  A diagonal
tile (rows = columns, which includes every run of at most 32 members) drops
every pair equal on some gap block, since its warp matches the values of
all its lanes.  These tests check that no step ever drops a pair the method
reports, and count the pairs left to evaluate."""
import itertools

import numpy as np
import pytest

import oracle
import workloads as W


def _block_values(Sq, ell, k):
    bits = np.unpackbits(Sq.view(np.uint8), axis=1, bitorder="little")[:, :ell]
    bv = np.zeros((Sq.shape[0], k), dtype=np.int64)
    for b in range(k):
        lo, hi = b * ell // k, (b + 1) * ell // k
        bv[:, b] = (bits[:, lo:hi].astype(np.int64) << np.arange(hi - lo, dtype=np.int64)).sum(1)
    return bits, bv


def _replay(S, ell, k, d, prefilter=True):
    """Per (replicate, kept set): in-group pairs, evaluated pairs and the set
    of evaluated point pairs, following the tile rule (and the reference
    prefilter)."""
    Q, n, _ = S.shape
    r = k - d
    ingroup = evaluated = 0
    kept = {}
    for q in range(Q):
        _, bv = _block_values(S[q], ell, k)
        for K in itertools.combinations(range(k), r):
            gaps = [b for b in range(max(K)) if b not in K]
            _, gid = np.unique(bv[:, list(K)], axis=0, return_inverse=True)
            gid = gid.ravel()
            sub = bv[:, gaps[0]] if gaps else np.zeros(n, dtype=np.int64)
            order = np.lexsort((np.arange(n), sub, gid))
            gs, ks = gid[order], sub[order]
            starts = np.flatnonzero(np.r_[True, gs[1:] != gs[:-1]])
            ends = np.r_[starts[1:], n]
            ev = set()
            for st, en in zip(starts, ends):
                L = int(en - st)
                if L < 2:
                    continue
                ingroup += L * (L - 1) // 2
                mem, key = order[st:en], ks[st:en]
                tiles = [(0, L, 0, L)] if L <= 32 else [
                    (32 * I, min(L, 32 * I + 32), 32 * J, min(L, 32 * J + 32))
                    for J in range((L + 31) // 32) for I in range(J + 1)]
                gv = bv[mem][:, gaps]
                for r0, r1, c0, c1 in tiles:
                    if gaps and key[r0] == key[c1 - 1]:
                        continue
                    drop = np.zeros((r1 - r0, c1 - c0), dtype=bool)
                    if prefilter and r0 == c0:  # diagonal: every equal gap block
                        for gi in range(len(gaps)):
                            drop |= gv[r0:r1, gi][:, None] == gv[c0:c1, gi][None, :]
                    elif prefilter:
                        for gi in range(len(gaps)):
                            ref = _ref_mode(gv[c0:c1, gi], c1 - c0)
                            drop |= ((gv[r0:r1, gi] == ref)[:, None] &
                                     (gv[c0:c1, gi] == ref)[None, :])
                    for a in range(r0, r1):
                        for b in range(max(c0, a + 1), c1):
                            if not drop[a - r0, b - c0]:
                                ev.add((min(mem[a], mem[b]), max(mem[a], mem[b])))
            evaluated += len(ev)
            kept[(q, K)] = ev
    return ingroup, evaluated, kept


def _ref_mode(vals, n):
    """The reference value of one gap block: lanes 0..31 hold the sampled
    column values (lanes >= n hold a value no block can have), and the lane
    with the most equal peers wins, ties to the highest lane."""
    lanes = [int(vals[i]) if i < n else -1 - i for i in range(32)]
    score = [(lanes.count(v), i) for i, v in enumerate(lanes)]
    return lanes[max(score)[1]]


def _strings(ell, k, Q, n, nc, flip):
    if nc:
        return W.random_strings(n, ell, Q, 31 * ell + k, n_centres=nc, flip=flip)
    # clustered points of the scale workload's geometry (D = 128, sigma 0.05)
    X = W.clustered(n, 128, 2, 0.05, 1002)
    return oracle.project(X, W.gaussian_R(Q, 128, ell, 2002))


# groups of hundreds of members, so that runs span many tiles and tiles mix
# sub-keys (a rule that looked at the rows alone would drop pairs here)
@pytest.mark.parametrize("ell,k,d,Q,n,nc,flip", [
    (64, 8, 4, 2, 300, 3, 0.04),
    (48, 6, 3, 2, 500, 2, 0.06),
    (64, 8, 4, 1, 600, 1, 0.05),
    (128, 10, 6, 2, 600, 0, 0.0),
])
def test_subkey_skip_keeps_every_reported_pair(ell, k, d, Q, n, nc, flip):
    S = _strings(ell, k, Q, n, nc, flip)
    ingroup, evaluated, kept = _replay(S, ell, k, d)
    got, st = oracle.msm(S, ell, k, d)
    # the replay sees the same groups as the oracle
    assert ingroup == st["checks"]
    assert evaluated <= ingroup
    # every reported pair lies in an evaluated tile of the replicate and the
    # kept set that report it: the first replicate within distance d, and
    # its k - d lowest-index agreeing blocks
    blocks = [_block_values(S[q], ell, k) for q in range(Q)]
    i_all, j_all = oracle.unpack_pairs(got)
    for i, j in zip(i_all.tolist(), j_all.tolist()):
        for q in range(Q):
            bits, bv = blocks[q]
            if int((bits[i] != bits[j]).sum()) <= d:
                break
        eq = [b for b in range(k) if bv[i, b] == bv[j, b]]
        K = tuple(eq[:k - d])
        assert (i, j) in kept[(q, K)], (i, j, q, K)


def test_subkey_skips_pairs_on_clustered_points():
    """On the strings of clustered points (the scale workload's geometry at
    a small size: D = 128, sigma = 0.05, ell = 128, k = 10, d = 6, clusters
    of ~300 points) the skip removes a share of the in-group pairs; the share
    grows with the cluster size (about half at 1000 points per cluster).
    With the prefilters the pairs left fall close to the pairs whose kept set
    is their first (about 4 % of the in-group pairs at 1000 points per
    cluster, against a floor of 3.4 %)."""
    X = W.clustered(600, 128, 2, 0.05, 1002)
    R = W.gaussian_R(1, 128, 128, 2002)
    S = oracle.project(X, R)
    ingroup, evaluated, _ = _replay(S, 128, 10, 6, prefilter=False)
    assert ingroup > 0 and evaluated < 0.95 * ingroup
    ingroup2, evaluated2, _ = _replay(S, 128, 10, 6)
    assert ingroup2 == ingroup and evaluated2 < 0.15 * ingroup
