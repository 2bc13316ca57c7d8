"""Seeded synthetic inputs shared by the tests, the CPU oracle and bench.py.

This module only draws random numbers and shapes them into the workloads the
method is evaluated on; it holds none of the method's arithmetic (no
projection, no string handling, no distances).  Both the CUDA path and the
oracle consume what it produces, so neither depends on the other.

Workload recipe (stand-in for the 1.6M Tiny Images set of Sec. 5.2, which is
not available here): cluster centres drawn uniformly from [-1, 1]^D, every
point picks a centre uniformly at random and adds isotropic Gaussian noise
of standard deviation sigma; for the cosine workloads (and the Euclidean one,
read on unit vectors as in Sec. 5.1) each point is then scaled to unit norm.
The projection matrix R of Eq. 3 is i.i.d. N(0, 1), one D x ell block per
replicate, laid out [Q][D][ell].
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


@dataclasses.dataclass(frozen=True)
class Workload:
    """One evaluated configuration of the method."""
    name: str
    n: int
    dim: int
    n_clusters: int
    sigma: float
    metric: str          # "cosine" or "euclidean"
    eps: float
    ell: int
    k: int
    d: int
    dtype: str           # storage type of X: "f32", "bf16" or "fp8e4m3"
    data_seed: int
    r_seed: int
    normalise: bool = True
    # batched form: n_sets independent sets, sizes log-uniform in
    # [set_min, set_max], n_clusters clusters in each set
    n_sets: int = 1
    set_min: int = 0
    set_max: int = 0

    @property
    def masks(self) -> int:
        return math.comb(self.k, self.d)


# The five evaluated configurations.  "small" is the case the CPU oracle
# finishes in seconds; "scale" is the 1M x 128 workload the headline
# throughput is quoted on.  For "batched" n is the expected total over the
# sets (the actual sizes come from set_sizes).
WORKLOADS = {
    "small": Workload("small", 20_000, 64, 50, 0.05, "cosine", 0.15, 64, 8, 4,
                      "f32", 1001, 2001),
    "scale": Workload("scale", 1_000_000, 128, 1_000, 0.05, "cosine", 0.10,
                      128, 10, 6, "f32", 1002, 2002),
    "precision": Workload("precision", 4_000_000, 256, 4_000, 0.05,
                          "euclidean", 0.30, 128, 12, 8, "bf16", 1003, 2003),
    "batched": Workload("batched", 9_600_000, 96, 20, 0.05, "cosine", 0.12, 64, 8, 4,
                        "f32", 1004, 2004, n_sets=256, set_min=1_000, set_max=200_000),
    "learned": Workload("learned", 8_000_000, 128, 10_000, 0.05, "cosine",
                        0.10, 96, 8, 4, "bf16", 1005, 2005),
}


def clustered(n: int, dim: int, n_clusters: int, sigma: float, seed: int,
              normalise: bool = True, chunk: int = 1 << 18,
              centres_seed: int | None = None) -> np.ndarray:
    """Gaussian-mixture points, float32 [n][dim], generated in chunks.

    Centres ~ U[-1,1]^dim; each point's centre is uniform over the mixture;
    noise ~ sigma * N(0, I).  With ``normalise`` every row is scaled to unit
    Euclidean norm (the normalisation used for the cosine experiments).
    ``centres_seed`` draws the centres from another stream, so samples with
    different ``seed`` share one mixture.
    """
    rng = np.random.default_rng(seed)
    centres = rng.uniform(-1.0, 1.0, size=(n_clusters, dim))
    if centres_seed is not None and centres_seed != seed:
        centres = np.random.default_rng(centres_seed).uniform(-1.0, 1.0, size=(n_clusters, dim))
    out = np.empty((n, dim), dtype=np.float32)
    for s in range(0, n, chunk):
        e = min(n, s + chunk)
        lab = rng.integers(0, n_clusters, size=e - s)
        x = centres[lab] + sigma * rng.standard_normal((e - s, dim))
        if normalise:
            x /= np.linalg.norm(x, axis=1, keepdims=True)
        out[s:e] = x
    return out


def clustered_split(n_first: int, n_second: int, dim: int, n_clusters: int,
                    sigma: float, seed: int, normalise: bool = True):
    """Two disjoint samples of the same mixture (same centres): the first
    n_first and the next n_second points of one draw."""
    X = clustered(n_first + n_second, dim, n_clusters, sigma, seed, normalise)
    return X[:n_first], X[n_first:]


def set_sizes(n_sets: int, lo: int, hi: int, seed: int) -> np.ndarray:
    """Sizes of the batched form's point sets: floor(exp(U[ln lo, ln hi]))."""
    rng = np.random.default_rng(seed)
    return np.floor(np.exp(rng.uniform(np.log(lo), np.log(hi), n_sets))).astype(np.int64)


def clustered_sets(sizes, dim: int, n_clusters: int, sigma: float, seed: int,
                   normalise: bool = True):
    """Independent point sets, each a mixture of its own n_clusters centres
    (drawn as in ``clustered`` from the stream [seed, s]), concatenated.
    Returns (X float32 [sum(sizes)][dim], offsets int64 [len(sizes) + 1])."""
    sizes = np.asarray(sizes, dtype=np.int64)
    off = np.zeros(len(sizes) + 1, dtype=np.int64)
    off[1:] = np.cumsum(sizes)
    X = np.empty((int(off[-1]), dim), dtype=np.float32)
    for s, m in enumerate(sizes):
        if m == 0:
            continue
        rng = np.random.default_rng([seed, s])
        centres = rng.uniform(-1.0, 1.0, size=(n_clusters, dim))
        lab = rng.integers(0, n_clusters, size=int(m))
        x = centres[lab] + sigma * rng.standard_normal((int(m), dim))
        if normalise:
            x /= np.linalg.norm(x, axis=1, keepdims=True)
        X[off[s]:off[s + 1]] = x
    return X, off


def cluster_labels(n: int, n_clusters: int, seed: int, dim: int,
                   chunk: int = 1 << 18) -> np.ndarray:
    """The mixture component of every point drawn by ``clustered`` (same seed)."""
    rng = np.random.default_rng(seed)
    rng.uniform(-1.0, 1.0, size=(n_clusters, dim))
    lab_all = np.empty(n, dtype=np.int64)
    for s in range(0, n, chunk):
        e = min(n, s + chunk)
        lab_all[s:e] = rng.integers(0, n_clusters, size=e - s)
        rng.standard_normal((e - s, dim))
    return lab_all


def gaussian_R(Q: int, dim: int, ell: int, seed: int) -> np.ndarray:
    """Projection matrices of Eq. 3: float32 [Q][dim][ell], i.i.d. N(0, 1)."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal((Q, dim, ell)).astype(np.float32)


def random_strings(n: int, ell: int, Q: int, seed: int,
                   n_centres: int = 0, flip: float = 0.0) -> np.ndarray:
    """Packed bit strings uint64 [Q][n][ceil(ell/64)], bit j in word j>>6.

    With ``n_centres`` > 0 every string copies one of ``n_centres`` random
    centre strings and flips each bit independently with probability
    ``flip`` (clustered pools with many small Hamming distances); otherwise
    every bit is a fair coin.  Bits at positions >= ell are zero.
    """
    rng = np.random.default_rng(seed)
    W = (ell + 63) // 64
    if n_centres > 0:
        centres = rng.integers(0, 2, size=(n_centres, ell), dtype=np.uint8)
        lab = rng.integers(0, n_centres, size=(Q, n))
        bits = centres[lab]
        bits ^= (rng.random((Q, n, ell)) < flip).astype(np.uint8)
    else:
        bits = rng.integers(0, 2, size=(Q, n, ell), dtype=np.uint8)
    padded = np.zeros((Q, n, W * 64), dtype=np.uint8)
    padded[:, :, :ell] = bits
    weights = (np.uint64(1) << np.arange(64, dtype=np.uint64))
    words = padded.reshape(Q, n, W, 64).astype(np.uint64) * weights
    return np.bitwise_or.reduce(words, axis=3)


def clustered_words(n: int, W: int, seed: int, n_centres: int, and_depth: int) -> np.ndarray:
    """Packed strings uint64 [1][n][W] of 64 W bits: every string copies one
    of ``n_centres`` random centre strings and flips each bit with
    probability 2^-and_depth (the AND of ``and_depth`` random words), drawn
    word-wise so that millions of strings stay cheap."""
    rng = np.random.default_rng(seed)
    centres = rng.integers(0, 2 ** 63, size=(n_centres, W), dtype=np.uint64) << np.uint64(1)
    centres ^= rng.integers(0, 2, size=(n_centres, W), dtype=np.uint64)
    out = centres[rng.integers(0, n_centres, size=n)]
    flips = np.full((n, W), np.uint64(0xFFFFFFFFFFFFFFFF), dtype=np.uint64)
    for _ in range(and_depth):
        flips &= (rng.integers(0, 2 ** 63, size=(n, W), dtype=np.uint64) << np.uint64(1)) | \
            rng.integers(0, 2, size=(n, W), dtype=np.uint64)
    return (out ^ flips)[None]


def to_bf16_values(x: np.ndarray) -> np.ndarray:
    """Round float32 values to the nearest bfloat16 (ties to even), returned
    as float32 holding exactly those bfloat16 values."""
    b = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    rounding = ((b >> 16) & 1) + 0x7FFF
    r = ((b + rounding) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).reshape(x.shape)
