"""Missing-edge-ratio bound of Sec. 4.2 and the replicate count it implies.

TEST INFRASTRUCTURE ONLY (part of the CPU oracle).  Plain double precision.
"""
from __future__ import annotations

import math


def p_cosine(eps: float) -> float:
    """Non-collision probability of one sign bit for a pair at cosine
    distance exactly eps: arccos(1 - eps) / pi (Sec. 4.2, with Eq. 4)."""
    return math.acos(1.0 - eps) / math.pi


def p_euclidean(eps: float) -> float:
    """The same for unit vectors at Euclidean distance eps: on the unit
    sphere |x - y|^2 = 2 * (cosine distance) (Sec. 5.1), so the cosine
    radius is eps^2 / 2."""
    return math.acos(1.0 - 0.5 * eps * eps) / math.pi


def e2lsh_p(w: float) -> float:
    """Non-collision probability of one E2LSH symbol floor(r^T x / W + u)
    (r ~ N(0, I), u ~ U[0, 1)) for a pair at Euclidean distance c = W / w,
    i.e. with the bucket width W = w times the distance.  r^T (x - y) ~ c N(0,1),
    and a uniform offset separates two values a distance s apart with
    probability min(s / W, 1), so the collision probability is
      integral over s >= 0 of 2 phi(s / c) / c * max(0, 1 - s / W) ds
      = 1 - 2 Phi(-w) - 2 / (sqrt(2 pi) w) (1 - exp(-w^2 / 2))
    (Datar et al. 2004).  Returns 1 minus that."""
    phi_neg = 0.5 * math.erfc(w / math.sqrt(2.0))
    coll = 1.0 - 2.0 * phi_neg - 2.0 / (math.sqrt(2.0 * math.pi) * w) * (1.0 - math.exp(-0.5 * w * w))
    return 1.0 - coll


def miss_bound(ell: int, d: int, p: float, Q: int) -> float:
    """(1 - sum_{t=0}^{floor(d)} C(ell, t) p^t (1-p)^(ell-t))^Q (Sec. 4.2)."""
    hit = math.fsum(math.comb(ell, t) * p ** t * (1.0 - p) ** (ell - t)
                    for t in range(0, int(math.floor(d)) + 1))
    return (1.0 - hit) ** Q


def solve_Q(ell: int, d: int, p: float, gamma: float, q_max: int = 1 << 20) -> int:
    """Smallest Q >= 1 with miss_bound(ell, d, p, Q) <= gamma (Sec. 4.3:
    'finally choose the minimum Q')."""
    for Q in range(1, q_max + 1):
        if miss_bound(ell, d, p, Q) <= gamma:
            return Q
    raise ValueError("no Q up to q_max meets gamma")


def choose_params(n: int, p: float, gamma: float, S: float):
    """Sec. 4.3: pick l first, then d, then the minimum Q.

    l is twice the number of bits that index n points (so that the k - d
    kept blocks can hold log2 n letters), halved when the estimated output S
    is close to 0 (read as S < 1); the number of replicates is limited to
    max(30 S / n, 5) and kept below 25; d is the smallest value whose minimum
    Q meets gamma within that limit; k = 2d is the fewest blocks for which
    k - d blocks hold half of the string (k = 1 when d = 0).
    Returns (l, k, d, Q)."""
    ell = 2 * math.ceil(math.log2(n)) if n > 1 else 0
    if S < 1.0:
        ell //= 2
    ell = min(max(ell, 1), 256)
    limit = min(24, max(math.ceil(30.0 * S / n), 5))
    d = 0
    while True:
        k = 2 * d if d > 0 else 1
        if k > ell or k > 32:
            raise ValueError("no d meets the replicate limit")
        try:
            Q = solve_Q(ell, d, p, gamma, q_max=limit)
        except ValueError:
            Q = None
        if Q is not None:
            return ell, k, d, Q
        d += 1
