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
