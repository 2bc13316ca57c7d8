"""Host-side checks of two numerical claims the CUDA kernels rest on, replayed
in numpy with the kernels' float32 operations (no GPU needed):

* the pair check finds the kept-block set (segment) of a batch position x as
  x / n from a float estimate -- trunc(rz(x) * (1 / n)), the product rounded
  to nearest -- which must be within one of the quotient for every quotient a
  batch can hold (segments fewer than C(16, 8) < 2^14), so that one exact
  comparison fixes it;
* the ε recheck's float sums of squared differences stay within the relative
  error bounds its decisions use: four fma chains per lane over 4 lanes
  ((m + 8) u, m terms per chain; the candidate-list recheck) and eight fma
  chains per pair ((dim / 8 + 8) u; the dense-tile recheck), u = 2^-24.
The fma is replayed exactly: a float32 square is exact in float64, and the
float64 sum is rounded to float32 once."""
import numpy as np
import pytest

U = 2.0 ** -24


def f32(x):
    return np.float32(x)


def rz_u32_to_f32(x):
    """__uint2float_rz: keep the top 24 significant bits of x."""
    x = int(x)
    if x < (1 << 24):
        return np.float32(x)
    shift = x.bit_length() - 24
    return np.float32((x >> shift) << shift)


def seg_estimate(x, n):
    inv = np.float32(1.0) / np.float32(n)
    prod = np.float32(rz_u32_to_f32(x) * inv)          # rounded to nearest
    return int(np.floor(np.float64(prod)))             # __float2uint_rz


@pytest.mark.parametrize("n", [1, 7, 1000, 4096, 65537, 1_000_000, 4_000_000,
                               16_777_217, 100_000_007, 300_000_000])
def test_segment_estimate_within_one(n):
    S = min((1 << 14) - 1, ((1 << 32) - 1) // n)
    rng = np.random.default_rng(n)
    segs = np.unique(np.concatenate([np.arange(min(S, 64)), rng.integers(0, S, 200), [S - 1]]))
    for s in segs.tolist():
        for x in (s * n, s * n + 1, s * n + n - 1, s * n + n // 2):
            if x >= min(S * n, 1 << 32):
                continue
            q = seg_estimate(x, n)
            assert abs(q - x // n) <= 1, (n, x, q)
            p = q * n                                    # the kernel's exact fix-up
            if p > x:
                q -= 1
            elif p + n <= x:
                q += 1
            assert q == x // n


def _fma(a, b, c):
    return np.float32(np.float64(a) * np.float64(b) + np.float64(c))


def chain_sum(t, chains):
    """Sum of t_c^2 in `chains` interleaved fma chains (chain c % chains),
    combined pairwise."""
    acc = [np.float32(0.0)] * chains
    for c, v in enumerate(t):
        acc[c % chains] = _fma(v, v, acc[c % chains])
    while len(acc) > 1:
        acc = [np.float32(acc[i] + acc[i + 1]) for i in range(0, len(acc), 2)]
    return acc[0]


def rows(dim, kind, rng):
    if kind == "near":      # nearly equal rows: small differences, large magnitudes
        a = rng.standard_normal(dim).astype(np.float32)
        b = (a + np.float32(1e-3) * rng.standard_normal(dim)).astype(np.float32)
    elif kind == "spread":  # one large difference among many tiny ones
        a = rng.standard_normal(dim).astype(np.float32)
        b = a.copy()
        b[0] += np.float32(10.0)
        b[1:] += np.float32(1e-4) * rng.standard_normal(dim - 1).astype(np.float32)
    else:
        a = rng.standard_normal(dim).astype(np.float32)
        b = rng.standard_normal(dim).astype(np.float32)
    return a, b


@pytest.mark.parametrize("dim", [64, 96, 128, 256])
@pytest.mark.parametrize("kind", ["near", "spread", "random"])
def test_recheck_sum_bounds(dim, kind):
    rng = np.random.default_rng(dim * 7 + len(kind))
    for _ in range(20):
        a, b = rows(dim, kind, rng)
        t = np.array([f32(x - y) for x, y in zip(a, b)], dtype=np.float32)  # rounded difference
        exact = float(np.sum((a.astype(np.float64) - b.astype(np.float64)) ** 2))
        # candidate list: 4 lanes of float4 strides, four chains per lane, 2-level tree
        lanes = []
        n4 = dim // 4
        for sl in range(4):
            coords = [4 * c4 + w for c4 in range(sl, n4, 4) for w in range(4)]
            acc = [np.float32(0.0)] * 4
            for c in coords:
                acc[c % 4] = _fma(t[c], t[c], acc[c % 4])
            lanes.append(np.float32((acc[0] + acc[1]) + (acc[2] + acc[3])))
        s4 = np.float32(np.float32(lanes[0] + lanes[1]) + np.float32(lanes[2] + lanes[3]))
        m = ((dim + 3) // 4 + 3) // 4
        assert abs(float(s4) - exact) <= (m + 8) * U * exact + 1e-30
        # dense tiles: eight chains, combined pairwise
        s8 = chain_sum(t, 8)
        assert abs(float(s8) - exact) <= (dim // 8 + 8) * U * exact + 1e-30
