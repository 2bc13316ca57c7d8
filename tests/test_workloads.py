"""Host-side checks of the seeded input generators (no GPU)."""
import numpy as np

import workloads as W


def test_set_sizes_log_uniform_and_seeded():
    wl = W.WORKLOADS["batched"]
    a = W.set_sizes(wl.n_sets, wl.set_min, wl.set_max, wl.data_seed)
    b = W.set_sizes(wl.n_sets, wl.set_min, wl.set_max, wl.data_seed)
    assert np.array_equal(a, b) and len(a) == 256
    assert a.min() >= wl.set_min and a.max() < wl.set_max
    # log-uniform: the median is near the geometric mean of the bounds
    assert abs(np.log(np.median(a)) - 0.5 * np.log(wl.set_min * wl.set_max)) < 0.5
    # total close to the expected (hi - lo) / ln(hi / lo) per set
    expect = wl.n_sets * (wl.set_max - wl.set_min) / np.log(wl.set_max / wl.set_min)
    assert abs(a.sum() / expect - 1) < 0.15


def test_clustered_sets_layout():
    X, off = W.clustered_sets([5, 0, 40, 1], 16, 3, 0.05, 9)
    assert off.tolist() == [0, 5, 5, 45, 46] and X.shape == (46, 16)
    assert np.allclose(np.linalg.norm(X, axis=1), 1.0, atol=1e-6)
    # each set is drawn from its own stream: regenerating a prefix of the
    # sizes gives the same rows
    Y, _ = W.clustered_sets([5, 0, 40], 16, 3, 0.05, 9)
    assert np.array_equal(X[:45], Y)


def test_clustered_words_flip_rate():
    S = W.clustered_words(200_000, 2, 3, n_centres=1, and_depth=3)
    bits = np.unpackbits(S.view(np.uint8), axis=-1).reshape(200_000, 128)
    # one centre: the bits that differ from the column majority flip w.p. 1/8
    maj = (bits.mean(0) > 0.5).astype(np.uint8)
    assert abs((bits != maj).mean() - 0.125) < 0.002
