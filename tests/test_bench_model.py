"""Host-side pieces of bench.py's roofline (no GPU): the word count of the
pair check's ALU model."""
import importlib.util
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_gap_words_hand_counts(bench):
    # k = 2, d = 1: K = {0} has no gap block, K = {1} has block 0 (word 0)
    assert bench.gap_words_mean(2, 1) == pytest.approx(0.5)
    # k = 4, d = 2, K over pairs of blocks, words = highest gap block // 2 + 1:
    # {0,1}: none -> 0; {0,2}: 1 -> 1; {0,3}: 1,2 -> 2; {1,2}: 0 -> 1;
    # {1,3}: 0,2 -> 2; {2,3}: 0,1 -> 1; total 7 over 6 sets
    assert bench.gap_words_mean(4, 2) == pytest.approx(7 / 6)


def test_gap_words_bounds(bench):
    # never more than the words holding fields, and d = 0 keeps every block
    # (the only kept set is all blocks: no gap)
    for k in range(2, 13):
        for d in range(0, k):
            m = bench.gap_words_mean(k, d)
            assert 0 <= m <= (k + 1) // 2
    assert bench.gap_words_mean(8, 0) == 0
