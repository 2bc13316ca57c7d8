"""Host-side pieces of bench.py's roofline (no GPU): the word count of the
pair check's ALU model, the algorithmic bytes of the HBM-bound kernels, and
the summary of the clock samples taken during the timed region."""
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


def test_algorithmic_bytes_hand_counts(bench):
    # one replicate batch of the scale workload: 210 kept sets x n items,
    # strings of W = 2 words, one point set (top-digit pass + bucket sort)
    st = {"masks": 12 * 210, "cand": 1000}
    n = 1000
    items = 210 * n
    # scatter class, two launches per replicate: the top-digit scatter writes
    # key + index (8 B), the bucket sort reads and writes them (16 B)
    b, unit, bound = bench.algorithmic("radix_scatter", st, n, 128, 12, 2)
    assert (b, unit, bound) == (items * 24 / 2, "GB/s", "hbm")
    # histogram: reads the 16-byte string of every item (from L2)
    b, _, bound = bench.algorithmic("radix_hist", st, n, 128, 12, 2)
    assert (b, bound) == (items * 16, "l2")
    # recheck: the pair (8 B), two float rows of 128 (1024 B), pair and
    # distance out (12 B)
    b, _, _ = bench.algorithmic("recheck", st, n, 128, 12, 2)
    assert b == 1000 * (8 + 1024 + 12)
    assert bench.algorithmic("pair_check", st, n, 128, 12, 2) == (None, None, None)


def test_exact_test_ops_hand_count(bench):
    # k = 10 blocks: 5 field words; per word 3 (gap) + 3 (Hamming) + 3
    # (replicate-0 Hamming), plus 2 compares
    assert bench.exact_test_ops(10) == 47
    assert bench.exact_test_ops(8) == 38


def test_clock_samples_summary(bench):
    # nvidia-smi --query-gpu=<ClockSampler.FIELDS> --format=csv,noheader,nounits
    lines = [
        "0, 2070, 2070, 674.97, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, 1980, 2070, 1390.2, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 1201.5, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, [N/A], 2070, 10.0, 0x0, Not Active, Not Active, Not Active, Not Active",   # skipped
        "truncated line",
    ]
    got = bench.parse_clocks(lines)
    assert got == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "samples": 3,
                   "reasons": ["sw_power_cap"]}
    hot = ["0, 1500, 2070, 900, 0x48, Active, Active, Not Active, Not Active"]
    assert bench.parse_clocks(hot)["reasons"] == ["hw_slowdown", "hw_thermal_slowdown"]
    assert bench.parse_clocks([]) is None
    # an unreadable max clock: the SM sample still counts, and with no
    # readable max at all the maximum falls back to the highest SM sample
    na = ["0, 1900, [N/A], 800, 0x0, Not Active, Not Active, Not Active, Not Active",
          "0, 2010, [N/A], 800, 0x0, Not Active, Not Active, Not Active, Not Active"]
    assert bench.parse_clocks(na) == {"sm_mhz": 1955.0, "sm_max_mhz": 2010.0, "samples": 2,
                                      "reasons": []}
    assert bench.parse_clocks(na + lines[:1])["sm_max_mhz"] == 2070.0


def test_cpu_oracle_copies_run_and_time_out(bench):
    import workloads as W
    import oracle
    wl = W.WORKLOADS["scale"]
    X = W.clustered(600, 128, 30, 0.05, 1002)
    R = oracle.gaussian(2002, 2 * 128 * 128).reshape(2, 128, 128)
    res = bench.cpu_oracle_copies(X, R, wl, 600, 2)
    assert res is not None
    wall, per = res
    assert len(per) == 2 and all(0 < p <= wall for p in per)
    # an impossible deadline: no result, and the copies are killed
    assert bench.cpu_oracle_copies(X, R, wl, 600, 2, timeout_s=1e-3) is None
    assert bench.usable_cores() >= 1


def test_cpu_sample_keeps_the_cluster_size(bench):
    import workloads as W
    wl = W.WORKLOADS["scale"]
    X, nc = bench.cpu_sample_points(wl, wl.n, 2000, 5)
    assert nc == 2 and X.shape == (2000, wl.dim)   # clusters of 1,000 points, as at 1M
    X, nc = bench.cpu_sample_points(wl, wl.n, 500, 5)
    assert nc == 1 and X.shape == (1000, wl.dim)   # never less than one whole cluster
