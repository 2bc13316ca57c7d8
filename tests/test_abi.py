"""The C-ABI library builds, loads, and exports every symbol include/msm.h
declares; the host-only entry points (replicate-count arithmetic of
Sec. 4.2-4.3, error strings) agree with the oracle.  No GPU needed."""
import math
import os
import re

import numpy as np
import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_0904_3151_gb300 import build as b
    b.build()
    import paper_0904_3151_gb300 as msm
    return msm.lib()


def _declared(header="msm.h"):
    src = open(os.path.join(ROOT, "include", header)).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return set(re.findall(r"^\s*(?:int|int64_t|double|void\*?|const char\*)\s+(msm_\w+)\s*\(", src,
                          flags=re.M))


def test_every_declared_symbol_is_exported(L):
    from paper_0904_3151_gb300 import _lib
    names = _declared()
    assert len(names) >= 12
    for nm in sorted(names):
        assert hasattr(L, nm), nm
    assert names == set(_lib.SIGNATURES), names ^ set(_lib.SIGNATURES)


def test_probe_library_is_separate(L):
    """The measurement aid lives in libmsm_probe.so, not in the method's
    library."""
    import ctypes
    from paper_0904_3151_gb300 import build as b
    names = _declared("msm_probe.h")
    assert names == {"msm_int_mix_probe"}
    P = ctypes.CDLL(b.PROBE_LIB)
    for nm in names:
        assert hasattr(P, nm)
        assert not hasattr(L, nm)


def test_version_and_strerror(L):
    assert L.msm_version() >= 100
    for code in [0, -1, -2, -3, -4, -5, -6, -7]:
        assert L.msm_strerror(code)
    assert L.msm_strerror(-99) == b"unknown status"


def test_collision_p_matches_oracle(L):
    for eps in [0.0, 0.0123, 0.1, 0.15, 0.7, 1.0, 1.9]:
        assert L.msm_collision_p(0, eps) == pytest.approx(oracle.p_cosine(eps), rel=1e-14, abs=1e-15)
    for eps in [0.0, 0.1, 0.3, 1.0]:
        assert L.msm_collision_p(1, eps) == pytest.approx(oracle.p_euclidean(eps), rel=1e-14, abs=1e-15)
    assert L.msm_collision_p(0, -0.5) == -1.0


@pytest.mark.parametrize("ell,d", [(50, 0), (50, 3), (64, 4), (128, 6), (128, 8), (96, 4), (256, 20)])
def test_miss_bound_and_solve_Q_match_oracle(L, ell, d):
    import ctypes
    for p in [0.01, 0.04, 0.1, 0.2]:
        b1 = oracle.miss_bound(ell, d, p, 1)
        for Q in [1, 3, 10]:
            a = L.msm_miss_bound(ell, d, p, Q)
            b = oracle.miss_bound(ell, d, p, Q)
            # 1 - sum(...) carries ~1e-16 absolute rounding in either
            # evaluation; raised to the power Q it scales by Q b1^(Q-1).
            tol = Q * b1 ** (Q - 1) * 4e-16
            assert a == pytest.approx(b, rel=1e-9, abs=tol + 1e-300)
        for gamma in [1e-2, 1e-6]:
            q = ctypes.c_int(0)
            rc = L.msm_solve_Q(ell, d, p, gamma, ctypes.byref(q))
            try:
                want = oracle.solve_Q(ell, d, p, gamma)
            except ValueError:       # beyond the oracle's 2^20 search range
                assert rc != 0 or q.value > (1 << 20)
                continue
            assert rc == 0
            if q.value != want:   # only a rounding tie at the threshold may differ
                b1 = oracle.miss_bound(ell, d, p, min(q.value, want))
                assert math.isclose(b1, gamma, rel_tol=1e-9)


def test_solve_Q_rejects_bad_input(L):
    import ctypes
    q = ctypes.c_int(0)
    assert L.msm_solve_Q(64, 4, 0.1, 0.0, ctypes.byref(q)) == -1
    assert L.msm_solve_Q(64, 4, 1.5, 1e-3, ctypes.byref(q)) == -1


def test_choose_params_matches_oracle(L):
    import paper_0904_3151_gb300 as msm
    for n in (2, 3, 1000, 1024, 20000, 1 << 20, 10_000_000):
        for eps in (0.0123, 0.05, 0.1, 0.15):
            for S in (0.0, 0.5, 10.0, 1e4, 1e8, 3e10):
                p = oracle.p_cosine(float(np.float32(eps)))
                try:
                    want = oracle.choose_params(n, p, 1e-6, S)
                except ValueError:
                    with pytest.raises(msm.MSMError):
                        msm.choose_params(n, p, 1e-6, S)
                    continue
                assert msm.choose_params(n, p, 1e-6, S) == want, (n, eps, S)


def test_e2lsh_probability_matches_oracle(L):
    for w in (0.25, 1.0, 3.5, 7.0, 12.0):
        assert L.msm_e2lsh_p(w) == pytest.approx(oracle.e2lsh_p(w), rel=1e-13, abs=1e-15)
    assert L.msm_e2lsh_p(0.0) == -1.0
