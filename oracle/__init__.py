"""CPU oracle for the LSH + multiple-sorting-method epsilon-graph.

TEST INFRASTRUCTURE ONLY: imported by the tests, by the package's smoke
check and by the benchmark's CPU-baseline leg, never by the product path.
The arithmetic lives in ``msm_oracle.c`` (plain C, double precision,
single thread) and in ``bound.py`` (the missing-edge-ratio bound of
Sec. 4.2); this module only builds the C file with gcc and marshals numpy
arrays.  It shares no code with the CUDA library.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

from .bound import (choose_params, e2lsh_p, miss_bound, p_cosine, p_euclidean,  # noqa: F401
                    solve_Q)

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "msm_oracle.c")
_LIB_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_LIB_DIR, "libmsm_oracle.so")

COSINE, EUCLIDEAN = 0, 1


def build(force: bool = False) -> str:
    """Compile msm_oracle.c into a shared object (gcc, no fast-math, no fp
    contraction beyond the explicit fma calls)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    os.makedirs(_LIB_DIR, exist_ok=True)
    tmp = _LIB + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared",
                           "-ffp-contract=off", "-fno-fast-math",
                           "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        P = ctypes.POINTER
        u64p, f64p, f32p, i64p = (P(ctypes.c_uint64), P(ctypes.c_double),
                                  P(ctypes.c_float), P(ctypes.c_int64))
        i64, i32 = ctypes.c_int64, ctypes.c_int
        L.orc_philox4x64_10.argtypes = [u64p, u64p, u64p]
        L.orc_gaussian.argtypes = [ctypes.c_uint64, i64, f32p]
        L.orc_project.argtypes = [f64p, i64, i32, f64p, i32, i32, u64p]
        L.orc_project_value.argtypes = [f64p, i32, f64p, i32, i32]
        L.orc_project_value.restype = ctypes.c_double
        L.orc_ham_pairs.argtypes = [u64p, i64, i32, i32, u64p, i64]
        L.orc_ham_pairs.restype = i64
        L.orc_msm.argtypes = [u64p, i64, i32, i32, i32, i32, u64p, i64, i64p]
        L.orc_msm.restype = i64
        L.orc_msm_positions.argtypes = [u64p, i64, i32, i32, u64p, i64, i64p]
        L.orc_msm_positions.restype = i64
        L.orc_distance.argtypes = [f64p, f64p, i32, i32]
        L.orc_distance.restype = ctypes.c_double
        L.orc_dist.argtypes = [f64p, i64, i32, i32, u64p, i64, f64p]
        L.orc_eps_bruteforce.argtypes = [f64p, i64, i32, i32, ctypes.c_double,
                                         u64p, f64p, i64]
        L.orc_eps_bruteforce.restype = i64
        L.orc_e2lsh_offsets.argtypes = [ctypes.c_uint64, i32, i32, f32p]
        L.orc_project_e2lsh.argtypes = [f64p, i64, i32, f64p, i32, i32, f32p,
                                        ctypes.c_double, i32, u64p]
        L.orc_sym_pairs.argtypes = [u64p, i64, i32, i32, i32, u64p, i64]
        L.orc_sym_pairs.restype = i64
        L.orc_msm_sym.argtypes = [u64p, i64, i32, i32, i32, i32, i32, u64p, i64, i64p]
        L.orc_msm_sym.restype = i64
        _lib = L
    return _lib


def _p(a, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


def _f64(x) -> np.ndarray:
    """Exact float64 copy of stored values (float32 / bfloat16-valued)."""
    return np.ascontiguousarray(np.asarray(x, dtype=np.float64))


def philox(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint64)
    k = np.ascontiguousarray(key, dtype=np.uint64)
    o = np.zeros(4, dtype=np.uint64)
    lib().orc_philox4x64_10(_p(c, ctypes.c_uint64), _p(k, ctypes.c_uint64),
                            _p(o, ctypes.c_uint64))
    return o


def gaussian(seed: int, count: int) -> np.ndarray:
    out = np.empty(count, dtype=np.float32)
    lib().orc_gaussian(ctypes.c_uint64(seed), count, _p(out, ctypes.c_float))
    return out


def project(X, R) -> np.ndarray:
    """Eq. 3 strings, uint64 [Q][n][W]."""
    X = _f64(X)
    R = _f64(R)
    n, D = X.shape
    Q, D2, ell = R.shape
    assert D2 == D
    W = (ell + 63) // 64
    S = np.zeros((Q, n, W), dtype=np.uint64)
    lib().orc_project(_p(X, ctypes.c_double), n, D, _p(R, ctypes.c_double),
                      Q, ell, _p(S, ctypes.c_uint64))
    return S


def project_value(x, Rq, c: int) -> float:
    x = _f64(x)
    Rq = _f64(Rq)
    return lib().orc_project_value(_p(x, ctypes.c_double), x.shape[0],
                                   _p(Rq, ctypes.c_double), Rq.shape[1], c)


def _grow_call(fn, cap0):
    cap = cap0
    while True:
        buf = np.zeros(max(cap, 1), dtype=np.uint64)
        m = fn(buf, cap)
        if m <= cap:
            return buf[:m], m
        cap = m


def ham_pairs(Sq, ell: int, d: int) -> np.ndarray:
    """Eq. 1 by definition on one pool Sq uint64 [n][W]."""
    Sq = np.ascontiguousarray(Sq, dtype=np.uint64)
    n = Sq.shape[0]
    out, _ = _grow_call(lambda b, cap: lib().orc_ham_pairs(
        _p(Sq, ctypes.c_uint64), n, ell, d, _p(b, ctypes.c_uint64), cap), 1 << 16)
    return out


def msm(S, ell: int, k: int, d: int):
    """Blockwise MSM over Q pools S uint64 [Q][n][W]; returns (pairs, stats)."""
    S = np.ascontiguousarray(S, dtype=np.uint64)
    Q, n, _ = S.shape
    st = np.zeros(3, dtype=np.int64)
    out, _ = _grow_call(lambda b, cap: lib().orc_msm(
        _p(S, ctypes.c_uint64), n, ell, k, d, Q, _p(b, ctypes.c_uint64), cap,
        _p(st, ctypes.c_int64)), 1 << 16)
    if int(st[2]) < 0:
        raise ValueError("invalid MSM parameters")
    return out, {"masks": int(st[0]), "checks": int(st[1]), "pairs": int(st[2])}


def msm_positions(Sq, ell: int, d: int):
    """Position masking of Sec. 2.1 on one pool; returns (pairs, sorts)."""
    Sq = np.ascontiguousarray(Sq, dtype=np.uint64)
    n = Sq.shape[0]
    sorts = np.zeros(1, dtype=np.int64)
    out, _ = _grow_call(lambda b, cap: lib().orc_msm_positions(
        _p(Sq, ctypes.c_uint64), n, ell, d, _p(b, ctypes.c_uint64), cap,
        _p(sorts, ctypes.c_int64)), 1 << 16)
    return out, int(sorts[0])


def distance(xi, xj, metric: int) -> float:
    xi, xj = _f64(xi), _f64(xj)
    return lib().orc_distance(_p(xi, ctypes.c_double), _p(xj, ctypes.c_double),
                              xi.shape[0], metric)


def dist(X, pairs, metric: int) -> np.ndarray:
    X = _f64(X)
    pairs = np.ascontiguousarray(pairs, dtype=np.uint64)
    out = np.zeros(pairs.shape[0], dtype=np.float64)
    lib().orc_dist(_p(X, ctypes.c_double), X.shape[0], X.shape[1], metric,
                   _p(pairs, ctypes.c_uint64), pairs.shape[0],
                   _p(out, ctypes.c_double))
    return out


def eps_bruteforce(X, metric: int, eps: float):
    """Def. 1.1 exhaustively; eps is compared as the double value given."""
    X = _f64(X)
    n, D = X.shape
    dbuf = {}

    def call(b, cap):
        dd = np.zeros(max(cap, 1), dtype=np.float64)
        dbuf["d"] = dd
        return lib().orc_eps_bruteforce(_p(X, ctypes.c_double), n, D, metric,
                                        float(eps), _p(b, ctypes.c_uint64),
                                        _p(dd, ctypes.c_double), cap)
    out, m = _grow_call(call, 1 << 20)
    return out, dbuf["d"][:m]


def eps_graph(X, R, ell: int, k: int, d: int, metric: int, eps: float):
    """The method of Sec. 4.1 end to end: strings (Eq. 3) for each replicate,
    blockwise MSM with replicate de-duplication (E = E_1 u ... u E_Q), then the
    exact distance of every pair in E, keeping those <= eps.  eps is the
    float32 value the library receives, compared in double.
    Returns (pairs, dist, info)."""
    S = project(X, R)
    E, st = msm(S, ell, k, d)
    dv = dist(X, E, metric)
    keep = dv <= float(np.float32(eps))
    info = dict(st)
    info["cand"] = int(E.shape[0])
    info["type1"] = int((~keep).sum())
    return E[keep], dv[keep], info


# ------------------------------------------------------------ E2LSH symbols

def e2lsh_offsets(seed: int, Q: int, ell: int) -> np.ndarray:
    """Bucket offsets u in [0, 1), float32 [Q][ell] (counter-based, key
    {seed, 2})."""
    out = np.empty(Q * ell, dtype=np.float32)
    lib().orc_e2lsh_offsets(ctypes.c_uint64(seed), Q, ell, _p(out, ctypes.c_float))
    return out.reshape(Q, ell)


def project_e2lsh(X, R, u, width: float, sw: int) -> np.ndarray:
    """Symbol strings uint64 [Q][n][W], W = ceil(ell sw / 64): symbol c is the
    low sw bits of floor(r_c^T x / width + u_c)."""
    X = _f64(X)
    R = _f64(R)
    u = np.ascontiguousarray(u, dtype=np.float32)
    n, D = X.shape
    Q, D2, ell = R.shape
    assert D2 == D and u.shape == (Q, ell)
    W = (ell * sw + 63) // 64
    S = np.zeros((Q, n, W), dtype=np.uint64)
    lib().orc_project_e2lsh(_p(X, ctypes.c_double), n, D, _p(R, ctypes.c_double), Q, ell,
                            _p(u, ctypes.c_float), float(width), sw, _p(S, ctypes.c_uint64))
    return S


def sym_pairs(Sq, ell: int, sw: int, d: int) -> np.ndarray:
    """Pairs of one pool with at most d differing symbols, by definition."""
    Sq = np.ascontiguousarray(Sq, dtype=np.uint64)
    n = Sq.shape[0]
    out, _ = _grow_call(lambda b, cap: lib().orc_sym_pairs(
        _p(Sq, ctypes.c_uint64), n, ell, sw, d, _p(b, ctypes.c_uint64), cap), 1 << 16)
    return out


def msm_sym(S, ell: int, sw: int, k: int, d: int):
    """Blockwise MSM over symbol strings; returns (pairs, stats)."""
    S = np.ascontiguousarray(S, dtype=np.uint64)
    Q, n, _ = S.shape
    st = np.zeros(3, dtype=np.int64)
    out, _ = _grow_call(lambda b, cap: lib().orc_msm_sym(
        _p(S, ctypes.c_uint64), n, ell, sw, k, d, Q, _p(b, ctypes.c_uint64), cap,
        _p(st, ctypes.c_int64)), 1 << 16)
    if int(st[2]) < 0:
        raise ValueError("invalid MSM parameters")
    return out, {"masks": int(st[0]), "checks": int(st[1]), "pairs": int(st[2])}


def eps_graph_e2lsh(X, R, u, width: float, sw: int, ell: int, k: int, d: int, metric: int,
                    eps: float):
    """The method with E2LSH symbol strings: symbols for each replicate,
    blockwise MSM over symbols with replicate de-duplication, exact distance
    filter.  Returns (pairs, dist, info)."""
    S = project_e2lsh(X, R, u, width, sw)
    E, st = msm_sym(S, ell, sw, k, d)
    dv = dist(X, E, metric)
    keep = dv <= float(np.float32(eps))
    info = dict(st)
    info["cand"] = int(E.shape[0])
    info["type1"] = int((~keep).sum())
    return E[keep], dv[keep], info


def unpack_pairs(p: np.ndarray):
    p = np.asarray(p, dtype=np.uint64)
    return (p >> np.uint64(32)).astype(np.int64), (p & np.uint64(0xFFFFFFFF)).astype(np.int64)
