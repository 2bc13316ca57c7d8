"""GB300 epsilon-neighbour graphs by sign random projection + the multiple
sorting method (Uno, Sugiyama, Tsuda).

Thin Python binding over the C ABI of libmsm.so (include/msm.h): argument
marshalling only.  Every step of the method runs in the library's CUDA
kernels; PyTorch supplies device memory (through the allocator callback)
and the current stream.
"""
from __future__ import annotations

import ctypes
import traceback

import numpy as np
import torch

from . import _lib
from ._lib import Allocator, Pairs, Params, Stats

__all__ = ["MSMError", "gaussian", "project", "enumerate_pairs", "recheck",
           "eps_graph", "enumerate_sets", "eps_graph_sets", "Plan", "autotune",
           "eps_count_exhaustive", "collision_p", "miss_bound", "choose_params",
           "estimate_output",
           "solve_Q", "unpack_pairs", "COSINE", "EUCLIDEAN", "lib"]

COSINE, EUCLIDEAN = 0, 1
DT_F32, DT_BF16 = 0, 1
OUT_PAIRS_DIST, OUT_PAIRS, OUT_COUNT = 0, 1, 2
HASH_SIGN, HASH_E2LSH = 0, 1
FLAG_CANONICAL = 1
FLAG_SIMT_PROJECTION = 2


class MSMError(RuntimeError):
    def __init__(self, status: int, where: str):
        L = lib()
        msg = L.msm_last_error().decode(errors="replace")
        super().__init__(f"{where}: {L.msm_strerror(status).decode()} ({status}): {msg}")
        self.status = status


def lib():
    return _lib.load()


def _check(status: int, where: str):
    if status != 0:
        raise MSMError(status, where)


def _metric(m) -> int:
    if isinstance(m, str):
        return {"cosine": COSINE, "euclidean": EUCLIDEAN}[m.lower()]
    return int(m)


def _dtype(t: torch.Tensor) -> int:
    if t.dtype == torch.float32:
        return DT_F32
    if t.dtype == torch.bfloat16:
        return DT_BF16
    raise TypeError(f"unsupported element type {t.dtype}")


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


class _TorchAllocator:
    """Device memory for the library from PyTorch's caching allocator."""

    def __init__(self, device):
        self.device = device
        self.live = {}
        self._a = _lib.ALLOC_FN(self._alloc)
        self._f = _lib.FREE_FN(self._free)
        self.struct = Allocator(self._a, self._f, None)

    def _alloc(self, nbytes, stream, ctx):
        try:
            t = torch.empty(int(nbytes), dtype=torch.uint8, device=self.device)
        except Exception:  # noqa: BLE001 - report as NULL to the library
            traceback.print_exc()
            return None
        p = t.data_ptr()
        self.live[p] = t
        return p

    def _free(self, ptr, stream, ctx):
        self.live.pop(ptr, None)

    def take(self, ptr, count, dtype):
        """Hand a library-allocated buffer to the caller as a tensor."""
        if not ptr:
            return torch.empty(0, dtype=dtype, device=self.device)
        t = self.live.pop(ptr)
        return t.view(dtype)[:count]


def gaussian(seed: int, count: int, device=None) -> torch.Tensor:
    """Step A0': `count` N(0,1) floats from the counter-based generator."""
    out = torch.empty(count, dtype=torch.float32, device=device or "cuda")
    _check(lib().msm_gaussian(ctypes.c_uint64(seed), count, ctypes.c_void_p(out.data_ptr()),
                              _stream()), "msm_gaussian")
    return out


def project(X: torch.Tensor, ell: int, Q: int, R: torch.Tensor | None = None,
            seed: int = 0, return_recomputed: bool = False, simt: bool = False):
    """Step A1 (Eq. 3): strings int64 view of uint64 [Q][n][ceil(ell/64)]."""
    assert X.is_cuda and X.is_contiguous() and X.dim() == 2
    n, dim = X.shape
    if R is not None:
        assert R.is_cuda and R.dtype == torch.float32 and R.is_contiguous()
        assert tuple(R.shape) == (Q, dim, ell)
    W = (ell + 63) // 64
    S = torch.empty((Q, n, W), dtype=torch.int64, device=X.device)
    rec = ctypes.c_int64(0)
    _check(lib().msm_project(ctypes.c_void_p(X.data_ptr()), n, dim, _dtype(X),
                             ctypes.c_void_p(R.data_ptr() if R is not None else 0),
                             ctypes.c_uint64(seed), ell, Q, FLAG_SIMT_PROJECTION if simt else 0,
                             ctypes.c_void_p(S.data_ptr()),
                             ctypes.byref(rec) if return_recomputed else None, _stream()),
           "msm_project")
    return (S, rec.value) if return_recomputed else S


def enumerate_pairs(strings: torch.Tensor, ell: int, k: int, d: int,
                    canonical: bool = False):
    """Steps A3-A7: all pairs within Hamming d in at least one pool, once.
    strings: int64/uint64 [Q][n][W] on the GPU.  Returns (pairs, stats)."""
    assert strings.is_cuda and strings.is_contiguous() and strings.dim() == 3
    Q, n, W = strings.shape
    assert W == (ell + 63) // 64
    A = _TorchAllocator(strings.device)
    out = Pairs()
    st = Stats()
    _check(lib().msm_enumerate(ctypes.c_void_p(strings.data_ptr()), n, ell, k, d, Q,
                               FLAG_CANONICAL if canonical else 0, ctypes.byref(A.struct),
                               ctypes.byref(out), ctypes.byref(st), _stream()), "msm_enumerate")
    pairs = A.take(out.pairs, out.count, torch.int64)
    return pairs, st.as_dict()


def recheck(X: torch.Tensor, cand: torch.Tensor, metric, eps: float):
    """Step A8: keep the candidate pairs with distance <= eps.
    Returns (pairs, dist, recomputed) in unspecified order."""
    assert X.is_cuda and X.is_contiguous() and cand.is_cuda and cand.is_contiguous()
    n, dim = X.shape
    m = cand.numel()
    pairs = torch.empty(max(m, 1), dtype=torch.int64, device=X.device)
    dist = torch.empty(max(m, 1), dtype=torch.float32, device=X.device)
    cnt = ctypes.c_int64(0)
    rec = ctypes.c_int64(0)
    _check(lib().msm_recheck(ctypes.c_void_p(X.data_ptr()), n, dim, _dtype(X), _metric(metric),
                             ctypes.c_float(eps), ctypes.c_void_p(cand.data_ptr()), m,
                             ctypes.c_void_p(pairs.data_ptr()), ctypes.c_void_p(dist.data_ptr()),
                             ctypes.byref(cnt), ctypes.byref(rec), _stream()), "msm_recheck")
    return pairs[:cnt.value], dist[:cnt.value], rec.value


def _params(ell, k, d, Q, seed, R, Y, n, out_mode, canonical, simt_projection, group_bits,
            cand_capacity, tuning=None, e2lsh=None):
    p = Params()
    p.ell, p.k, p.d, p.Q = ell, k, d, Q
    p.seed = seed
    p.R = R.data_ptr() if R is not None else None
    if Y is not None:
        assert Y.is_cuda and Y.is_contiguous() and Y.shape[0] == n
        p.Y, p.dim_y, p.dtype_y = Y.data_ptr(), Y.shape[1], _dtype(Y)
    p.out_mode = out_mode
    p.flags = (FLAG_CANONICAL if canonical else 0) | (FLAG_SIMT_PROJECTION if simt_projection else 0)
    p.group_bits = group_bits
    p.cand_capacity = cand_capacity
    for key, v in (tuning or {}).items():
        assert key in ("masks_per_batch", "check_ctas_per_sm", "check_min_blocks"), key
        setattr(p, key, int(v))
    if e2lsh is not None:
        p.hash = HASH_E2LSH
        p.symbol_bits = int(e2lsh.get("symbol_bits", 4))
        p.width = float(e2lsh.get("width", 0.0))
    return p


def eps_graph(X: torch.Tensor, metric, eps: float, ell: int, k: int, d: int,
              Q: int = 0, miss_ratio: float = 1e-6, R: torch.Tensor | None = None,
              seed: int = 0, out_mode: int = OUT_PAIRS_DIST, canonical: bool = False,
              group_bits: int = 0, cand_capacity: int = 0, simt_projection: bool = False,
              Y: torch.Tensor | None = None, device=None, tuning: dict | None = None,
              e2lsh: dict | None = None):
    """The whole method.  X may be a CUDA tensor or a (pinned) CPU tensor,
    which the library copies in.  With Y (CUDA [n][dim_y], e.g. learned
    features) the strings come from Y while the recheck uses X.  ``e2lsh``
    (dict with symbol_bits, width) selects E2LSH symbol strings of ell
    symbols (d then counts differing symbols).  ``tuning``
    sets launch knobs of msm_params (masks_per_batch, check_ctas_per_sm,
    check_min_blocks); results do not depend on them.
    Returns (pairs, dist, stats)."""
    assert X.is_contiguous() and X.dim() == 2
    n, dim = X.shape
    dev = X.device if X.is_cuda else torch.device(device or "cuda")
    p = _params(ell, k, d, Q, seed, R, Y, n, out_mode, canonical, simt_projection, group_bits,
                cand_capacity, tuning, e2lsh)
    A = _TorchAllocator(dev)
    out = Pairs()
    st = Stats()
    with torch.cuda.device(dev):
        _check(lib().msm_eps_graph(ctypes.c_void_p(X.data_ptr()), n, dim, _dtype(X),
                                   _metric(metric), ctypes.c_float(eps), ctypes.c_double(miss_ratio),
                                   ctypes.byref(p), ctypes.byref(A.struct), ctypes.byref(out),
                                   ctypes.byref(st), _stream()), "msm_eps_graph")
    pairs = A.take(out.pairs, out.count, torch.int64) if out_mode != OUT_COUNT else None
    dist = A.take(out.dist, out.count, torch.float32) if out_mode == OUT_PAIRS_DIST else None
    s = st.as_dict()
    s["count"] = int(out.count)
    return pairs, dist, s


def _offsets(set_offsets):
    off = np.ascontiguousarray(np.asarray(set_offsets, dtype=np.int64))
    assert off.ndim == 1 and off.size >= 2
    return off, off.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), off.size - 1


def enumerate_sets(strings: torch.Tensor, set_offsets, ell: int, k: int, d: int,
                   canonical: bool = False):
    """enumerate_pairs over independent point sets: set s is rows
    [set_offsets[s], set_offsets[s+1]) of the pool; pairs never cross sets.
    Returns (pairs, stats)."""
    assert strings.is_cuda and strings.is_contiguous() and strings.dim() == 3
    Q, n, W = strings.shape
    off, offp, S = _offsets(set_offsets)
    assert off[-1] == n and W == (ell + 63) // 64
    A = _TorchAllocator(strings.device)
    out = Pairs()
    st = Stats()
    _check(lib().msm_enumerate_sets(ctypes.c_void_p(strings.data_ptr()), offp, S, ell, k, d, Q,
                                    FLAG_CANONICAL if canonical else 0, ctypes.byref(A.struct),
                                    ctypes.byref(out), ctypes.byref(st), _stream()),
           "msm_enumerate_sets")
    return A.take(out.pairs, out.count, torch.int64), st.as_dict()


def eps_graph_sets(X: torch.Tensor, set_offsets, metric, eps: float, ell: int, k: int, d: int,
                   Q: int = 0, miss_ratio: float = 1e-6, R: torch.Tensor | None = None,
                   seed: int = 0, out_mode: int = OUT_COUNT, canonical: bool = False,
                   group_bits: int = 0, cand_capacity: int = 0, simt_projection: bool = False,
                   device=None, tuning: dict | None = None):
    """eps_graph over independent point sets (rows [set_offsets[s],
    set_offsets[s+1]) of X form set s).  Returns (pairs, dist, set_counts,
    stats); set_counts is a numpy int64 [S] of result pairs per set.  The
    default output mode is count-only, which stores no pair list."""
    assert X.is_contiguous() and X.dim() == 2
    n, dim = X.shape
    off, offp, S = _offsets(set_offsets)
    assert off[-1] == n
    dev = X.device if X.is_cuda else torch.device(device or "cuda")
    p = _params(ell, k, d, Q, seed, R, None, n, out_mode, canonical, simt_projection, group_bits,
                cand_capacity, tuning)
    counts = np.zeros(S, dtype=np.int64)
    A = _TorchAllocator(dev)
    out = Pairs()
    st = Stats()
    with torch.cuda.device(dev):
        _check(lib().msm_eps_graph_sets(
            ctypes.c_void_p(X.data_ptr()), offp, S, dim, _dtype(X), _metric(metric),
            ctypes.c_float(eps), ctypes.c_double(miss_ratio), ctypes.byref(p),
            ctypes.byref(A.struct), ctypes.byref(out),
            counts.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), ctypes.byref(st), _stream()),
            "msm_eps_graph_sets")
    pairs = A.take(out.pairs, out.count, torch.int64) if out_mode != OUT_COUNT else None
    dist = A.take(out.dist, out.count, torch.float32) if out_mode == OUT_PAIRS_DIST else None
    s = st.as_dict()
    s["count"] = int(out.count)
    return pairs, dist, counts, s


def autotune(X: torch.Tensor, set_offsets, metric, eps: float, ell: int, k: int, d: int,
             Q: int, seed: int = 0, R: torch.Tensor | None = None, cache_path: str | None = None,
             simt_projection: bool = False) -> dict:
    """msm_autotune: the fastest launch knobs for count-only runs of this
    shape (timed on X; cached per device and shape in ``cache_path``).
    Returns the ``tuning`` dict for eps_graph / eps_graph_sets / Plan."""
    assert X.is_contiguous() and X.dim() == 2
    n, dim = X.shape
    off, offp, S = _offsets(set_offsets if set_offsets is not None else [0, n])
    assert off[-1] == n
    p = _params(ell, k, d, Q, seed, R, None, n, OUT_COUNT, False, simt_projection, 0, 0)
    A = _TorchAllocator(X.device if X.is_cuda else torch.device("cuda"))
    _check(lib().msm_autotune(ctypes.c_void_p(X.data_ptr()), offp, S, dim, _dtype(X),
                              _metric(metric), ctypes.c_float(eps), ctypes.byref(p),
                              cache_path.encode() if cache_path else None,
                              ctypes.byref(A.struct), _stream()), "msm_autotune")
    return {"check_min_blocks": p.check_min_blocks, "check_ctas_per_sm": p.check_ctas_per_sm,
            "masks_per_batch": p.masks_per_batch}


class Plan:
    """msm_plan: a reusable count-only run of eps_graph_sets for inputs of
    one shape.  The first run executes directly, the second captures a CUDA
    graph, later runs are one graph launch each.  ``input`` is the device
    buffer the plan reads (fill it and call run() without X to skip a copy)."""

    def __init__(self, set_offsets, dim: int, dtype, metric, eps: float, ell: int, k: int,
                 d: int, Q: int, seed: int = 0, R: torch.Tensor | None = None,
                 miss_ratio: float = 1e-6, simt_projection: bool = False,
                 tuning: dict | None = None, device=None):
        self.off, offp, self.S = _offsets(set_offsets)
        self.n, self.dim = int(self.off[-1]), dim
        self.dtype = dtype
        self.device = torch.device(device or "cuda")
        self._R = R
        p = _params(ell, k, d, Q, seed, R, None, self.n, OUT_COUNT, False, simt_projection, 0, 0,
                    tuning)
        self._A = _TorchAllocator(self.device)
        h = ctypes.c_void_p()
        dt = DT_BF16 if dtype == torch.bfloat16 else DT_F32
        with torch.cuda.device(self.device):
            _check(lib().msm_plan_create(offp, self.S, dim, dt, _metric(metric),
                                         ctypes.c_float(eps), ctypes.c_double(miss_ratio),
                                         ctypes.byref(p), ctypes.byref(self._A.struct),
                                         ctypes.byref(h)), "msm_plan_create")
        self._h = h
        ptr = lib().msm_plan_input(h)
        self.input = self._A.live[ptr].view(dtype)[: self.n * dim].view(self.n, dim)

    def run(self, X: torch.Tensor | None = None):
        """Returns (count, set_counts numpy int64 [S], stats)."""
        cnt = ctypes.c_int64(0)
        counts = np.zeros(self.S, dtype=np.int64)
        st = Stats()
        if X is not None:
            assert X.is_contiguous() and tuple(X.shape) == (self.n, self.dim) and X.dtype == self.dtype
        with torch.cuda.device(self.device):
            _check(lib().msm_plan_run(self._h, ctypes.c_void_p(X.data_ptr()) if X is not None else None,
                                      ctypes.byref(cnt),
                                      counts.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                      ctypes.byref(st), _stream()), "msm_plan_run")
        s = st.as_dict()
        s["count"] = int(cnt.value)
        return int(cnt.value), counts, s

    @property
    def is_graph(self) -> bool:
        return bool(lib().msm_plan_is_graph(self._h))

    def close(self):
        if getattr(self, "_h", None):
            lib().msm_plan_destroy(self._h, None)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001 - interpreter shutdown
            pass


class MLPProjection:
    """Learned feature map y = W2 gelu(W1 x + b1) + b2 (bf16 weights, float
    master copy and Adam moments), trained with the library's kernels on
    pairs labelled neighbour / non-neighbour."""

    def __init__(self, dim: int, hidden: int = 512, dim_out: int = 128, seed: int = 0,
                 device="cuda"):
        g = torch.Generator(device="cpu").manual_seed(seed)
        W1 = torch.randn(hidden, dim, generator=g) / dim ** 0.5
        W2 = torch.randn(dim_out, hidden, generator=g) / hidden ** 0.5
        self.dim, self.hidden, self.dim_out = dim, hidden, dim_out
        self.params = torch.cat([W1.reshape(-1), torch.zeros(hidden), W2.reshape(-1),
                                 torch.zeros(dim_out)]).to(device)
        self.m = torch.zeros_like(self.params)
        self.v = torch.zeros_like(self.params)
        self.W1h = W1.to(device, torch.bfloat16).contiguous()
        self.W2h = W2.to(device, torch.bfloat16).contiguous()
        self.step = 0

    def _views(self):
        h, d, o = self.hidden, self.dim, self.dim_out
        b1 = self.params[h * d: h * d + h]
        b2 = self.params[h * d + h + o * h:]
        return b1, b2

    def features(self, X: torch.Tensor) -> torch.Tensor:
        assert X.is_cuda and X.is_contiguous() and X.shape[1] == self.dim
        b1, b2 = self._views()
        Y = torch.empty((X.shape[0], self.dim_out), dtype=torch.float32, device=X.device)
        _check(lib().msm_mlp_forward(ctypes.c_void_p(X.data_ptr()), X.shape[0], self.dim, _dtype(X),
                                     ctypes.c_void_p(self.W1h.data_ptr()),
                                     ctypes.c_void_p(b1.data_ptr()),
                                     ctypes.c_void_p(self.W2h.data_ptr()),
                                     ctypes.c_void_p(b2.data_ptr()), self.hidden, self.dim_out,
                                     ctypes.c_void_p(Y.data_ptr()), _stream()), "msm_mlp_forward")
        return Y

    def grad(self, X, pi, pj, label, m_pos=0.98, m_neg=0.5):
        """(loss, grads) of one batch; pi, pj int32 CUDA, label uint8 CUDA."""
        b1, b2 = self._views()
        grads = torch.empty_like(self.params)
        loss = ctypes.c_float(0.0)
        _check(lib().msm_mlp_grad(ctypes.c_void_p(X.data_ptr()), X.shape[0], self.dim, _dtype(X),
                                  ctypes.c_void_p(self.W1h.data_ptr()), ctypes.c_void_p(b1.data_ptr()),
                                  ctypes.c_void_p(self.W2h.data_ptr()), ctypes.c_void_p(b2.data_ptr()),
                                  self.hidden, self.dim_out, ctypes.c_void_p(pi.data_ptr()),
                                  ctypes.c_void_p(pj.data_ptr()), ctypes.c_void_p(label.data_ptr()),
                                  pi.numel(), ctypes.c_float(m_pos), ctypes.c_float(m_neg),
                                  ctypes.c_void_p(grads.data_ptr()), ctypes.byref(loss), _stream()),
               "msm_mlp_grad")
        return loss.value, grads

    def adam(self, grads, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
        self.step += 1
        _check(lib().msm_mlp_adam(ctypes.c_void_p(self.params.data_ptr()),
                                  ctypes.c_void_p(grads.data_ptr()), ctypes.c_void_p(self.m.data_ptr()),
                                  ctypes.c_void_p(self.v.data_ptr()), self.params.numel(), self.step,
                                  ctypes.c_float(lr), ctypes.c_float(beta1), ctypes.c_float(beta2),
                                  ctypes.c_float(eps), ctypes.c_void_p(self.W1h.data_ptr()),
                                  ctypes.c_void_p(self.W2h.data_ptr()), self.hidden, self.dim,
                                  self.dim_out, _stream()), "msm_mlp_adam")

    def train(self, X, pi, pj, label, steps=200, batch=4096, lr=1e-3, m_pos=0.98,
              m_neg=0.5, seed=0):
        """Minibatch Adam over the labelled pairs (CUDA int32 pi, pj, uint8
        label); returns the loss history."""
        g = torch.Generator(device=X.device).manual_seed(seed)
        hist = []
        for _ in range(steps):
            sel = torch.randint(0, pi.numel(), (min(batch, pi.numel()),), device=X.device,
                                generator=g)
            loss, grads = self.grad(X, pi[sel].contiguous(), pj[sel].contiguous(),
                                    label[sel].contiguous(), m_pos, m_neg)
            self.adam(grads, lr)
            hist.append(loss)
        return hist


def eps_count_exhaustive(X: torch.Tensor, metric, eps: float) -> int:
    """Exact number of pairs within eps by exhaustive comparison (a
    measurement aid for the missing-edge ratio)."""
    assert X.is_cuda and X.is_contiguous()
    n, dim = X.shape
    c = ctypes.c_int64(0)
    _check(lib().msm_eps_count_exhaustive(ctypes.c_void_p(X.data_ptr()), n, dim, _dtype(X),
                                          _metric(metric), ctypes.c_float(eps), ctypes.byref(c),
                                          _stream()), "msm_eps_count_exhaustive")
    return c.value


def e2lsh_p(w: float) -> float:
    """Non-collision probability of one E2LSH symbol at bucket width w times
    the distance (Datar et al.)."""
    return lib().msm_e2lsh_p(float(w))


def e2lsh_offsets(seed: int, count: int, device=None) -> torch.Tensor:
    out = torch.empty(count, dtype=torch.float32, device=device or "cuda")
    _check(lib().msm_e2lsh_offsets(ctypes.c_uint64(seed), count, ctypes.c_void_p(out.data_ptr()),
                                   _stream()), "msm_e2lsh_offsets")
    return out


def project_e2lsh(X: torch.Tensor, R: torch.Tensor, u: torch.Tensor, width: float,
                  symbol_bits: int, return_recomputed: bool = False):
    """E2LSH symbol strings int64 [Q][n][W] (W = ceil(ell * symbol_bits / 64))."""
    assert X.is_cuda and X.is_contiguous() and R.is_cuda and R.is_contiguous() and u.is_cuda
    n, dim = X.shape
    Q, D2, ell = R.shape
    assert D2 == dim and u.numel() == Q * ell
    Wd = (ell * symbol_bits + 63) // 64
    S = torch.empty((Q, n, Wd), dtype=torch.int64, device=X.device)
    rec = ctypes.c_int64(0)
    _check(lib().msm_project_e2lsh(ctypes.c_void_p(X.data_ptr()), n, dim, _dtype(X),
                                   ctypes.c_void_p(R.data_ptr()), ctypes.c_void_p(u.data_ptr()),
                                   ctypes.c_float(width), ell, Q, symbol_bits,
                                   ctypes.c_void_p(S.data_ptr()), ctypes.byref(rec), _stream()),
           "msm_project_e2lsh")
    return (S, rec.value) if return_recomputed else S


def enumerate_symbols(strings: torch.Tensor, ell: int, symbol_bits: int, k: int, d: int,
                      canonical: bool = False):
    """enumerate_pairs over symbol strings (ell symbols of symbol_bits bits)."""
    assert strings.is_cuda and strings.is_contiguous() and strings.dim() == 3
    Q, n, Wd = strings.shape
    assert Wd == (ell * symbol_bits + 63) // 64
    A = _TorchAllocator(strings.device)
    out = Pairs()
    st = Stats()
    _check(lib().msm_enumerate_symbols(ctypes.c_void_p(strings.data_ptr()), n, ell, symbol_bits,
                                       k, d, Q, FLAG_CANONICAL if canonical else 0,
                                       ctypes.byref(A.struct), ctypes.byref(out),
                                       ctypes.byref(st), _stream()), "msm_enumerate_symbols")
    return A.take(out.pairs, out.count, torch.int64), st.as_dict()


def choose_params(n: int, p: float, gamma: float, S: float):
    """Sec. 4.3 parameter rule: (ell, k, d, Q) for n points, non-collision
    probability p at the radius, missing-ratio bound gamma and output-size
    estimate S."""
    e, k, d, Q = (ctypes.c_int() for _ in range(4))
    _check(lib().msm_choose_params(int(n), ctypes.c_double(p), ctypes.c_double(gamma),
                                   ctypes.c_double(S), ctypes.byref(e), ctypes.byref(k),
                                   ctypes.byref(d), ctypes.byref(Q)), "msm_choose_params")
    return e.value, k.value, d.value, Q.value


def estimate_output(X: torch.Tensor, metric, eps: float, samples: int = 1 << 22,
                    seed: int = 0) -> float:
    """Sec. 4.3 output-size estimate from `samples` random pairs."""
    assert X.is_cuda and X.is_contiguous() and X.dim() == 2
    n, dim = X.shape
    S = ctypes.c_double()
    _check(lib().msm_estimate_output(ctypes.c_void_p(X.data_ptr()), n, dim, _dtype(X),
                                     _metric(metric), ctypes.c_float(eps), int(samples),
                                     ctypes.c_uint64(seed), ctypes.byref(S), _stream()),
           "msm_estimate_output")
    return S.value


def collision_p(metric, eps: float) -> float:
    return lib().msm_collision_p(_metric(metric), eps)


def miss_bound(ell: int, d: int, p: float, Q: int) -> float:
    return lib().msm_miss_bound(ell, d, p, Q)


def solve_Q(ell: int, d: int, p: float, gamma: float) -> int:
    q = ctypes.c_int(0)
    _check(lib().msm_solve_Q(ell, d, p, gamma, ctypes.byref(q)), "msm_solve_Q")
    return q.value


def unpack_pairs(p: torch.Tensor):
    return p >> 32, p & 0xFFFFFFFF
