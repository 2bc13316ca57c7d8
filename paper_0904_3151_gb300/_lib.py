"""ctypes view of libmsm.so (the C ABI declared in include/msm.h).

The shared object must have been built (``paper_0904_3151_gb300.build``);
there is no fallback: importing the compute functions without it raises.
"""
from __future__ import annotations

import ctypes
import os

from . import build as _build

u64p = ctypes.POINTER(ctypes.c_uint64)
i64p = ctypes.POINTER(ctypes.c_int64)
f32p = ctypes.POINTER(ctypes.c_float)
vp = ctypes.c_void_p

ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)


class Allocator(ctypes.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("ctx", ctypes.c_void_p)]


class Pairs(ctypes.Structure):
    _fields_ = [("pairs", ctypes.c_void_p), ("dist", ctypes.c_void_p), ("count", ctypes.c_int64)]


class Stats(ctypes.Structure):
    _fields_ = [("Q", ctypes.c_int64), ("masks", ctypes.c_int64), ("checks", ctypes.c_int64),
                ("cand", ctypes.c_int64), ("type1", ctypes.c_int64),
                ("proj_recompute", ctypes.c_int64), ("dist_recompute", ctypes.c_int64),
                ("overflow_retries", ctypes.c_int64), ("ms", ctypes.c_float * 8),
                ("kernel_ms", ctypes.c_float * 8), ("kernel_launches", ctypes.c_int64 * 8),
                ("ell", ctypes.c_int), ("k", ctypes.c_int), ("d", ctypes.c_int),
                ("reserved", ctypes.c_int), ("S_est", ctypes.c_double),
                ("evaluated", ctypes.c_int64)]

    PHASES = ["norms_R", "project", "group_sort", "group_bounds", "group_check",
              "recheck", "canonical", "total"]
    KERNELS = ["project", "radix_hist", "radix_scatter", "scan", "group_bounds",
               "pair_check", "recheck", "other"]

    def as_dict(self):
        skip = ("ms", "kernel_ms", "kernel_launches", "reserved")
        d = {f: getattr(self, f) for f, _ in self._fields_ if f not in skip}
        d["ms"] = {k: float(v) for k, v in zip(self.PHASES, self.ms)}
        d["kernel_ms"] = {k: float(v) for k, v in zip(self.KERNELS, self.kernel_ms)}
        d["kernel_launches"] = {k: int(v) for k, v in zip(self.KERNELS, self.kernel_launches)}
        return d


class Params(ctypes.Structure):
    _fields_ = [("ell", ctypes.c_int), ("k", ctypes.c_int), ("d", ctypes.c_int), ("Q", ctypes.c_int),
                ("seed", ctypes.c_uint64), ("R", ctypes.c_void_p), ("out_mode", ctypes.c_int),
                ("flags", ctypes.c_int), ("group_bits", ctypes.c_int),
                ("check_min_blocks", ctypes.c_int), ("cand_capacity", ctypes.c_int64),
                ("Y", ctypes.c_void_p), ("dim_y", ctypes.c_int), ("dtype_y", ctypes.c_int),
                ("masks_per_batch", ctypes.c_int), ("check_ctas_per_sm", ctypes.c_int),
                ("hash", ctypes.c_int), ("symbol_bits", ctypes.c_int), ("width", ctypes.c_float)]


# Every symbol include/msm.h declares, with its ctypes signature.
SIGNATURES = {
    "msm_version": (ctypes.c_int, []),
    "msm_set_wait_limit": (ctypes.c_int, [ctypes.c_uint32]),
    "msm_launch_count": (ctypes.c_int64, []),
    "msm_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "msm_last_error": (ctypes.c_char_p, []),
    "msm_collision_p": (ctypes.c_double, [ctypes.c_int, ctypes.c_double]),
    "msm_miss_bound": (ctypes.c_double, [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_int]),
    "msm_solve_Q": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                   ctypes.POINTER(ctypes.c_int)]),
    "msm_gaussian": (ctypes.c_int, [ctypes.c_uint64, ctypes.c_int64, vp, vp]),
    "msm_e2lsh_p": (ctypes.c_double, [ctypes.c_double]),
    "msm_e2lsh_offsets": (ctypes.c_int, [ctypes.c_uint64, ctypes.c_int64, vp, vp]),
    "msm_project_e2lsh": (ctypes.c_int, [vp, ctypes.c_int64, ctypes.c_int, ctypes.c_int, vp, vp,
                                         ctypes.c_float, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                         vp, i64p, vp]),
    "msm_enumerate_symbols": (ctypes.c_int, [vp, ctypes.c_int64, ctypes.c_int, ctypes.c_int,
                                             ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                             ctypes.c_int, ctypes.POINTER(Allocator),
                                             ctypes.POINTER(Pairs), ctypes.POINTER(Stats), vp]),
    "msm_choose_params": (ctypes.c_int, [ctypes.c_int64, ctypes.c_double, ctypes.c_double,
                                         ctypes.c_double, ctypes.POINTER(ctypes.c_int),
                                         ctypes.POINTER(ctypes.c_int),
                                         ctypes.POINTER(ctypes.c_int),
                                         ctypes.POINTER(ctypes.c_int)]),
    "msm_estimate_output": (ctypes.c_int, [vp, ctypes.c_int64, ctypes.c_int, ctypes.c_int,
                                           ctypes.c_int, ctypes.c_float, ctypes.c_int64,
                                           ctypes.c_uint64, ctypes.POINTER(ctypes.c_double),
                                           vp]),
    "msm_project": (ctypes.c_int, [vp, ctypes.c_int64, ctypes.c_int, ctypes.c_int, vp, ctypes.c_uint64,
                                   ctypes.c_int, ctypes.c_int, ctypes.c_int, vp, i64p, vp]),
    "msm_enumerate": (ctypes.c_int, [vp, ctypes.c_int64, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                     ctypes.c_int, ctypes.c_int, ctypes.POINTER(Allocator),
                                     ctypes.POINTER(Pairs), ctypes.POINTER(Stats), vp]),
    "msm_recheck": (ctypes.c_int, [vp, ctypes.c_int64, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                   ctypes.c_float, vp, ctypes.c_int64, vp, vp, i64p, i64p, vp]),
    "msm_recheck_noalloc": (ctypes.c_int, [vp, ctypes.c_int64, ctypes.c_int, ctypes.c_int,
                                           ctypes.c_int, ctypes.c_float, vp, ctypes.c_int64, vp,
                                           vp, i64p, i64p, vp]),
    "msm_eps_graph": (ctypes.c_int, [vp, ctypes.c_int64, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                     ctypes.c_float, ctypes.c_double, ctypes.POINTER(Params),
                                     ctypes.POINTER(Allocator), ctypes.POINTER(Pairs),
                                     ctypes.POINTER(Stats), vp]),
    "msm_enumerate_sets": (ctypes.c_int, [vp, i64p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                          ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                          ctypes.POINTER(Allocator), ctypes.POINTER(Pairs),
                                          ctypes.POINTER(Stats), vp]),
    "msm_eps_graph_sets": (ctypes.c_int, [vp, i64p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                          ctypes.c_int, ctypes.c_float, ctypes.c_double,
                                          ctypes.POINTER(Params), ctypes.POINTER(Allocator),
                                          ctypes.POINTER(Pairs), i64p, ctypes.POINTER(Stats), vp]),
    "msm_plan_create": (ctypes.c_int, [i64p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                       ctypes.c_int, ctypes.c_float, ctypes.c_double,
                                       ctypes.POINTER(Params), ctypes.POINTER(Allocator),
                                       ctypes.POINTER(ctypes.c_void_p)]),
    "msm_plan_input": (ctypes.c_void_p, [vp]),
    "msm_plan_run": (ctypes.c_int, [vp, vp, i64p, i64p, ctypes.POINTER(Stats), vp]),
    "msm_plan_is_graph": (ctypes.c_int, [vp]),
    "msm_plan_destroy": (None, [vp, vp]),
    "msm_autotune": (ctypes.c_int, [vp, i64p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                    ctypes.c_int, ctypes.c_float, ctypes.POINTER(Params),
                                    ctypes.c_char_p, ctypes.POINTER(Allocator), vp]),
    "msm_free_pairs": (None, [ctypes.POINTER(Pairs), ctypes.POINTER(Allocator), vp]),
    "msm_mlp_forward": (ctypes.c_int, [vp, ctypes.c_int64, ctypes.c_int, ctypes.c_int, vp, vp, vp,
                                       vp, ctypes.c_int, ctypes.c_int, vp, vp]),
    "msm_mlp_grad": (ctypes.c_int, [vp, ctypes.c_int64, ctypes.c_int, ctypes.c_int, vp, vp, vp, vp,
                                    ctypes.c_int, ctypes.c_int, vp, vp, vp, ctypes.c_int64,
                                    ctypes.c_float, ctypes.c_float, vp,
                                    ctypes.POINTER(ctypes.c_float), vp]),
    "msm_mlp_adam": (ctypes.c_int, [vp, vp, vp, vp, ctypes.c_int64, ctypes.c_int, ctypes.c_float,
                                    ctypes.c_float, ctypes.c_float, ctypes.c_float, vp, vp,
                                    ctypes.c_int, ctypes.c_int, ctypes.c_int, vp]),
    "msm_eps_count_exhaustive": (ctypes.c_int, [vp, ctypes.c_int64, ctypes.c_int, ctypes.c_int,
                                                ctypes.c_int, ctypes.c_float, i64p, vp]),
}

_handle = None


def lib_path() -> str:
    return _build.LIB


def load():
    """Load libmsm.so; raises if it has not been built."""
    global _handle
    if _handle is None:
        path = _build.LIB
        if not os.path.exists(path):
            raise ImportError(
                f"{path} is missing: build it with "
                "`python -c 'import __graft_entry__ as g; g.build()'`")
        L = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _handle = L
    return _handle
