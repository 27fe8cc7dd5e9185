"""GB300 MLMC level batch for Darcy flow in randomly layered media.

Thin ctypes binding of ``libmlmc.so`` (C ABI in ``include/mlmc.h``): argument
marshalling only; every step of the level batch runs in the library's CUDA
kernels.  PyTorch supplies device memory and the CUDA stream.

Functions keep the C names: ``mlmc_create`` -> :class:`Context`,
``mlmc_level_batch`` -> :meth:`Context.level_batch`, ``mlmc_estimate`` ->
:meth:`Context.estimate`, and so on.  There is no CPU fallback: without the
built library, or without a GPU, the calls raise.
"""
import ctypes
import os

from . import build as _build_mod

MAX_LAYERS = 8
MAX_LEVELS = 12
LIB_PATH = _build_mod.LIB

_lib = None


class Model(ctypes.Structure):
    _fields_ = [
        ("n_layers", ctypes.c_int32), ("k_kind", ctypes.c_int32),
        ("if_lo", ctypes.c_double), ("if_hi", ctypes.c_double),
        ("mu", ctypes.c_double * MAX_LAYERS), ("sigma2", ctypes.c_double * MAX_LAYERS),
        ("lam", ctypes.c_double * MAX_LAYERS),
        ("norm_r", ctypes.c_int32), ("m0", ctypes.c_int32), ("L", ctypes.c_int32),
        ("cgv", ctypes.c_int32), ("prec", ctypes.c_int32),
        ("tol", ctypes.c_double), ("max_it", ctypes.c_int32),
        ("problem", ctypes.c_int32), ("qoi_box", ctypes.c_double * 4),
        ("geometry", ctypes.c_int32), ("line_lo", ctypes.c_double * 4), ("line_hi", ctypes.c_double * 4),
        ("dim", ctypes.c_int32), ("embed", ctypes.c_int32),
    ]


SUM_FIELDS = ("s_qf", "s_qf2", "s_qc", "s_qc2", "s_y", "s_y2", "s_qcg", "s_qcg2", "s_yg", "s_yg2")


class LevelSums(ctypes.Structure):
    _fields_ = ([("n", ctypes.c_int64), ("n_failed", ctypes.c_int64), ("iters_total", ctypes.c_int64)]
                + [(k, ctypes.c_double) for k in SUM_FIELDS] + [("seconds", ctypes.c_double)])

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class EstimateOut(ctypes.Structure):
    _fields_ = [
        ("q_hat", ctypes.c_double), ("var_hat", ctypes.c_double),
        ("N", ctypes.c_int64 * MAX_LEVELS), ("V", ctypes.c_double * MAX_LEVELS),
        ("mean", ctypes.c_double * MAX_LEVELS), ("C", ctypes.c_double * MAX_LEVELS),
        ("sums", LevelSums * MAX_LEVELS), ("rounds", ctypes.c_int32), ("seconds", ctypes.c_double),
        ("alpha", ctypes.c_double), ("bias", ctypes.c_double), ("bias_flag", ctypes.c_int32),
    ]


PROFILE_CLASSES = 8


class ProfileStats(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_int64 * 4), ("ms", ctypes.c_double * 4),
                ("cell_iters", ctypes.c_double), ("cells", ctypes.c_double),
                ("fft_row_points", ctypes.c_double), ("fft_col_points", ctypes.c_double),
                ("samples", ctypes.c_double), ("solve_flops", ctypes.c_double), ("fft_flops", ctypes.c_double),
                ("solve_bytes", ctypes.c_double), ("fft_bytes", ctypes.c_double),
                ("cell_iters_c", ctypes.c_double), ("solve_flops_c", ctypes.c_double),
                ("solve_bytes_c", ctypes.c_double), ("n_classes", ctypes.c_int32)] + [
                (name, ctypes.c_int32 * PROFILE_CLASSES) for name in
                ("class_mode", "class_threads", "class_cluster", "class_smem", "class_levels",
                 "class_launches")] + [
                (name, ctypes.c_double * PROFILE_CLASSES) for name in
                ("class_ms", "class_cell_iters", "class_flops", "class_bytes")]


STAGES = ("fields", "solve", "reduce", "solve_coarse")


class TuneReport(ctypes.Structure):
    _fields_ = [("threads", ctypes.c_int32 * MAX_LEVELS), ("warp", ctypes.c_int32 * MAX_LEVELS),
                ("cap_blocks_per_sm", ctypes.c_int32 * MAX_LEVELS), ("cluster", ctypes.c_int32 * MAX_LEVELS),
                ("gamma", ctypes.c_int32 * MAX_LEVELS), ("nu", ctypes.c_int32 * MAX_LEVELS),
                ("nu_coarse", ctypes.c_int32 * MAX_LEVELS),
                ("inner_tol", ctypes.c_double * MAX_LEVELS), ("reliable", ctypes.c_int32 * MAX_LEVELS),
                ("candidates", ctypes.c_int32 * MAX_LEVELS),
                ("ms_default", ctypes.c_double * MAX_LEVELS), ("ms_best", ctypes.c_double * MAX_LEVELS),
                ("smem", ctypes.c_int32 * MAX_LEVELS),
                ("c_threads", ctypes.c_int32 * MAX_LEVELS), ("c_warp", ctypes.c_int32 * MAX_LEVELS),
                ("c_cluster", ctypes.c_int32 * MAX_LEVELS), ("c_cap_blocks_per_sm", ctypes.c_int32 * MAX_LEVELS),
                ("c_gamma", ctypes.c_int32 * MAX_LEVELS), ("c_nu", ctypes.c_int32 * MAX_LEVELS),
                ("c_nu_coarse", ctypes.c_int32 * MAX_LEVELS), ("c_inner_tol", ctypes.c_double * MAX_LEVELS),
                ("c_reliable", ctypes.c_int32 * MAX_LEVELS), ("c_smem", ctypes.c_int32 * MAX_LEVELS)]


class MLMCError(RuntimeError):
    pass


EXPORTS = {
    "mlmc_create": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(Model), ctypes.c_void_p,
                                   ctypes.POINTER(ctypes.c_void_p)]),
    "mlmc_destroy": (None, [ctypes.c_void_p]),
    "mlmc_level_batch": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_int64,
                                        ctypes.c_uint64, ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(LevelSums)]),
    "mlmc_level_batch_host": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int64,
                                             ctypes.c_int64, ctypes.c_uint64, ctypes.c_void_p,
                                             ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                             ctypes.POINTER(LevelSums)]),
    "mlmc_estimate": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_double, ctypes.c_uint64, ctypes.c_int32,
                                     ctypes.c_int32, ctypes.POINTER(EstimateOut)]),
    "mlmc_multilevel_batch": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(ctypes.c_int64),
                                             ctypes.POINTER(ctypes.c_int64), ctypes.c_uint64, ctypes.c_int32,
                                             ctypes.POINTER(LevelSums)]),
    "mlmc_multilevel_batch_host": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(ctypes.c_int64),
                                                  ctypes.POINTER(ctypes.c_int64), ctypes.c_uint64, ctypes.c_int32,
                                                  ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                                  ctypes.POINTER(LevelSums)]),
    "mlmc_autotune": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64, ctypes.POINTER(TuneReport)]),
    "mlmc_estimate_ex": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_double, ctypes.c_uint64, ctypes.c_int32,
                                        ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(EstimateOut)]),
    "mlmc_checkpoint": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_char_p]),
    "mlmc_resume": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_char_p]),
    "mlmc_checkpoint_check": (ctypes.c_int, [ctypes.POINTER(Model), ctypes.c_char_p]),
    "mlmc_set_launch": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int32, ctypes.c_int32,
                                       ctypes.c_int32, ctypes.c_int32, ctypes.c_int32]),
    "mlmc_set_launch_coarse": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int32, ctypes.c_int32,
                                              ctypes.c_int32, ctypes.c_int32, ctypes.c_int32]),
    "mlmc_set_solver": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int32, ctypes.c_double]),
    "mlmc_set_schedule": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32]),
    "mlmc_calibrate_costs": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p]),
    "mlmc_set_costs": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "mlmc_set_launch_ex": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                          ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                          ctypes.c_int32, ctypes.c_int32, ctypes.c_double]),
    "mlmc_autotune_schedule": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_double, ctypes.c_uint64, ctypes.c_int32,
                                              ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(ctypes.c_double),
                                              ctypes.POINTER(TuneReport)]),
    "mlmc_ce_info": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_int32),
                                    ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]),
    "mlmc_philox_words": (ctypes.c_int, [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64,
                                         ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int64,
                                         ctypes.c_void_p, ctypes.c_void_p]),
    "mlmc_normals": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64,
                                    ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int64, ctypes.c_void_p]),
    "mlmc_sample_fields": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_int64,
                                          ctypes.c_uint64, ctypes.c_void_p, ctypes.c_void_p]),
    "mlmc_solve_k": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p,
                                    ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "mlmc_solve_k_static": (ctypes.c_int, [ctypes.c_int, ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p,
                                           ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                           ctypes.c_double, ctypes.c_int32, ctypes.c_int32,
                                           ctypes.c_void_p]),
    "mlmc_profile": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "mlmc_profile_read": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ProfileStats)]),
    "mlmc_fma_peak": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int32, ctypes.POINTER(ctypes.c_double),
                                     ctypes.POINTER(ctypes.c_double)]),
    "mlmc_error_string": (ctypes.c_char_p, [ctypes.c_int]),
    "mlmc_last_error": (ctypes.c_char_p, []),
}


def lib():
    """The loaded library; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise MLMCError("libmlmc.so is not built (run paper_1506_04694_gb300.build.build())")
        h = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in EXPORTS.items():
            fn = getattr(h, name)
            fn.restype = res
            fn.argtypes = args
        _lib = h
    return _lib


def _check(rc, allow_failed=True):
    if rc < 0 or (rc > 0 and not allow_failed):
        L = lib()
        raise MLMCError("%s: %s" % (L.mlmc_error_string(rc).decode(), L.mlmc_last_error().decode()))
    return rc


def make_model(d):
    """C model struct from a dict with the fields of ``Model``."""
    m = Model()
    for name, ctype in Model._fields_:
        if name not in d:
            continue
        v = d[name]
        if name in ("mu", "sigma2", "lam"):
            arr = list(v) + [v[-1]] * (MAX_LAYERS - len(v))
            setattr(m, name, (ctypes.c_double * MAX_LAYERS)(*arr[:MAX_LAYERS]))
        elif name in ("qoi_box", "line_lo", "line_hi"):
            setattr(m, name, (ctypes.c_double * 4)(*v))
        else:
            setattr(m, name, v)
    return m


def _ptr(t, dtype=None):
    if t is None:
        return None
    import torch
    if not t.is_cuda:
        raise MLMCError("expected a CUDA tensor")
    if dtype is not None and t.dtype != dtype:
        raise MLMCError("expected dtype %s, got %s" % (dtype, t.dtype))
    if not t.is_contiguous():
        raise MLMCError("expected a contiguous tensor")
    del torch
    return ctypes.c_void_p(t.data_ptr())


def _stream_handle(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


class Context:
    """An ``mlmc_ctx``: model, per-level embedding tables and workspaces on one GPU."""

    def __init__(self, model, device=0, stream=None):
        import torch
        if not torch.cuda.is_available():
            raise MLMCError("no CUDA device: the MLMC level batch has no CPU fallback")
        self.model_dict = dict(model)
        self.model = make_model(model)
        self.device = device
        with torch.cuda.device(device):
            self.stream = stream if stream is not None else torch.cuda.current_stream(device)
        h = ctypes.c_void_p()
        _check(lib().mlmc_create(device, ctypes.byref(self.model), _stream_handle(self.stream),
                                 ctypes.byref(h)), allow_failed=False)
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            lib().mlmc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def m(self, level):
        return self.model.m0 << level

    def level_batch(self, level, n, seed, first=0, qf=None, qc=None, qc_cgv=None, iters=None):
        """mlmc_level_batch: per-sample outputs in the given CUDA tensors (float64
        / int32, length n, optional) and the level sums as a dict."""
        import torch
        s = LevelSums()
        rc = _check(lib().mlmc_level_batch(self._h, level, first, n, seed, _ptr(qf, torch.float64),
                                           _ptr(qc, torch.float64), _ptr(qc_cgv, torch.float64),
                                           _ptr(iters, torch.int32), ctypes.byref(s)))
        d = s.as_dict()
        d["rc"] = rc
        return d

    def level_batch_host(self, level, n, seed, first=0, want_arrays=True):
        """mlmc_level_batch_host: per-sample outputs copied to host numpy arrays."""
        import numpy as np
        s = LevelSums()
        qf = np.empty(n) if want_arrays else None
        qc = np.empty(n) if want_arrays else None
        qg = np.empty(n) if want_arrays else None
        it = np.empty(n, dtype=np.int32) if want_arrays else None
        p = (lambda a: None if a is None else a.ctypes.data_as(ctypes.c_void_p))
        rc = _check(lib().mlmc_level_batch_host(self._h, level, first, n, seed, p(qf), p(qc), p(qg),
                                                p(it), ctypes.byref(s)))
        d = s.as_dict()
        d["rc"] = rc
        return d, qf, qc, qg, it

    def estimate(self, eps, seed, n_pilot=64, cost_model=0, max_rounds=None):
        """mlmc_estimate (mlmc_estimate_ex with max_rounds): adaptive MLMC
        estimate with sampling error <= eps^2/2."""
        out = EstimateOut()
        if max_rounds is None:
            rc = _check(lib().mlmc_estimate(self._h, eps, seed, n_pilot, cost_model, ctypes.byref(out)))
        else:
            rc = _check(lib().mlmc_estimate_ex(self._h, eps, seed, n_pilot, cost_model, max_rounds,
                                               ctypes.byref(out)))
        L = self.model.L + 1
        return {"q_hat": out.q_hat, "var_hat": out.var_hat, "N": list(out.N[:L]), "V": list(out.V[:L]),
                "mean": list(out.mean[:L]), "C": list(out.C[:L]), "rounds": out.rounds,
                "seconds": out.seconds, "sums": [out.sums[i].as_dict() for i in range(L)], "rc": rc,
                "alpha": out.alpha, "bias": out.bias, "bias_flag": out.bias_flag}

    def checkpoint(self, path):
        """mlmc_checkpoint: write the last estimate's state to a file."""
        _check(lib().mlmc_checkpoint(self._h, os.fsencode(path)), allow_failed=False)

    def resume(self, path):
        """mlmc_resume: the next estimate continues from a checkpoint file."""
        _check(lib().mlmc_resume(self._h, os.fsencode(path)), allow_failed=False)

    def multilevel_batch(self, n, seed, first=None, use_graph=True):
        """mlmc_multilevel_batch: levels 0..len(n)-1 in one call; list of level-sum dicts."""
        k = len(n)
        first = first or [0] * k
        S = (LevelSums * k)()
        rc = _check(lib().mlmc_multilevel_batch(self._h, k, (ctypes.c_int64 * k)(*first), (ctypes.c_int64 * k)(*n),
                                                seed, 1 if use_graph else 0, S))
        out = [S[i].as_dict() for i in range(k)]
        for o in out:
            o["rc"] = rc
        return out

    def multilevel_batch_host(self, n, seed, first=None, use_graph=True):
        """mlmc_multilevel_batch_host: levels 0..len(n)-1 in one call, per-sample outputs copied to
        host numpy arrays; list of (level-sum dict, qf, qc, qc_cgv, iters) per level."""
        import numpy as np
        k = len(n)
        first = first or [0] * k
        arrs = [(np.empty(n[l]), np.empty(n[l]), np.empty(n[l]), np.empty(n[l], dtype=np.int32)) for l in range(k)]
        ptrs = [(ctypes.c_void_p * k)(*[arrs[l][j].ctypes.data if n[l] > 0 else None for l in range(k)])
                for j in range(4)]
        S = (LevelSums * k)()
        rc = _check(lib().mlmc_multilevel_batch_host(self._h, k, (ctypes.c_int64 * k)(*first),
                                                     (ctypes.c_int64 * k)(*n), seed, 1 if use_graph else 0,
                                                     ptrs[0], ptrs[1], ptrs[2], ptrs[3], S))
        out = []
        for l in range(k):
            d = S[l].as_dict()
            d["rc"] = rc
            out.append((d,) + arrs[l])
        return out

    def autotune(self, seed=0):
        """mlmc_autotune: time the solver's launch plans per level, keep the fastest."""
        r = TuneReport()
        _check(lib().mlmc_autotune(self._h, seed, ctypes.byref(r)), allow_failed=False)
        return self._plans(r)

    def autotune_schedule(self, eps, seed=0, n_pilot=64, cost_model=0, reps=2):
        """mlmc_autotune_schedule: launch shapes of the large levels re-timed on whole estimates under
        the work-queue schedule; returns (ms before, ms after, plans)."""
        r = TuneReport()
        ms = (ctypes.c_double * 2)()
        _check(lib().mlmc_autotune_schedule(self._h, eps, seed, n_pilot, cost_model, reps, ms, ctypes.byref(r)),
               allow_failed=False)
        return ms[0], ms[1], self._plans(r)

    def _plans(self, r):
        L = self.model.L + 1
        return [{"threads": r.threads[i], "warp": r.warp[i], "cap_blocks_per_sm": r.cap_blocks_per_sm[i],
                 "cluster": r.cluster[i], "gamma": r.gamma[i], "nu": r.nu[i], "nu_coarse": r.nu_coarse[i],
                 "inner_tol": r.inner_tol[i], "reliable": r.reliable[i],
                 "candidates": r.candidates[i], "ms_per_sample_default": r.ms_default[i],
                 "ms_per_sample_best": r.ms_best[i], "smem": r.smem[i],
                 "coarse": None if i == 0 or r.c_threads[i] == 0 else {
                     "threads": r.c_threads[i], "warp": r.c_warp[i], "cluster": r.c_cluster[i],
                     "cap_blocks_per_sm": r.c_cap_blocks_per_sm[i], "gamma": r.c_gamma[i], "nu": r.c_nu[i],
                     "nu_coarse": r.c_nu_coarse[i], "inner_tol": r.c_inner_tol[i], "reliable": r.c_reliable[i],
                     "smem": r.c_smem[i]}} for i in range(L)]

    def profile(self, enable=True):
        """mlmc_profile: reset and start (or stop) per-stage event timing."""
        _check(lib().mlmc_profile(self._h, 1 if enable else 0), allow_failed=False)

    def profile_read(self):
        """mlmc_profile_read: per-stage launches and milliseconds plus work counters."""
        p = ProfileStats()
        _check(lib().mlmc_profile_read(self._h, ctypes.byref(p)), allow_failed=False)
        return {"launches": dict(zip(STAGES, p.launches)), "ms": dict(zip(STAGES, p.ms)),
                "cell_iters": p.cell_iters, "cells": p.cells, "fft_row_points": p.fft_row_points,
                "fft_col_points": p.fft_col_points, "samples": p.samples, "solve_flops": p.solve_flops,
                "fft_flops": p.fft_flops, "solve_bytes": p.solve_bytes, "fft_bytes": p.fft_bytes,
                "cell_iters_c": p.cell_iters_c, "solve_flops_c": p.solve_flops_c, "solve_bytes_c": p.solve_bytes_c,
                "classes": [{"mode": p.class_mode[k], "threads": p.class_threads[k],
                             "cluster": p.class_cluster[k], "smem": p.class_smem[k],
                             "levels": [l for l in range(MAX_LEVELS) if p.class_levels[k] >> l & 1],
                             "launches": p.class_launches[k], "ms": p.class_ms[k],
                             "cell_iters": p.class_cell_iters[k], "flops": p.class_flops[k],
                             "bytes": p.class_bytes[k]} for k in range(p.n_classes)]}

    def set_launch(self, level, mode, threads=256, cluster=0, gamma=1, nu=1):
        """mlmc_set_launch: fix a level's solver launch (0 block, 1 warp, 2 cluster; <0 default),
        its multigrid cycle (gamma 1 V, 2 W) and smoothing sweep pairs nu."""
        _check(lib().mlmc_set_launch(self._h, level, mode, threads, cluster, gamma, nu), allow_failed=False)

    def set_launch_coarse(self, level, mode, threads=256, cluster=0, gamma=1, nu=1):
        """mlmc_set_launch_coarse: a launch plan of its own for the coarse systems of a level >= 1
        (mode < 0: one launch for all the level's systems again)."""
        _check(lib().mlmc_set_launch_coarse(self._h, level, mode, threads, cluster, gamma, nu), allow_failed=False)

    def set_plan(self, level, plan, part=0):
        """mlmc_set_launch_ex: replay one plan dict as autotune() / autotune_schedule() report it
        (part 0 the fine systems, 1 the coarse ones)."""
        mode = 2 if plan["cluster"] else 3 if plan["warp"] == 2 else 1 if plan["warp"] else 0
        _check(lib().mlmc_set_launch_ex(self._h, level, part, mode, plan["threads"], plan["cluster"], plan["gamma"],
                                        plan["nu"], plan["nu_coarse"], plan["cap_blocks_per_sm"], plan["reliable"],
                                        plan["inner_tol"]), allow_failed=False)

    def set_plans(self, plans):
        """Replay a whole list of per-level plans (fine, and coarse where the level has its own)."""
        for level, p in enumerate(plans):
            self.set_plan(level, p, 0)
            if p.get("coarse"):
                self.set_plan(level, p["coarse"], 1)

    def set_solver(self, level, reliable, inner_tol):
        """mlmc_set_solver: mixed-precision scheme of a level (reliable updates or restarted
        refinement) and its FP32 tolerance."""
        _check(lib().mlmc_set_solver(self._h, level, reliable, inner_tol), allow_failed=False)

    def calibrate_costs(self, seed=0):
        """mlmc_calibrate_costs: per-sample GPU seconds of each level at GPU-filling batch sizes,
        kept for estimates with cost_model=2; returns the list."""
        L = self.model.L + 1
        C = (ctypes.c_double * L)()
        _check(lib().mlmc_calibrate_costs(self._h, seed, C), allow_failed=False)
        return list(C)

    def set_costs(self, costs):
        """mlmc_set_costs: fix the per-sample costs used by estimates with cost_model=2."""
        L = self.model.L + 1
        C = (ctypes.c_double * L)(*costs[:L])
        _check(lib().mlmc_set_costs(self._h, C), allow_failed=False)

    def set_schedule(self, schedule):
        """mlmc_set_schedule: 1 = one work-queue launch per launch shape across the levels of a
        multilevel batch, 0 = one launch chain per level."""
        _check(lib().mlmc_set_schedule(self._h, schedule), allow_failed=False)

    def ce_info(self, level):
        M = ctypes.c_int32()
        lo = ctypes.c_double()
        hi = ctypes.c_double()
        _check(lib().mlmc_ce_info(self._h, level, ctypes.byref(M), ctypes.byref(lo), ctypes.byref(hi)))
        return M.value, lo.value, hi.value

    def normals(self, seed, level, sample, stream_id, first_call, n_calls):
        """mlmc_normals: the four Box-Muller normals of each Philox call, [n_calls, 4]."""
        import torch
        out = torch.empty((n_calls, 4), dtype=torch.float64, device="cuda:%d" % self.device)
        _check(lib().mlmc_normals(self._h, seed, level, sample, stream_id, first_call, n_calls, _ptr(out)),
               allow_failed=False)
        return out

    def sample_fields(self, level, n, seed, first=0):
        """mlmc_sample_fields: fine per-layer fields g [n, n_layers, m, m] (3-D:
        [n, n_layers, m, m, m]) and sorted interfaces [n, n_layers-1], as CUDA
        float64 tensors."""
        import torch
        m = self.m(level)
        nl = self.model.n_layers
        shape = (n, nl, m, m, m) if self.model.dim == 3 else (n, nl, m, m)
        g = torch.empty(shape, dtype=torch.float64, device="cuda:%d" % self.device)
        n_ends = 4 if self.model.geometry == 1 else nl - 1
        eta = torch.empty((n, max(n_ends, 1)), dtype=torch.float64, device=g.device)
        _check(lib().mlmc_sample_fields(self._h, level, first, n, seed, _ptr(g), _ptr(eta)),
               allow_failed=False)
        return g, eta[:, :n_ends]

    def solve_k(self, k, want_p=True):
        """mlmc_solve_k: solve the systems of a CUDA float64 tensor k [n, m, m]
        (3-D contexts: [n, m, m, m]); returns (p or None, Q, iterations)."""
        import torch
        n, m = _check_systems(k, 3 if self.model.dim == 3 else 2)
        if k.device != torch.device("cuda", self.device):
            raise MLMCError("k is on %s, the context on cuda:%d" % (k.device, self.device))
        q = torch.empty(n, dtype=torch.float64, device=k.device)
        it = torch.empty(n, dtype=torch.int32, device=k.device)
        p = torch.empty_like(k) if want_p else None
        _check(lib().mlmc_solve_k(self._h, m, n, _ptr(k.contiguous(), torch.float64), _ptr(p), _ptr(q),
                                  _ptr(it)), allow_failed=False)
        return p, q, it


def _check_systems(k, dim=2):
    """Shape checks of a solver input k [n, m, m] (3-D: [n, m, m, m])."""
    if k.dim() != dim + 1 or any(k.shape[d] != k.shape[1] for d in range(2, dim + 1)):
        raise MLMCError("k must be [n, m, m]%s with equal sides, got %s"
                        % (" (3-D: [n, m, m, m])" if dim == 3 else "", tuple(k.shape)))
    return k.shape[0], k.shape[1]


def solve_k_static(k, q, p=None, iters=None, tol=1e-10, max_it=500, prec=0, stream=None):
    """mlmc_solve_k_static: the solver with no device allocation at all, for
    callers that cannot allocate; the caller supplies every output tensor
    (q float64 [n]; optional p float64 [n, m, m] and iters int32 [n]), all on
    k's device.  The work is queued on `stream` (default: the current stream
    of k's device) and not waited for."""
    import torch
    n, m = _check_systems(k)
    dev = k.device
    if dev.type != "cuda":
        raise MLMCError("k must be a CUDA tensor")
    for name, t in (("q", q), ("p", p), ("iters", iters)):
        if t is not None and t.device != dev:
            raise MLMCError("%s is on %s, k on %s: every tensor must be on k's device" % (name, t.device, dev))
    if q.numel() < n:
        raise MLMCError("q holds %d values, needs n = %d" % (q.numel(), n))
    if iters is not None and iters.numel() < n:
        raise MLMCError("iters holds %d values, needs n = %d" % (iters.numel(), n))
    if p is not None and tuple(p.shape) != tuple(k.shape):
        raise MLMCError("p must have k's shape %s, got %s" % (tuple(k.shape), tuple(p.shape)))
    if stream is None:
        stream = torch.cuda.current_stream(dev)
    elif stream.device != dev:
        raise MLMCError("the stream belongs to %s, k to %s" % (stream.device, dev))
    rc = lib().mlmc_solve_k_static(dev.index, m, n, _ptr(k, torch.float64), _ptr(p, torch.float64),
                                   _ptr(q, torch.float64), _ptr(iters, torch.int32), tol, max_it, prec,
                                   ctypes.c_void_p(stream.cuda_stream))
    if rc != 0:
        raise MLMCError("mlmc_solve_k_static: %s: %s" % (lib().mlmc_error_string(rc).decode(),
                                                        lib().mlmc_last_error().decode()))


def checkpoint_check(model, path):
    """mlmc_checkpoint_check: raises MLMCError unless the checkpoint file at
    `path` was written for `model` (a dict with the fields of ``Model``);
    needs no GPU."""
    m = make_model(model)
    _check(lib().mlmc_checkpoint_check(ctypes.byref(m), os.fsencode(path)), allow_failed=False)


def fma_peak(device=0, fp64=True, iters=20000):
    """mlmc_fma_peak: measured FMA throughput of the GPU in TFLOP/s (and the
    probe kernel's event time in ms)."""
    t = ctypes.c_double()
    ms = ctypes.c_double()
    _check(lib().mlmc_fma_peak(device, 1 if fp64 else 0, iters, ctypes.byref(t), ctypes.byref(ms)),
           allow_failed=False)
    return t.value, ms.value


def philox_words(seed, level, sample, stream_id, first_call, n_calls, device=0):
    """mlmc_philox_words: raw Philox4x64-10 words [n_calls, 4] as a CUDA int64
    tensor (bit patterns of the uint64 words)."""
    import torch
    out = torch.empty((n_calls, 4), dtype=torch.int64, device="cuda:%d" % device)
    _check(lib().mlmc_philox_words(seed, level, sample, stream_id, first_call, n_calls, _ptr(out),
                                   _stream_handle(None)), allow_failed=False)
    return out
