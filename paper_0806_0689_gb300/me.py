"""Thin ctypes binding of libme (include/me.h): argument marshalling only.

Every function here forwards to the C-ABI entry point of the same name;
frames and outputs are torch CUDA tensors whose device pointers are passed
through.  There is no fallback: if libme.so is missing or no sm_103 device is
present the calls raise.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

ME_OK, ME_ERR_ARG, ME_ERR_CUDA, ME_ERR_UNSUPPORTED, ME_ERR_TIMEOUT, ME_ERR_NOMEM = range(6)
ME_ALGO_FS, ME_ALGO_DCDS, ME_ALGO_DCDS_S, ME_ALGO_DCDS_LEARNED = range(4)
ME_MAX_RANGE = 32
ME_STATIC_MAX_FRAMES = 64
ME_NSUMS = 8
ALGOS = {"fs": ME_ALGO_FS, "dcds": ME_ALGO_DCDS, "dcds_s": ME_ALGO_DCDS_S, "dcds_learned": ME_ALGO_DCDS_LEARNED}

EXPORTS = ["me_init", "me_free", "me_last_error", "me_estimate", "me_estimate_batch", "me_graph_create",
           "me_graph_launch", "me_graph_free", "me_eval", "me_eval_batch", "me_stats_from_sums", "me_tune",
           "me_absdiff_peak", "me_check_status", "me_estimate_batch_noalloc", "me_tune_batch",
           "me_proposal_create", "me_proposal_free", "me_proposal_set_params", "me_proposal_get_params",
           "me_proposal_train_step", "me_proposal_logits", "me_estimate_learned_batch",
           "me_estimate_eval_batch", "me_graph_create_eval", "me_estimate_median_batch", "me_mvp_stats",
           "me_fs_dual_batch", "me_estimate_host_batch", "me_inject_wait_timeout", "me_proposal_save",
           "me_proposal_load", "me_set_tracing", "me_last_call_ms", "me_noalloc_check_status",
           "me_proposal_train"]
ME_PROPOSAL_NPARAMS = 37668
ME_PROPOSAL_NLOGITS = 68


class MeError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"libme error {code}: {msg}")
        self.code = code


class FrameDesc(ctypes.Structure):
    _fields_ = [("cur", ctypes.c_void_p), ("ref", ctypes.c_void_p), ("w", ctypes.c_int32),
                ("h", ctypes.c_int32), ("pitch", ctypes.c_int32), ("range", ctypes.c_int32),
                ("mv", ctypes.c_void_p), ("sad", ctypes.c_void_p), ("nsp", ctypes.c_void_p)]


class EvalDesc(ctypes.Structure):
    _fields_ = [("cur", ctypes.c_void_p), ("ref", ctypes.c_void_p), ("w", ctypes.c_int32),
                ("h", ctypes.c_int32), ("pitch", ctypes.c_int32), ("mv", ctypes.c_void_p),
                ("mv_fs", ctypes.c_void_p), ("nsp", ctypes.c_void_p)]


class TrainCfg(ctypes.Structure):
    _fields_ = [("descs", ctypes.c_void_p), ("n", ctypes.c_int32), ("steps", ctypes.c_int32),
                ("pairs_per_step", ctypes.c_int32), ("lr", ctypes.c_float), ("seed", ctypes.c_uint64),
                ("losses", ctypes.c_void_p), ("stream", ctypes.c_void_p)]


class Stats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in ("mad", "mse", "nsp", "psnr", "distance", "probability")]


_lock = threading.Lock()
_lib = None


def lib_path():
    return _build.paths(_build.variant())[1]


def load(build_if_missing: bool = True):
    """Load libme.so (building it first if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build() if build_if_missing else lib_path()
            if not os.path.exists(path):
                raise FileNotFoundError(f"{path} is missing; run paper_0806_0689_gb300.build")
            L = ctypes.CDLL(path)
            P, I = ctypes.c_void_p, ctypes.c_int
            L.me_init.argtypes = [ctypes.POINTER(P), I, ctypes.c_char_p]
            L.me_free.argtypes = [P]
            L.me_free.restype = None
            L.me_last_error.argtypes = [P]
            L.me_last_error.restype = ctypes.c_char_p
            L.me_estimate.argtypes = [P, P, P, I, I, I, I, I, P, P, P, P]
            L.me_estimate_batch.argtypes = [P, ctypes.POINTER(FrameDesc), I, I, I, P]
            L.me_graph_create.argtypes = [P, ctypes.POINTER(FrameDesc), I, I, I, ctypes.POINTER(P)]
            L.me_graph_launch.argtypes = [P, P, P]
            L.me_graph_free.argtypes = [P]
            L.me_graph_free.restype = None
            L.me_eval.argtypes = [P, P, P, I, I, I, P, P, P, P, P]
            L.me_eval_batch.argtypes = [P, ctypes.POINTER(EvalDesc), I, I, P, P]
            L.me_stats_from_sums.argtypes = [P, ctypes.POINTER(Stats)]
            L.me_tune.argtypes = [P, P, P, I, I, I, I, I, P, P, P, ctypes.POINTER(I), P]
            L.me_tune_batch.argtypes = [P, ctypes.POINTER(FrameDesc), I, I, I, ctypes.POINTER(I), P]
            L.me_absdiff_peak.argtypes = [P, I, ctypes.POINTER(ctypes.c_double), I, ctypes.POINTER(I), P]
            L.me_check_status.argtypes = [P, P]
            L.me_estimate_batch_noalloc.argtypes = [ctypes.POINTER(FrameDesc), I, I, I, P, ctypes.c_char_p, I]
            L.me_noalloc_check_status.argtypes = [P, ctypes.c_char_p, I]
            L.me_proposal_create.argtypes = [P, ctypes.POINTER(P)]
            L.me_proposal_free.argtypes = [P]
            L.me_proposal_free.restype = None
            L.me_proposal_set_params.argtypes = [P, P, P]
            L.me_proposal_get_params.argtypes = [P, P, P]
            L.me_proposal_save.argtypes = [P, P, ctypes.c_char_p]
            L.me_proposal_load.argtypes = [P, P, ctypes.c_char_p]
            L.me_proposal_train_step.argtypes = [P, P, ctypes.POINTER(FrameDesc), I, ctypes.c_float,
                                                 ctypes.POINTER(ctypes.c_float), P, P]
            L.me_proposal_logits.argtypes = [P, P, ctypes.POINTER(FrameDesc), P, P]
            L.me_estimate_learned_batch.argtypes = [P, P, ctypes.POINTER(FrameDesc), I, I, P, P]
            L.me_proposal_train.argtypes = [P, P, ctypes.POINTER(TrainCfg)]
            L.me_estimate_host_batch.argtypes = [P, ctypes.POINTER(FrameDesc), P, I, I, I, P, I, P]
            L.me_estimate_eval_batch.argtypes = [P, ctypes.POINTER(FrameDesc), P, I, I, I, P, P]
            L.me_graph_create_eval.argtypes = [P, ctypes.POINTER(FrameDesc), P, I, I, I, P, ctypes.POINTER(P)]
            L.me_fs_dual_batch.argtypes = [P, ctypes.POINTER(FrameDesc), ctypes.POINTER(FrameDesc), I, P]
            L.me_mvp_stats.argtypes = [P, ctypes.POINTER(FrameDesc), I, I, P, P]
            L.me_estimate_median_batch.argtypes = [P, ctypes.POINTER(FrameDesc), I, I, P, P]
            L.me_inject_wait_timeout.argtypes = [P, I]
            L.me_set_tracing.argtypes = [P, I]
            L.me_last_call_ms.argtypes = [P, ctypes.POINTER(ctypes.c_float)]
            missing = [n for n in EXPORTS if getattr(L, n).argtypes is None]
            assert not missing, f"argument types not declared for {missing}"
            for n in EXPORTS:
                if n not in ("me_free", "me_last_error", "me_graph_free", "me_proposal_free"):
                    getattr(L, n).restype = I
            _lib = L
    return _lib


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream) if hasattr(stream, "cuda_stream") else ctypes.c_void_p(stream)


class Context:
    """Owns one me_ctx.  Methods mirror the C-ABI entry points."""

    def __init__(self, device: int = 0, tune_cache_path: str | None = None):
        self.L = load()
        self.h = ctypes.c_void_p()
        rc = self.L.me_init(ctypes.byref(self.h), device,
                            tune_cache_path.encode() if tune_cache_path else None)
        if rc != ME_OK:
            raise MeError(rc, "me_init failed (no sm_103 device, or CUDA unavailable)")

    def close(self):
        if self.h:
            self.L.me_free(self.h)
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc):
        if rc != ME_OK:
            raise MeError(rc, self.L.me_last_error(self.h).decode())

    # -- search -----------------------------------------------------------
    def me_estimate(self, cur, ref, block, rng, algo, mv, sad, nsp=None, stream=None):
        h, w = cur.shape[-2:]
        self._check(self.L.me_estimate(self.h, _ptr(cur), _ptr(ref), w, h, block, rng, ALGOS.get(algo, algo),
                                       _ptr(mv), _ptr(sad), _ptr(nsp), _stream(stream)))

    @staticmethod
    def frame_descs(items):
        """items: iterable of (cur, ref, range, mv, sad, nsp) torch tensors."""
        items = list(items)
        arr = (FrameDesc * len(items))()
        for i, (cur, ref, rng, mv, sad, nsp) in enumerate(items):
            h, w = cur.shape[-2:]
            arr[i] = FrameDesc(cur.data_ptr(), ref.data_ptr(), w, h, cur.stride(-2), rng, mv.data_ptr(),
                               sad.data_ptr(), None if nsp is None else nsp.data_ptr())
        return arr

    def me_estimate_batch(self, descs, block, algo, stream=None):
        self._check(self.L.me_estimate_batch(self.h, descs, len(descs), block, ALGOS.get(algo, algo),
                                             _stream(stream)))

    def me_graph_create(self, descs, block, algo):
        g = ctypes.c_void_p()
        self._check(self.L.me_graph_create(self.h, descs, len(descs), block, ALGOS.get(algo, algo),
                                           ctypes.byref(g)))
        return g

    @staticmethod
    def _fs_ptrs(mv_fs, n):
        if mv_fs is None:
            return None
        arr = (ctypes.c_void_p * n)(*[None if t is None else t.data_ptr() for t in mv_fs])
        return arr

    def me_estimate_eval_batch(self, descs, mv_fs, block, algo, sums, stream=None):
        """DCDS with the evaluation sums fused in; mv_fs: list of device
        tensors (or None entries) or None; sums: device int64 [n][ME_NSUMS]."""
        arr = self._fs_ptrs(mv_fs, len(descs))
        self._check(self.L.me_estimate_eval_batch(self.h, descs, arr, len(descs), block, ALGOS.get(algo, algo),
                                                  _ptr(sums), _stream(stream)))

    def me_estimate_host_batch(self, descs, block, algo, mv_fs=None, sums=None, chunk=0, stream=None):
        """The search (with sums: search and evaluation) on HOST tensors,
        pinned for the copies to overlap; descs built by frame_descs from
        host tensors; mv_fs: list of host tensors (or None entries) or None;
        sums: host int64 [n][ME_NSUMS] or None; chunk: pairs per chunk (0:
        the library's choice)."""
        arr = self._fs_ptrs(mv_fs, len(descs))
        self._check(self.L.me_estimate_host_batch(self.h, descs, arr,
                                                  len(descs), block, ALGOS.get(algo, algo), _ptr(sums), chunk,
                                                  _stream(stream)))

    def me_graph_create_eval(self, descs, mv_fs, block, algo, sums):
        g = ctypes.c_void_p()
        arr = self._fs_ptrs(mv_fs, len(descs))
        self._check(self.L.me_graph_create_eval(self.h, descs, arr, len(descs), block, ALGOS.get(algo, algo),
                                                _ptr(sums), ctypes.byref(g)))
        return g

    def me_graph_launch(self, g, stream=None):
        self._check(self.L.me_graph_launch(self.h, g, _stream(stream)))

    def me_graph_free(self, g):
        self.L.me_graph_free(g)

    # -- evaluation -------------------------------------------------------
    def me_eval(self, cur, ref, block, mv, sums, mv_fs=None, nsp=None, stream=None):
        h, w = cur.shape[-2:]
        self._check(self.L.me_eval(self.h, _ptr(cur), _ptr(ref), w, h, block, _ptr(mv), _ptr(mv_fs), _ptr(nsp),
                                   _ptr(sums), _stream(stream)))

    @staticmethod
    def eval_descs(items):
        """items: iterable of (cur, ref, mv, mv_fs, nsp) torch tensors (mv_fs, nsp may be None)."""
        items = list(items)
        arr = (EvalDesc * len(items))()
        for i, (cur, ref, mv, mv_fs, nsp) in enumerate(items):
            h, w = cur.shape[-2:]
            arr[i] = EvalDesc(cur.data_ptr(), ref.data_ptr(), w, h, cur.stride(-2), mv.data_ptr(),
                              None if mv_fs is None else mv_fs.data_ptr(), None if nsp is None else nsp.data_ptr())
        return arr

    def me_eval_batch(self, descs, block, sums, stream=None):
        self._check(self.L.me_eval_batch(self.h, descs, len(descs), block, _ptr(sums), _stream(stream)))

    def me_stats_from_sums(self, sums_row):
        a = np.ascontiguousarray(np.asarray(sums_row, dtype=np.uint64))
        st = Stats()
        self._check(self.L.me_stats_from_sums(ctypes.c_void_p(a.ctypes.data), ctypes.byref(st)))
        return {n: getattr(st, n) for n, _ in Stats._fields_}

    # -- tuning / microbenchmark / status -----------------------------------
    def me_tune(self, cur, ref, block, rng, algo, mv, sad, nsp=None, stream=None):
        h, w = cur.shape[-2:]
        chosen = ctypes.c_int(-1)
        self._check(self.L.me_tune(self.h, _ptr(cur), _ptr(ref), w, h, block, rng, ALGOS.get(algo, algo),
                                   _ptr(mv), _ptr(sad), _ptr(nsp), ctypes.byref(chosen), _stream(stream)))
        return chosen.value

    def me_tune_batch(self, descs, block, algo, stream=None):
        chosen = ctypes.c_int(-1)
        self._check(self.L.me_tune_batch(self.h, descs, len(descs), block, ALGOS.get(algo, algo),
                                         ctypes.byref(chosen), _stream(stream)))
        return chosen.value

    def me_absdiff_peak(self, iters=4096, n_variants=4, stream=None):
        out = (ctypes.c_double * n_variants)()
        used = ctypes.c_int(-1)
        self._check(self.L.me_absdiff_peak(self.h, iters, out, n_variants, ctypes.byref(used), _stream(stream)))
        return list(out), used.value

    # -- learned start proposal ----------------------------------------------
    def me_proposal_create(self):
        h = ctypes.c_void_p()
        self._check(self.L.me_proposal_create(self.h, ctypes.byref(h)))
        return h

    def me_proposal_free(self, prop):
        self.L.me_proposal_free(prop)

    def me_proposal_set_params(self, prop, params):
        a = np.ascontiguousarray(params, dtype=np.float32)
        assert a.size == ME_PROPOSAL_NPARAMS
        self._check(self.L.me_proposal_set_params(self.h, prop, ctypes.c_void_p(a.ctypes.data)))

    def me_proposal_get_params(self, prop):
        a = np.zeros(ME_PROPOSAL_NPARAMS, np.float32)
        self._check(self.L.me_proposal_get_params(self.h, prop, ctypes.c_void_p(a.ctypes.data)))
        return a

    def me_proposal_save(self, prop, path):
        self._check(self.L.me_proposal_save(self.h, prop, os.fsencode(path)))

    def me_proposal_load(self, prop, path):
        self._check(self.L.me_proposal_load(self.h, prop, os.fsencode(path)))

    def me_proposal_train_step(self, prop, descs, lr, want_grad=False, stream=None):
        loss = ctypes.c_float(0.0)
        g = np.zeros(ME_PROPOSAL_NPARAMS, np.float32) if want_grad else None
        self._check(self.L.me_proposal_train_step(self.h, prop, descs, len(descs), lr, ctypes.byref(loss),
                                                  None if g is None else ctypes.c_void_p(g.ctypes.data),
                                                  _stream(stream)))
        return (loss.value, g) if want_grad else loss.value

    def me_proposal_logits(self, prop, desc, logits, stream=None):
        self._check(self.L.me_proposal_logits(self.h, prop, desc, _ptr(logits), _stream(stream)))

    def me_estimate_learned_batch(self, prop, descs, starts=None, stream=None, block=16):
        self._check(self.L.me_estimate_learned_batch(self.h, prop, descs, len(descs), block, _ptr(starts),
                                                     _stream(stream)))

    def me_fs_dual_batch(self, d16, d8, stream=None):
        """Full search for 16x16 (d16) and 8x8 (d8: outputs only) in one sweep."""
        self._check(self.L.me_fs_dual_batch(self.h, d16, d8, len(d16), _stream(stream)))

    def me_mvp_stats(self, descs, rng, out, stream=None):
        """Counts of the Sec. II-C statistics; out: device int64 [35 * (2*rng+1)**2]."""
        self._check(self.L.me_mvp_stats(self.h, descs, len(descs), rng, _ptr(out), _stream(stream)))

    def me_estimate_median_batch(self, descs, starts=None, stream=None, block=16):
        self._check(self.L.me_estimate_median_batch(self.h, descs, len(descs), block, _ptr(starts),
                                                    _stream(stream)))

    def me_check_status(self, stream=None):
        self._check(self.L.me_check_status(self.h, _stream(stream)))

    def me_set_tracing(self, on):
        self._check(self.L.me_set_tracing(self.h, int(bool(on))))

    def me_last_call_ms(self):
        ms = ctypes.c_float(0.0)
        self._check(self.L.me_last_call_ms(self.h, ctypes.byref(ms)))
        return ms.value

    def me_inject_wait_timeout(self, on):
        """Failure-detection test hook: while on, DCDS tile-kernel launches
        give up their first copy's (bounded) wait and report ME_ERR_TIMEOUT."""
        self._check(self.L.me_inject_wait_timeout(self.h, int(bool(on))))


def proposal_init_params(seed=0):
    """He-normal initial parameters of the proposal network (host, float32, the
    parameter order of include/me.h)."""
    rng = np.random.default_rng(seed)
    parts = []
    for cin in (2, 32, 32, 32):
        parts.append(rng.normal(0.0, np.sqrt(2.0 / (9 * cin)), 32 * cin * 9))
        parts.append(np.full(32, 0.01))
    parts.append(rng.normal(0.0, np.sqrt(1.0 / 136), 68 * 136))
    parts.append(np.zeros(68))
    p = np.concatenate(parts).astype(np.float32)
    assert p.size == ME_PROPOSAL_NPARAMS
    return p


def train_proposal(ctx, prop, descs, steps, lr=2e-3, pairs_per_step=2, seed=0, stream=None):
    """me_proposal_train: `steps` training steps over pairs drawn from descs
    (a FrameDesc array whose mv fields hold the label fields); the loop runs in
    the library.  prop None trains the context's own proposal.  Returns the
    list of step losses."""
    losses = np.zeros(max(steps, 1), np.float32)
    cfg = TrainCfg(ctypes.cast(descs, ctypes.c_void_p).value, len(descs), steps, min(pairs_per_step, len(descs)),
                   lr, seed, losses.ctypes.data, _stream(stream).value)
    ctx._check(ctx.L.me_proposal_train(ctx.h, prop, ctypes.byref(cfg)))
    return losses[:steps].tolist()
