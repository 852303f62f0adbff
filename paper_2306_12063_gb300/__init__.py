"""Python binding of libldpc (include/ldpc.h): layered min-sum decoding and
direct encoding of QC-LDPC codes on GB300.

This layer only marshals arguments: torch supplies device memory and the
current CUDA stream, every step of the work runs in the library's kernels.
Importing works without a GPU; any call that would launch work raises if the
compiled library is missing (run ``_build.build()``), never falls back.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Tuple

import numpy as np

from . import _build

__all__ = ["LdpcError", "Code", "load", "gen_info", "awgn_llr", "quantize_pack_i8",
           "awgn_llr_frames", "snr_sigma", "adam_step", "CodeSet", "MixedPlan", "MixedGraph",
           "quantize_i16", "set_grid_cap", "F32", "I8X4", "I16W", "symbols"]

F32 = 0
I8X4 = 1
I16W = 2

_STATUS = {0: "OK", 1: "INVALID_ARG", 2: "BAD_STRUCTURE", 3: "NOMEM", 4: "CUDA",
           5: "TIMEOUT", 6: "UNSUPPORTED"}


class LdpcError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"libldpc {_STATUS.get(status, status)}: {msg}")
        self.status = status


class _Params(ctypes.Structure):
    _fields_ = [("max_iters", ctypes.c_int), ("alpha", ctypes.c_float),
                ("normalise", ctypes.c_int), ("early_stop", ctypes.c_int)]


class _GroupLaunch(ctypes.Structure):
    _fields_ = [("frames_per_item", ctypes.c_int), ("blocks_per_sm", ctypes.c_int),
                ("warps_per_frame", ctypes.c_int), ("frames_per_block", ctypes.c_int)]


class _LearnedParams(ctypes.Structure):
    _fields_ = [("max_iters", ctypes.c_int), ("early_stop", ctypes.c_int),
                ("stop_iter", ctypes.c_int * 2), ("stop_frac", ctypes.c_float * 2)]


def _learned_params(max_iters, early_stop, stop_iter, stop_frac):
    lp = _LearnedParams()
    lp.max_iters = int(max_iters or 0)
    lp.early_stop = int(bool(early_stop))
    for j in range(2):
        lp.stop_iter[j] = int(stop_iter[j])
        lp.stop_frac[j] = float(stop_frac[j])
    return lp


_lib = None


def symbols():
    """Function names declared in include/ldpc.h."""
    import re
    hdr = os.path.join(_build.ROOT, "include", "ldpc.h")
    txt = open(hdr).read()
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\s*\**\s*(ldpc_\w+)\s*\(", txt, re.M)))


def load(build_if_missing: bool = False):
    """The loaded library (ctypes).  Raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_build.LIB):
        if not build_if_missing:
            raise RuntimeError(f"libldpc is not built ({_build.LIB} missing); "
                               "run paper_2306_12063_gb300._build.build()")
        _build.build()
    L = ctypes.CDLL(_build.LIB)
    vp, i32, i64, u64, f32, sz = (ctypes.c_void_p, ctypes.c_int, ctypes.c_int64,
                                  ctypes.c_uint64, ctypes.c_float, ctypes.c_size_t)
    P = ctypes.POINTER
    sig = {
        "ldpc_set_device": ([i32], i32),
        "ldpc_code_create": ([vp, i32, i32, i32, P(vp)], i32),
        "ldpc_code_destroy": ([vp], None),
        "ldpc_code_info": ([vp, P(i32), P(i32), P(i32), P(i32), P(i32)], i32),
        "ldpc_gen_info": ([u64, i64, i64, i32, vp, vp], i32),
        "ldpc_encode": ([vp, vp, vp, i64, vp], i32),
        "ldpc_awgn_llr": ([vp, i64, i64, i32, u64, f32, f32, vp, vp], i32),
        "ldpc_quantize_pack_i8": ([vp, vp, i64, i32, f32, i32, vp], i32),
        "ldpc_decode_layered_minsum": ([vp, i32, vp, i64, P(_Params), vp, vp, vp, vp], i32),
        "ldpc_frame_stats": ([vp, vp, vp, vp, i64, i32, vp, vp], i32),
        "ldpc_paired_frame_errors": ([vp, vp, vp, vp, i64, vp, vp], i32),
        "ldpc_decode_host_workspace_bytes": ([vp, i32, i64], sz),
        "ldpc_decode_host": ([vp, i32, vp, i64, P(_Params), vp, vp, vp, sz, i64, vp], i32),
        "ldpc_sync": ([vp, vp, ctypes.c_double], i32),
        "ldpc_decode_layered_minsum_noalloc": ([vp, i32, i32, i32, i32, vp, i64, P(_Params),
                                                vp, vp, vp, vp], i32),
        "ldpc_decode_learned_minsum": ([vp, vp, i64, vp, i32, i32, vp, vp, vp, vp], i32),
        "ldpc_decode_learned_minsum_ex": ([vp, vp, i64, vp, i32, P(_LearnedParams), vp, vp, vp,
                                           vp], i32),
        "ldpc_decode_mixed_learned_ex": ([vp, vp, P(_LearnedParams), vp, vp, vp, vp], i32),
        "ldpc_mixed_autotune_learned": ([vp, vp, P(_LearnedParams), vp, vp, i32, vp], i32),
        "ldpc_mixed_group_launch": ([vp, i32, i32, P(_GroupLaunch), P(_GroupLaunch)], i32),
        "ldpc_learned_fallback_workspace_bytes": ([vp, i64], sz),
        "ldpc_decode_learned_fallback": ([vp, vp, i64, vp, i32, P(_Params), f32, i32, vp, vp,
                                          P(i64), vp, sz, vp], i32),
        "ldpc_learned_train_forward": ([vp, vp, vp, i64, vp, i32, vp, vp, vp, f32, vp, vp], i32),
        "ldpc_learned_train_workspace_bytes": ([vp, i64, i32], sz),
        "ldpc_learned_train_backward": ([vp, vp, vp, i64, vp, i32, vp, vp, f32, vp, vp, vp, sz,
                                         vp], i32),
        "ldpc_adam_step": ([vp, vp, vp, vp, i64, i32, f32, f32, f32, f32, vp], i32),
        "ldpc_snr_sigma": ([u64, i64, i64, f32, f32, f32, vp, vp], i32),
        "ldpc_awgn_llr_frames": ([vp, i64, i64, i32, u64, vp, vp, vp], i32),
        "ldpc_codeset_create": ([vp, i32, P(vp)], i32),
        "ldpc_codeset_destroy": ([vp], None),
        "ldpc_mixed_plan_create": ([vp, vp, i64, P(vp)], i32),
        "ldpc_mixed_plan_destroy": ([vp], None),
        "ldpc_mixed_plan_sizes": ([vp, P(i64), P(i64), P(i64), P(i64), P(i32)], i32),
        "ldpc_mixed_plan_offsets": ([vp, vp, vp, vp], i32),
        "ldpc_mixed_group_info": ([vp, i32] + [P(i32)] * 8, i32),
        "ldpc_mixed_quantize": ([vp, vp, vp, f32, i32, vp], i32),
        "ldpc_mixed_plan_serial": ([vp, P(i32), P(i32)], i32),
        "ldpc_decode_mixed": ([vp, i32, vp, P(_Params), vp, vp, vp, vp], i32),
        "ldpc_mixed_stats": ([vp, vp, vp, vp, i32, vp, vp, vp], i32),
        "ldpc_mixed_autotune": ([vp, i32, vp, P(_Params), vp, vp, i32, vp], i32),
        "ldpc_mixed_scatter": ([vp, i32, i32, vp, vp, vp], i32),
        "ldpc_mixed_graph_create": ([vp, i32, vp, vp, f32, i32, P(_Params), vp, vp, vp, vp, vp,
                                     P(vp)], i32),
        "ldpc_mixed_graph_launch": ([vp, vp], i32),
        "ldpc_mixed_graph_destroy": ([vp], None),
        "ldpc_quantize_i16": ([vp, vp, i64, f32, i32, vp], i32),
        "ldpc_encode_bitmap": ([vp, vp, vp, i64, vp], i32),
        "ldpc_decode_flooding_minsum": ([vp, vp, i64, P(_Params), vp, vp, vp, vp], i32),
        "ldpc_mixed_set_weights": ([vp, vp, vp], i32),
        "ldpc_decode_mixed_learned": ([vp, vp, i32, vp, vp, vp, vp], i32),
        "ldpc_mixed_frame_flags": ([vp, vp, vp, vp], i32),
        "ldpc_mixed_move_frames": ([vp, vp, vp, i32, vp, vp, vp], i32),
        "ldpc_mixed_paired_errors": ([vp, vp, vp, vp, vp, vp], i32),
        "ldpc_check_bounded_wait": ([vp, ctypes.c_uint32, vp], i32),
        "ldpc_test_set_grid_cap": ([i32], i32),
        "ldpc_debug_saturation_count": ([vp, vp, P(i64)], i32),
        "ldpc_last_error": ([], ctypes.c_char_p),
    }
    for name, (args, res) in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = res
    _lib = L
    return L


def _check(status: int):
    if status != 0:
        msg = load().ldpc_last_error().decode(errors="replace")
        raise LdpcError(status, msg)


def _torch():
    import torch
    return torch


def _stream(stream=None) -> int:
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


def _ptr(t) -> Optional[int]:
    return None if t is None else int(t.data_ptr())


def _bind_device(dev):
    torch = _torch()
    idx = torch.device(dev).index
    if idx is None:
        idx = torch.cuda.current_device()
    _check(load().ldpc_set_device(idx))
    return idx


class Code:
    """A QC-LDPC code from its base matrix (Section 1, eq. 2) on one GPU."""

    def __init__(self, hbm, z: int, device="cuda"):
        hbm = np.ascontiguousarray(hbm, dtype=np.int16)
        self.device_index = _bind_device(device)
        self.hbm = hbm
        self._h = ctypes.c_void_p()
        _check(load().ldpc_code_create(hbm.ctypes.data_as(ctypes.c_void_p), hbm.shape[0],
                                       hbm.shape[1], int(z), ctypes.byref(self._h)))
        vals = [ctypes.c_int() for _ in range(5)]
        _check(load().ldpc_code_info(self._h, *[ctypes.byref(v) for v in vals]))
        self.n, self.k, self.m, self.z, self.max_row_deg = [v.value for v in vals]
        self.nwords = (self.n + 31) // 32

    def __del__(self):
        h = getattr(self, "_h", None)
        if h and _lib is not None:
            _lib.ldpc_code_destroy(h)
            self._h = None

    @property
    def device(self):
        return _torch().device("cuda", self.device_index)

    def encode(self, info, out=None, stream=None):
        """eq. (8)-(15): uint8[F][K] -> uint8[F][N] on the GPU."""
        torch = _torch()
        F = info.shape[0]
        if out is None:
            out = torch.empty((F, self.n), dtype=torch.uint8, device=info.device)
        _check(load().ldpc_encode(self._h, _ptr(info), _ptr(out), F, _stream(stream)))
        return out

    def decode(self, llr, frames: Optional[int] = None, dtype: int = F32, max_iters: int = 10,
               alpha: float = 0.75, normalise: bool = True, early_stop: bool = False,
               want_post: bool = False, out=None, stream=None):
        """Layered min-sum (Section 4).  llr: float32[F][N] (F32), the packed
        int32/uint32 [ceil(F/4)][N] words of quantize_pack_i8 (I8X4), or
        int16[F][N] from quantize_i16 (I16W, Section 5 wrap-around).
        Returns (hard int32[F][ceil(N/32)], iters int32[F], post or None)."""
        torch = _torch()
        if frames is None:
            frames = 4 * llr.shape[0] if dtype == I8X4 else llr.shape[0]
        dev = llr.device
        if out is None:
            hard = torch.empty((frames, self.nwords), dtype=torch.int32, device=dev)
            iters = torch.empty((frames,), dtype=torch.int32, device=dev)
            post = None
            if want_post:
                post = torch.empty((frames, self.n),
                                   dtype={F32: torch.float32, I8X4: torch.int8,
                                          I16W: torch.int16}[dtype],
                                   device=dev)
        else:
            hard, iters, post = out
        p = _Params(int(max_iters), float(alpha), int(bool(normalise)), int(bool(early_stop)))
        _check(load().ldpc_decode_layered_minsum(self._h, int(dtype), _ptr(llr), int(frames),
                                                 ctypes.byref(p), _ptr(hard), _ptr(iters),
                                                 _ptr(post), _stream(stream)))
        return hard, iters, post

    def encode_bitmap(self, info_words, out=None, stream=None):
        """Alg. A1 bitmap encoder (Z % 32 == 0): uint32/int32[F][K/32] packed
        info -> [F][N/32] packed codeword."""
        torch = _torch()
        F = info_words.shape[0]
        if out is None:
            out = torch.empty((F, self.n // 32), dtype=torch.int32, device=info_words.device)
        _check(load().ldpc_encode_bitmap(self._h, _ptr(info_words), _ptr(out), int(F),
                                         _stream(stream)))
        return out

    def decode_flooding(self, llr, max_iters: int = 10, alpha: float = 0.75,
                        normalise: bool = True, early_stop: bool = False,
                        want_post: bool = False, stream=None):
        """Flooding min-sum (eq. 18-21), FP32."""
        torch = _torch()
        F = llr.shape[0]
        hard = torch.empty((F, self.nwords), dtype=torch.int32, device=llr.device)
        iters = torch.empty((F,), dtype=torch.int32, device=llr.device)
        post = (torch.empty((F, self.n), dtype=torch.float32, device=llr.device)
                if want_post else None)
        p = _Params(int(max_iters), float(alpha), int(bool(normalise)), int(bool(early_stop)))
        _check(load().ldpc_decode_flooding_minsum(self._h, _ptr(llr), int(F), ctypes.byref(p),
                                                  _ptr(hard), _ptr(iters), _ptr(post),
                                                  _stream(stream)))
        return hard, iters, post

    @property
    def nnz_blocks(self) -> int:
        """Nonzero blocks of H_bm: the number of learned weights per iteration."""
        return int((self.hbm >= 0).sum())

    def decode_learned(self, llr, weights, early_stop: bool = True, want_post: bool = False,
                       out=None, stream=None, max_iters: Optional[int] = None,
                       stop_iter=(0, 0), stop_frac=(0.0, 0.0)):
        """Learned normalised min-sum: weights float32[T][nnz_blocks] on the GPU.
        max_iters (default T) may exceed T: later iterations repeat the last
        weight row; (stop_iter[j], stop_frac[j]) are give-up checkpoints
        (ldpc_learned_params)."""
        torch = _torch()
        F, T = llr.shape[0], weights.shape[0]
        if out is None:
            hard = torch.empty((F, self.nwords), dtype=torch.int32, device=llr.device)
            iters = torch.empty((F,), dtype=torch.int32, device=llr.device)
            post = (torch.empty((F, self.n), dtype=torch.float32, device=llr.device)
                    if want_post else None)
        else:
            hard, iters, post = out
        if max_iters is None and not any(stop_iter):
            _check(load().ldpc_decode_learned_minsum(self._h, _ptr(llr), int(F), _ptr(weights),
                                                     int(T), int(bool(early_stop)), _ptr(hard),
                                                     _ptr(iters), _ptr(post), _stream(stream)))
        else:
            lp = _learned_params(max_iters, early_stop, stop_iter, stop_frac)
            _check(load().ldpc_decode_learned_minsum_ex(self._h, _ptr(llr), int(F),
                                                        _ptr(weights), int(T), ctypes.byref(lp),
                                                        _ptr(hard), _ptr(iters), _ptr(post),
                                                        _stream(stream)))
        return hard, iters, post

    def learned_workspace_bytes(self, frames: int) -> int:
        return int(load().ldpc_learned_fallback_workspace_bytes(self._h, int(frames)))

    def decode_learned_fallback(self, llr, weights, fallback_iters: int = 20,
                                quant_scale: float = 4.0, quant_clip: int = 63, workspace=None,
                                out=None, stream=None):
        """Learned decoding, then int8 plain min-sum on the frames that still
        fail a parity check.  Returns (hard, iters, number of fallback frames)."""
        torch = _torch()
        F, T = llr.shape[0], weights.shape[0]
        if out is None:
            hard = torch.empty((F, self.nwords), dtype=torch.int32, device=llr.device)
            iters = torch.empty((F,), dtype=torch.int32, device=llr.device)
        else:
            hard, iters = out
        if workspace is None:
            workspace = torch.empty(self.learned_workspace_bytes(F), dtype=torch.uint8,
                                    device=llr.device)
        fb = _Params(int(fallback_iters), 0.75, 1, 1)
        cnt = ctypes.c_int64(0)
        _check(load().ldpc_decode_learned_fallback(
            self._h, _ptr(llr), int(F), _ptr(weights), int(T), ctypes.byref(fb),
            float(quant_scale), int(quant_clip), _ptr(hard), _ptr(iters), ctypes.byref(cnt),
            _ptr(workspace), int(workspace.numel()), _stream(stream)))
        return hard, iters, int(cnt.value)

    def train_forward(self, llr, bits, weights, loss_scale: float = 1.0, out=None,
                      stream=None):
        """Training forward (T = weights.shape[0] iterations, no early stop).
        Returns (post float32[T][F][N], rows int32[T-1][F][M][4], loss
        float32[F], loss_sum float32[1] = loss_scale * sum(loss))."""
        torch = _torch()
        F, T = llr.shape[0], weights.shape[0]
        dev = llr.device
        if out is None:
            post = torch.empty((T, F, self.n), dtype=torch.float32, device=dev)
            rows = torch.empty((max(T - 1, 0), F, self.m, 4), dtype=torch.int32, device=dev)
            loss = torch.empty((F,), dtype=torch.float32, device=dev)
            loss_sum = torch.empty((1,), dtype=torch.float32, device=dev)
        else:
            post, rows, loss, loss_sum = out
        _check(load().ldpc_learned_train_forward(
            self._h, _ptr(llr), _ptr(bits), int(F), _ptr(weights), int(T), _ptr(post),
            _ptr(rows) if rows.numel() else None, _ptr(loss), float(loss_scale),
            _ptr(loss_sum), _stream(stream)))
        return post, rows, loss, loss_sum

    def train_workspace_bytes(self, frames: int, T: int) -> int:
        return int(load().ldpc_learned_train_workspace_bytes(self._h, int(frames), int(T)))

    def train_backward(self, llr, bits, weights, post, rows, loss_scale: float = 1.0,
                       want_llr_grad: bool = False, workspace=None, out=None, stream=None):
        """Gradients of loss_scale * sum(loss) from the training forward's
        checkpoints: (d/d weights float32[T][nnz_blocks], d/d llr or None)."""
        torch = _torch()
        F, T = llr.shape[0], weights.shape[0]
        dev = llr.device
        if out is None:
            gw = torch.empty((T, self.nnz_blocks), dtype=torch.float32, device=dev)
            gx = (torch.empty((F, self.n), dtype=torch.float32, device=dev)
                  if want_llr_grad else None)
        else:
            gw, gx = out
        if workspace is None:
            workspace = torch.empty(max(self.train_workspace_bytes(F, T), 1), dtype=torch.uint8,
                                    device=dev)
        _check(load().ldpc_learned_train_backward(
            self._h, _ptr(llr), _ptr(bits), int(F), _ptr(weights), int(T), _ptr(post),
            _ptr(rows) if rows.numel() else None, float(loss_scale), _ptr(gw), _ptr(gx),
            _ptr(workspace), int(workspace.numel()), _stream(stream)))
        return gw, gx

    def frame_stats(self, info, hard, iters, max_iters: int, out=None, stream=None):
        """int64[4 + max_iters + 1]: bit errors, frame errors, undetected
        errors, iteration sum, iteration histogram."""
        torch = _torch()
        if out is None:
            out = torch.empty((5 + max_iters,), dtype=torch.int64, device=hard.device)
        _check(load().ldpc_frame_stats(self._h, _ptr(info), _ptr(hard), _ptr(iters),
                                       int(hard.shape[0]), int(max_iters), _ptr(out),
                                       _stream(stream)))
        return out

    def paired_frame_errors(self, info, hard_a, hard_b, out=None, stream=None):
        """int64[4]: frames both right, only B wrong, only A wrong, both wrong."""
        torch = _torch()
        if out is None:
            out = torch.empty((4,), dtype=torch.int64, device=hard_a.device)
        _check(load().ldpc_paired_frame_errors(self._h, _ptr(info), _ptr(hard_a), _ptr(hard_b),
                                               int(hard_a.shape[0]), _ptr(out),
                                               _stream(stream)))
        return out

    def host_workspace_bytes(self, dtype: int, chunk_frames: int) -> int:
        return int(load().ldpc_decode_host_workspace_bytes(self._h, int(dtype),
                                                           int(chunk_frames)))

    def decode_host(self, h_llr, frames: int, dtype: int, h_hard, h_iters, workspace,
                    chunk_frames: int, max_iters: int = 20, alpha: float = 0.75,
                    normalise: bool = True, early_stop: bool = True, stream=None):
        """End-to-end decode of host (pinned) buffers through the library's
        copy/decode pipeline; outputs land in h_hard / h_iters."""
        p = _Params(int(max_iters), float(alpha), int(bool(normalise)), int(bool(early_stop)))
        _check(load().ldpc_decode_host(self._h, int(dtype), _ptr(h_llr), int(frames),
                                       ctypes.byref(p), _ptr(h_hard), _ptr(h_iters),
                                       _ptr(workspace), int(workspace.numel()),
                                       int(chunk_frames), _stream(stream)))

    def saturation_count(self, stream=None) -> int:
        """Debug builds: int8 clamps taken since the last call (waits for the
        stream); raises LdpcError in release builds."""
        v = ctypes.c_int64(0)
        _check(load().ldpc_debug_saturation_count(self._h, _stream(stream), ctypes.byref(v)))
        return int(v.value)

    def check_bounded_wait(self, polls: int = 4096, stream=None):
        """Runs the failure-path check; the next sync() raises the timeout."""
        _check(load().ldpc_check_bounded_wait(self._h, int(polls), _stream(stream)))

    def sync(self, timeout_s: float = 60.0, stream=None):
        _check(load().ldpc_sync(self._h, _stream(stream), float(timeout_s)))


class CodeSet:
    """Codes decoded together in mixed batches (the handles are kept alive)."""

    def __init__(self, codes):
        self.codes = list(codes)
        arr = (ctypes.c_void_p * len(self.codes))(*[c._h.value for c in self.codes])
        self._h = ctypes.c_void_p()
        _check(load().ldpc_codeset_create(arr, len(self.codes), ctypes.byref(self._h)))

    def __del__(self):
        h = getattr(self, "_h", None)
        if h and _lib is not None:
            _lib.ldpc_codeset_destroy(h)
            self._h = None

    def __len__(self):
        return len(self.codes)


class MixedPlan:
    """Layout and launch plan of a batch whose frame f uses code
    code_of_frame[f] of the set."""

    def __init__(self, codeset: CodeSet, code_of_frame):
        cof = np.ascontiguousarray(code_of_frame, dtype=np.int32)
        self.codeset = codeset
        self.code_of_frame = cof
        self.frames = int(cof.size)
        self._h = ctypes.c_void_p()
        _check(load().ldpc_mixed_plan_create(codeset._h, cof.ctypes.data_as(ctypes.c_void_p),
                                             self.frames, ctypes.byref(self._h)))
        v = [ctypes.c_int64() for _ in range(4)]
        ng = ctypes.c_int()
        _check(load().ldpc_mixed_plan_sizes(self._h, *[ctypes.byref(x) for x in v],
                                            ctypes.byref(ng)))
        self.llr_elems, self.info_elems, self.hard_words, self.q_words = [x.value for x in v]
        self.n_groups = ng.value
        self.llr_off = np.zeros(self.frames + 1, dtype=np.int64)
        self.info_off = np.zeros(self.frames + 1, dtype=np.int64)
        self.hard_off = np.zeros(self.frames + 1, dtype=np.int64)
        _check(load().ldpc_mixed_plan_offsets(self._h, self.llr_off.ctypes.data_as(ctypes.c_void_p),
                                              self.info_off.ctypes.data_as(ctypes.c_void_p),
                                              self.hard_off.ctypes.data_as(ctypes.c_void_p)))

    def __del__(self):
        h = getattr(self, "_h", None)
        if h and _lib is not None:
            _lib.ldpc_mixed_plan_destroy(h)
            self._h = None

    def groups(self):
        out = []
        for g in range(self.n_groups):
            v = [ctypes.c_int() for _ in range(8)]
            _check(load().ldpc_mixed_group_info(self._h, g, *[ctypes.byref(x) for x in v]))
            keys = ("slot_class", "codes", "smem_f32", "smem_i8", "chunk_f32", "chunk_i8",
                    "blocks_per_sm_f32", "blocks_per_sm_i8")
            d = dict(zip(keys, [x.value for x in v]))
            t = _GroupLaunch()
            _check(load().ldpc_mixed_group_launch(self._h, g, F32, None, ctypes.byref(t)))
            d["warps_per_frame_f32"] = t.warps_per_frame
            d["frames_per_block_f32"] = t.frames_per_block
            out.append(d)
        return out

    def group_launch(self, group: int, dtype: int = F32, frames_per_item=None,
                     blocks_per_sm=None, warps_per_frame=None, frames_per_block=None):
        """The launch settings of one group (ldpc_group_launch as a dict);
        any argument given replaces that setting first."""
        cur = _GroupLaunch()
        _check(load().ldpc_mixed_group_launch(self._h, int(group), int(dtype), None,
                                              ctypes.byref(cur)))
        new = {"frames_per_item": frames_per_item, "blocks_per_sm": blocks_per_sm,
               "warps_per_frame": warps_per_frame, "frames_per_block": frames_per_block}
        if any(v is not None for v in new.values()):
            for k, v in new.items():
                if v is not None:
                    setattr(cur, k, int(v))
            _check(load().ldpc_mixed_group_launch(self._h, int(group), int(dtype),
                                                  ctypes.byref(cur), ctypes.byref(cur)))
        return {k: getattr(cur, k) for k, _ in _GroupLaunch._fields_}

    def serial(self):
        a, b = ctypes.c_int(), ctypes.c_int()
        _check(load().ldpc_mixed_plan_serial(self._h, ctypes.byref(a), ctypes.byref(b)))
        return {"fp32": bool(a.value), "int8": bool(b.value)}

    def _dev(self):
        return self.codeset.codes[0].device

    def empty_outputs(self):
        torch = _torch()
        dev = self._dev()
        return (torch.empty((self.hard_words,), dtype=torch.int32, device=dev),
                torch.empty((self.frames,), dtype=torch.int32, device=dev))

    def quantize(self, llr, scale: float = 4.0, clip: int = 63, out=None, stream=None):
        torch = _torch()
        if out is None:
            out = torch.empty((max(self.q_words, 1),), dtype=torch.int32, device=llr.device)
        _check(load().ldpc_mixed_quantize(self._h, _ptr(llr), _ptr(out), float(scale), int(clip),
                                          _stream(stream)))
        return out

    def decode(self, d_in, dtype: int = F32, max_iters: int = 20, alpha: float = 0.75,
               normalise: bool = True, early_stop: bool = True, want_post: bool = False,
               out=None, stream=None):
        """Returns (hard int32[hard_words], iters int32[frames], post or None)."""
        torch = _torch()
        if out is None:
            hard, iters = self.empty_outputs()
            post = None
            if want_post:
                post = torch.empty((self.llr_elems,),
                                   dtype=torch.float32 if dtype == F32 else torch.int8,
                                   device=d_in.device)
        else:
            hard, iters, post = out
        p = _Params(int(max_iters), float(alpha), int(bool(normalise)), int(bool(early_stop)))
        _check(load().ldpc_decode_mixed(self._h, int(dtype), _ptr(d_in), ctypes.byref(p),
                                        _ptr(hard), _ptr(iters), _ptr(post), _stream(stream)))
        return hard, iters, post

    def stats(self, info, hard, iters, max_iters: int, per_code: bool = True, stream=None):
        torch = _torch()
        cnt = torch.empty((5 + max_iters,), dtype=torch.int64, device=hard.device)
        fe = (torch.empty((len(self.codeset),), dtype=torch.int64, device=hard.device)
              if per_code else None)
        _check(load().ldpc_mixed_stats(self._h, _ptr(info), _ptr(hard), _ptr(iters),
                                       int(max_iters), _ptr(cnt), _ptr(fe), _stream(stream)))
        return cnt, fe

    def autotune(self, d_in, dtype: int = F32, max_iters: int = 20, alpha: float = 0.75,
                 normalise: bool = True, early_stop: bool = True, reps: int = 3, out=None,
                 stream=None):
        hard, iters = out if out is not None else self.empty_outputs()
        p = _Params(int(max_iters), float(alpha), int(bool(normalise)), int(bool(early_stop)))
        _check(load().ldpc_mixed_autotune(self._h, int(dtype), _ptr(d_in), ctypes.byref(p),
                                          _ptr(hard), _ptr(iters), int(reps), _stream(stream)))
        return self.groups()

    def set_weights(self, weights):
        """weights: per code of the set, a float32 [T][nnz_blocks] device tensor
        (or None for codes without frames)."""
        n = len(self.codeset)
        ptrs = (ctypes.c_void_p * n)(*[(_ptr(w) if w is not None else None) for w in weights])
        T = np.array([(w.shape[0] if w is not None else 0) for w in weights], dtype=np.int32)
        self._weights = list(weights)
        self.T = T
        _check(load().ldpc_mixed_set_weights(self._h, ptrs, T.ctypes.data_as(ctypes.c_void_p)))

    def decode_learned(self, llr, early_stop: bool = True, want_post: bool = False, out=None,
                       stream=None, max_iters: int = 0, stop_iter=(0, 0),
                       stop_frac=(0.0, 0.0)):
        """Learned decoding of every frame with its code's weights; max_iters
        0 runs T_c iterations per code, more repeat each table's last row;
        (stop_iter[j], stop_frac[j]) are give-up checkpoints."""
        torch = _torch()
        if out is None:
            hard, iters = self.empty_outputs()
            post = (torch.empty((self.llr_elems,), dtype=torch.float32, device=llr.device)
                    if want_post else None)
        else:
            hard, iters, post = out
        if not max_iters and not any(stop_iter):
            _check(load().ldpc_decode_mixed_learned(self._h, _ptr(llr), int(bool(early_stop)),
                                                    _ptr(hard), _ptr(iters), _ptr(post),
                                                    _stream(stream)))
        else:
            lp = _learned_params(max_iters, early_stop, stop_iter, stop_frac)
            _check(load().ldpc_decode_mixed_learned_ex(self._h, _ptr(llr), ctypes.byref(lp),
                                                       _ptr(hard), _ptr(iters), _ptr(post),
                                                       _stream(stream)))
        return hard, iters, post

    def autotune_learned(self, llr, max_iters: int = 0, stop_iter=(0, 0), stop_frac=(0.0, 0.0),
                         reps: int = 3, out=None, stream=None):
        """Tune the work items, residency caps and concurrency the learned
        (and FP32) launches share, timing the learned decoder."""
        hard, iters = out if out is not None else self.empty_outputs()
        lp = _learned_params(max_iters, True, stop_iter, stop_frac)
        _check(load().ldpc_mixed_autotune_learned(self._h, _ptr(llr), ctypes.byref(lp),
                                                  _ptr(hard), _ptr(iters), int(reps),
                                                  _stream(stream)))
        return self.groups()

    def frame_flags(self, hard, out=None, stream=None):
        torch = _torch()
        if out is None:
            out = torch.empty((self.frames,), dtype=torch.uint8, device=hard.device)
        _check(load().ldpc_mixed_frame_flags(self._h, _ptr(hard), _ptr(out), _stream(stream)))
        return out

    def move_frames(self, sub, d_index, what: int, a, b, stream=None):
        """Frame s of plan `sub` is frame d_index[s] of this plan (see
        ldpc_mixed_move_frames for `what`)."""
        _check(load().ldpc_mixed_move_frames(self._h, sub._h, _ptr(d_index), int(what), _ptr(a),
                                             _ptr(b), _stream(stream)))

    def paired_errors(self, info, hard_a, hard_b, stream=None):
        torch = _torch()
        out = torch.empty((4,), dtype=torch.int64, device=hard_a.device)
        _check(load().ldpc_mixed_paired_errors(self._h, _ptr(info), _ptr(hard_a), _ptr(hard_b),
                                               _ptr(out), _stream(stream)))
        return out

    def scatter(self, code_index: int, what: int, src, dst, stream=None):
        _check(load().ldpc_mixed_scatter(self._h, int(code_index), int(what), _ptr(src),
                                         _ptr(dst), _stream(stream)))

    def graph(self, dtype: int, llr, q, hard, iters, info=None, counters=None, code_fe=None,
              max_iters: int = 20, alpha: float = 0.75, normalise: bool = True,
              early_stop: bool = True, quant_scale: float = 4.0, quant_clip: int = 63):
        return MixedGraph(self, dtype, llr, q, hard, iters, info, counters, code_fe,
                          _Params(int(max_iters), float(alpha), int(bool(normalise)),
                                  int(bool(early_stop))), quant_scale, quant_clip)


class MixedGraph:
    """CUDA graph of one mixed step (quantise, decode launches, stats)."""

    def __init__(self, plan, dtype, llr, q, hard, iters, info, counters, code_fe, params,
                 quant_scale, quant_clip):
        self.plan = plan
        self._keep = (llr, q, hard, iters, info, counters, code_fe)
        self._h = ctypes.c_void_p()
        _check(load().ldpc_mixed_graph_create(
            plan._h, int(dtype), _ptr(llr), _ptr(q), float(quant_scale), int(quant_clip),
            ctypes.byref(params), _ptr(hard), _ptr(iters), _ptr(info), _ptr(counters),
            _ptr(code_fe), ctypes.byref(self._h)))

    def launch(self, stream=None):
        _check(load().ldpc_mixed_graph_launch(self._h, _stream(stream)))

    def __del__(self):
        h = getattr(self, "_h", None)
        if h and _lib is not None:
            _lib.ldpc_mixed_graph_destroy(h)
            self._h = None


def gen_info(seed: int, frame0: int, frames: int, k: int, device="cuda", out=None,
             stream=None):
    """Philox info bits uint8[frames][k] on the GPU."""
    torch = _torch()
    _bind_device(device)
    if out is None:
        out = torch.empty((frames, k), dtype=torch.uint8, device=device)
    _check(load().ldpc_gen_info(int(seed), int(frame0), int(frames), int(k), _ptr(out),
                                _stream(stream)))
    return out


def awgn_llr(cw, frame0: int, seed: int, sigma: float, llr_scale: Optional[float] = None,
             out=None, stream=None):
    """eq. (16)-(17) channel on the GPU; llr_scale defaults to the float32 value
    of 2 / sigma^2."""
    torch = _torch()
    F, n = cw.shape
    sig = np.float32(sigma)
    if llr_scale is None:
        llr_scale = float(np.float32(2.0 / (float(sig) ** 2)))
    if out is None:
        out = torch.empty((F, n), dtype=torch.float32, device=cw.device)
    _check(load().ldpc_awgn_llr(_ptr(cw), int(frame0), int(F), int(n), int(seed), float(sig),
                                float(llr_scale), _ptr(out), _stream(stream)))
    return out


def quantize_i16(llr, scale: float = 16.0, qb: int = 10, out=None, stream=None):
    """Section 5 channel: float32[...] -> int16 rint(clamp(scale * llr, +-(2^qb - 1)))."""
    torch = _torch()
    if out is None:
        out = torch.empty(llr.shape, dtype=torch.int16, device=llr.device)
    _check(load().ldpc_quantize_i16(_ptr(llr), _ptr(out), int(llr.numel()), float(scale),
                                    int(qb), _stream(stream)))
    return out


def quantize_pack_i8(llr, scale: float = 4.0, clip: int = 63, out=None, stream=None):
    """float32[F][N] -> int32[ceil(F/4)][N] words of four int8 frames."""
    torch = _torch()
    F, n = llr.shape
    if out is None:
        out = torch.empty(((F + 3) // 4, n), dtype=torch.int32, device=llr.device)
    _check(load().ldpc_quantize_pack_i8(_ptr(llr), _ptr(out), int(F), int(n), float(scale),
                                        int(clip), _stream(stream)))
    return out


def awgn_llr_frames(cw, frame0: int, seed: int, sigma, out=None, stream=None):
    """eq. (16)-(17) with a noise level per frame: sigma float32[F] on the GPU."""
    torch = _torch()
    F, n = cw.shape
    if out is None:
        out = torch.empty((F, n), dtype=torch.float32, device=cw.device)
    _check(load().ldpc_awgn_llr_frames(_ptr(cw), int(frame0), int(F), int(n), int(seed),
                                       _ptr(sigma), _ptr(out), _stream(stream)))
    return out


def snr_sigma(seed: int, frame0: int, frames: int, ebn0_lo_db: float, ebn0_hi_db: float,
              rate: float, device="cuda", out=None, stream=None):
    """Per-frame noise sigma float32[frames] for Eb/N0 uniform in [lo, hi) dB."""
    torch = _torch()
    _bind_device(device)
    if out is None:
        out = torch.empty((frames,), dtype=torch.float32, device=device)
    _check(load().ldpc_snr_sigma(int(seed), int(frame0), int(frames), float(ebn0_lo_db),
                                 float(ebn0_hi_db), float(rate), _ptr(out), _stream(stream)))
    return out


def set_grid_cap(blocks: int) -> None:
    """Testing aid: cap the single-code decoders' persistent grids at
    `blocks` blocks (0 removes the cap) for every later launch."""
    _check(load().ldpc_test_set_grid_cap(int(blocks)))


def adam_step(param, grad, m, v, step: int, lr: float = 1e-3, beta1: float = 0.9,
              beta2: float = 0.999, eps: float = 1e-8, stream=None):
    """One in-place Adam update of float32 device tensors."""
    _check(load().ldpc_adam_step(_ptr(param), _ptr(grad), _ptr(m), _ptr(v),
                                 int(param.numel()), int(step), float(lr), float(beta1),
                                 float(beta2), float(eps), _stream(stream)))
