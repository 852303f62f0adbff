"""Python handle on the CPU oracle (oracle/ldpc_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by tests/, by the smoke check and by the
CPU-baseline leg of the benchmark.  The CUDA library never uses it.

Each wrapper takes and returns numpy arrays; the C code is built on first
use (gcc, -O2 -ffp-contract=off) next to this file.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading
from typing import Optional, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ldpc_oracle.c")
_LIB_PATH = os.path.join(_HERE, "libldpc_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle into a shared library; returns its path."""
    stale = (not os.path.exists(_LIB_PATH)
             or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC)
             or os.path.getmtime(_LIB_PATH) < os.path.getmtime(
                 os.path.join(_HERE, "ldpc_oracle.h")))
    if force or stale:
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-std=c99", "-O2", "-ffp-contract=off", "-fno-fast-math",
               "-Wall", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True, cwd=_HERE)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Params(ctypes.Structure):
    _fields_ = [("max_iters", ctypes.c_int), ("alpha", ctypes.c_float),
                ("normalise", ctypes.c_int), ("early_stop", ctypes.c_int)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB_PATH)
            vp, i32, i64, u64, f32 = (ctypes.c_void_p, ctypes.c_int,
                                      ctypes.c_int64, ctypes.c_uint64,
                                      ctypes.c_float)
            L.ldpc_ref_code_create.argtypes = [vp, i32, i32, i32, i32,
                                               ctypes.POINTER(vp)]
            L.ldpc_ref_code_destroy.argtypes = [vp]
            L.ldpc_ref_code_destroy.restype = None
            L.ldpc_ref_code_info.argtypes = [vp] + [ctypes.POINTER(i32)] * 7
            L.ldpc_ref_row_vars.argtypes = [vp, i32, vp, i32]
            L.ldpc_ref_encode.argtypes = [vp, vp, vp, i64]
            L.ldpc_ref_syndrome_weight.argtypes = [vp, vp]
            L.ldpc_ref_philox4x32_10.argtypes = [vp, vp, vp]
            L.ldpc_ref_philox4x32_10.restype = None
            L.ldpc_ref_gen_info.argtypes = [u64, i64, i64, i32, vp]
            L.ldpc_ref_box_muller.argtypes = [ctypes.c_uint32, ctypes.c_uint32,
                                              ctypes.POINTER(f32),
                                              ctypes.POINTER(f32)]
            L.ldpc_ref_box_muller.restype = None
            L.ldpc_ref_lnf.argtypes = [f32]
            L.ldpc_ref_lnf.restype = f32
            L.ldpc_ref_sincos_turn.argtypes = [ctypes.c_uint32,
                                               ctypes.POINTER(f32),
                                               ctypes.POINTER(f32)]
            L.ldpc_ref_sincos_turn.restype = None
            L.ldpc_ref_awgn_llr.argtypes = [vp, i64, i64, i32, u64, f32, f32, vp]
            L.ldpc_ref_quantize_i8.argtypes = [vp, vp, i64, f32, i32]
            L.ldpc_ref_quantize_i16.argtypes = [vp, vp, i64, f32, i32]
            L.ldpc_ref_decode_layered_i16w.argtypes = [vp, vp, i64, ctypes.POINTER(_Params),
                                                       vp, vp, vp, ctypes.POINTER(i64)]
            L.ldpc_ref_encode_bitmap.argtypes = [vp, vp, vp, i64]
            L.ldpc_ref_rotate_block.argtypes = [vp, i32, i32, vp]
            L.ldpc_ref_rotate_block.restype = None
            for name in ("ldpc_ref_decode_layered_f32",
                         "ldpc_ref_decode_flooding_f32"):
                getattr(L, name).argtypes = [vp, vp, i64,
                                             ctypes.POINTER(_Params), vp, vp, vp]
            L.ldpc_ref_decode_layered_weighted_f32.argtypes = [vp, vp, i64, vp, i32, i32,
                                                               vp, vp, vp]
            L.ldpc_ref_decode_learned_f32.argtypes = [vp, vp, i64, vp, i32, i32, i32, vp, vp,
                                                      vp, vp, vp]
            L.ldpc_ref_decode_layered_i8.argtypes = [
                vp, vp, i64, ctypes.POINTER(_Params), vp, vp, vp,
                ctypes.POINTER(i64)]
            _lib = L
    return _lib


def _ptr(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


class OracleError(RuntimeError):
    pass


def _check(status: int, what: str):
    if status != 0:
        raise OracleError(f"{what} failed with status {status}")


class RefCode:
    """Oracle view of a code: the explicit sparse H built from H_bm."""

    def __init__(self, hbm: np.ndarray, z: int, require_encodable: bool = True):
        hbm = np.ascontiguousarray(hbm, dtype=np.int16)
        self.hbm = hbm
        self._h = ctypes.c_void_p()
        st = lib().ldpc_ref_code_create(_ptr(hbm), hbm.shape[0], hbm.shape[1],
                                        int(z), int(require_encodable),
                                        ctypes.byref(self._h))
        _check(st, "ldpc_ref_code_create")
        vals = [ctypes.c_int() for _ in range(7)]
        lib().ldpc_ref_code_info(self._h, *[ctypes.byref(v) for v in vals])
        (self.n, self.k, self.m, self.z, self.max_row_deg, self.y,
         self.encodable) = [v.value for v in vals]

    def __del__(self):
        h = getattr(self, "_h", None)
        if h and _lib is not None:
            _lib.ldpc_ref_code_destroy(h)
            self._h = None

    @property
    def nwords(self) -> int:
        return (self.n + 31) // 32

    def row_vars(self, row: int) -> np.ndarray:
        buf = np.zeros(64, dtype=np.int32)
        d = lib().ldpc_ref_row_vars(self._h, row, _ptr(buf), 64)
        return buf[:d].copy()

    def encode(self, info: np.ndarray) -> np.ndarray:
        info = np.ascontiguousarray(info, dtype=np.uint8).reshape(-1, self.k)
        out = np.zeros((info.shape[0], self.n), dtype=np.uint8)
        _check(lib().ldpc_ref_encode(self._h, _ptr(info), _ptr(out),
                                     info.shape[0]), "ldpc_ref_encode")
        return out

    def syndrome_weight(self, bits: np.ndarray) -> int:
        bits = np.ascontiguousarray(bits, dtype=np.uint8).reshape(self.n)
        return int(lib().ldpc_ref_syndrome_weight(self._h, _ptr(bits)))

    def _decode(self, fn, llr, dtype, max_iters, alpha, normalise, early_stop,
                want_post, post_dtype):
        llr = np.ascontiguousarray(llr, dtype=dtype).reshape(-1, self.n)
        F = llr.shape[0]
        hard = np.zeros((F, self.nwords), dtype=np.uint32)
        iters = np.zeros(F, dtype=np.int32)
        post = np.zeros((F, self.n), dtype=post_dtype) if want_post else None
        p = _Params(int(max_iters), float(alpha), int(normalise), int(early_stop))
        return llr, F, hard, iters, post, p

    def decode_layered_f32(self, llr, max_iters=10, alpha=0.75, normalise=True,
                           early_stop=False, want_post=True):
        llr, F, hard, iters, post, p = self._decode(
            None, llr, np.float32, max_iters, alpha, normalise, early_stop,
            want_post, np.float32)
        _check(lib().ldpc_ref_decode_layered_f32(
            self._h, _ptr(llr), F, ctypes.byref(p), _ptr(hard), _ptr(iters),
            _ptr(post)), "ldpc_ref_decode_layered_f32")
        return hard, iters, post

    @property
    def nnz_blocks(self) -> int:
        return int((self.hbm >= 0).sum())

    def decode_layered_weighted_f32(self, llr, weights, T=None, early_stop=True,
                                    want_post=True):
        """Learned normalised min-sum: weights f32[T][nnz(H_bm)]."""
        w = np.ascontiguousarray(weights, dtype=np.float32)
        T = w.shape[0] if T is None else int(T)
        assert w.size >= T * self.nnz_blocks
        llr, F, hard, iters, post, _ = self._decode(
            None, llr, np.float32, T, 1.0, False, early_stop, want_post, np.float32)
        _check(lib().ldpc_ref_decode_layered_weighted_f32(
            self._h, _ptr(llr), F, _ptr(w), T, int(early_stop), _ptr(hard), _ptr(iters),
            _ptr(post)), "ldpc_ref_decode_layered_weighted_f32")
        return hard, iters, post

    def decode_learned_f32(self, llr, weights, max_iters=None, early_stop=True,
                           stop_iter=(0, 0), stop_frac=(0.0, 0.0), want_post=True):
        """Learned normalised min-sum run for up to max_iters iterations
        (rows past the table's T repeat its last row), with give-up
        checkpoints (stop_iter[j], stop_frac[j]); see ldpc_oracle.h."""
        w = np.ascontiguousarray(weights, dtype=np.float32)
        T = w.shape[0]
        max_iters = T if max_iters is None else int(max_iters)
        si = np.ascontiguousarray(stop_iter, dtype=np.int32)
        sf = np.ascontiguousarray(stop_frac, dtype=np.float32)
        llr, F, hard, iters, post, _ = self._decode(
            None, llr, np.float32, max_iters, 1.0, False, early_stop, want_post, np.float32)
        _check(lib().ldpc_ref_decode_learned_f32(
            self._h, _ptr(llr), F, _ptr(w), T, max_iters, int(early_stop), _ptr(si), _ptr(sf),
            _ptr(hard), _ptr(iters), _ptr(post)), "ldpc_ref_decode_learned_f32")
        return hard, iters, post

    def decode_flooding_f32(self, llr, max_iters=10, alpha=0.75, normalise=True,
                            early_stop=False, want_post=True):
        llr, F, hard, iters, post, p = self._decode(
            None, llr, np.float32, max_iters, alpha, normalise, early_stop,
            want_post, np.float32)
        _check(lib().ldpc_ref_decode_flooding_f32(
            self._h, _ptr(llr), F, ctypes.byref(p), _ptr(hard), _ptr(iters),
            _ptr(post)), "ldpc_ref_decode_flooding_f32")
        return hard, iters, post

    def decode_layered_i16w(self, llr_q, max_iters=10, normalise=False,
                            early_stop=False, want_post=True):
        """Section 5 int16 wrap-around decoder: (hard, iters, post, wrap events)."""
        llr, F, hard, iters, post, p = self._decode(
            None, llr_q, np.int16, max_iters, 0.75, normalise, early_stop,
            want_post, np.int16)
        ev = ctypes.c_int64(0)
        _check(lib().ldpc_ref_decode_layered_i16w(
            self._h, _ptr(llr), F, ctypes.byref(p), _ptr(hard), _ptr(iters),
            _ptr(post), ctypes.byref(ev)), "ldpc_ref_decode_layered_i16w")
        return hard, iters, post, int(ev.value)

    def encode_bitmap(self, info_words: np.ndarray) -> np.ndarray:
        """Alg. A1 bitmap encoder: u32[F][K/32] -> u32[F][N/32] (Z % 32 == 0)."""
        w = np.ascontiguousarray(info_words, dtype=np.uint32).reshape(-1, self.k // 32)
        out = np.zeros((w.shape[0], self.n // 32), dtype=np.uint32)
        _check(lib().ldpc_ref_encode_bitmap(self._h, _ptr(w), _ptr(out), w.shape[0]),
               "ldpc_ref_encode_bitmap")
        return out

    def decode_layered_i8(self, llr_q, max_iters=10, normalise=True,
                          early_stop=False, want_post=True
                          ) -> Tuple[np.ndarray, np.ndarray, np.ndarray, int]:
        llr, F, hard, iters, post, p = self._decode(
            None, llr_q, np.int8, max_iters, 0.75, normalise, early_stop,
            want_post, np.int8)
        ev = ctypes.c_int64(0)
        _check(lib().ldpc_ref_decode_layered_i8(
            self._h, _ptr(llr), F, ctypes.byref(p), _ptr(hard), _ptr(iters),
            _ptr(post), ctypes.byref(ev)), "ldpc_ref_decode_layered_i8")
        return hard, iters, post, int(ev.value)


def quantize_i16(llr: np.ndarray, scale: float = 16.0, qb: int = 10) -> np.ndarray:
    """Section 5 channel: rint(clamp(scale * llr, +-(2^qb - 1))) as int16."""
    x = np.ascontiguousarray(llr, dtype=np.float32)
    out = np.zeros(x.shape, dtype=np.int16)
    _check(lib().ldpc_ref_quantize_i16(_ptr(x), _ptr(out), x.size, float(scale), int(qb)),
           "ldpc_ref_quantize_i16")
    return out


def rotate_block(words: np.ndarray, s: int) -> np.ndarray:
    """P_s on one packed block (Alg. A1 split)."""
    w = np.ascontiguousarray(words, dtype=np.uint32)
    out = np.zeros_like(w)
    lib().ldpc_ref_rotate_block(_ptr(w), int(w.size), int(s), _ptr(out))
    return out


def philox4x32_10(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().ldpc_ref_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def gen_info(seed: int, frame0: int, frames: int, k: int) -> np.ndarray:
    out = np.zeros((frames, k), dtype=np.uint8)
    _check(lib().ldpc_ref_gen_info(seed, frame0, frames, k, _ptr(out)),
           "ldpc_ref_gen_info")
    return out


def lnf(u: float) -> float:
    return float(lib().ldpc_ref_lnf(u))


def sincos_turn(k24: int) -> Tuple[float, float]:
    s, c = ctypes.c_float(), ctypes.c_float()
    lib().ldpc_ref_sincos_turn(k24, ctypes.byref(s), ctypes.byref(c))
    return s.value, c.value


def box_muller(w0: int, w1: int) -> Tuple[float, float]:
    a, b = ctypes.c_float(), ctypes.c_float()
    lib().ldpc_ref_box_muller(w0, w1, ctypes.byref(a), ctypes.byref(b))
    return a.value, b.value


def awgn_llr(cw: np.ndarray, frame0: int, seed: int, sigma: float,
             llr_scale: Optional[float] = None) -> np.ndarray:
    """eq. (16)-(17) with the Philox noise stream; llr_scale defaults to the
    float32 value of 2 / sigma^2."""
    cw = np.ascontiguousarray(cw, dtype=np.uint8)
    F, n = cw.shape
    sig = np.float32(sigma)
    if llr_scale is None:
        llr_scale = float(np.float32(2.0 / (float(sig) ** 2)))
    out = np.zeros((F, n), dtype=np.float32)
    _check(lib().ldpc_ref_awgn_llr(_ptr(cw), frame0, F, n, seed, float(sig),
                                   float(llr_scale), _ptr(out)),
           "ldpc_ref_awgn_llr")
    return out


def snr_sigma(seed: int, frame0: int, frames: int, lo: float, hi: float,
              rate: float) -> np.ndarray:
    """Noise level of frames frame0 .. frame0 + frames - 1 of a batch whose
    Eb/N0 is uniform in [lo, hi) dB per frame: u = (top 24 bits of word 0 of
    Philox4x32-10 at counter {0, f mod 2^32, f / 2^32, 0} under key
    {seed mod 2^32, (seed / 2^32) xor 0x534E5253} + 1/2) 2^-24,
    Eb/N0 = lo + (hi - lo) u, and sigma = sqrt(1 / (2 R 10^(Eb/N0 / 10))) for
    unit-energy BPSK, evaluated in double precision (each operation rounded
    once) and rounded to float32.  lo, hi and R are float32 values, as the
    library's interface takes them."""
    lo = float(np.float32(lo))
    hi = float(np.float32(hi))
    rate = float(np.float32(rate))
    key = [seed & 0xFFFFFFFF, ((seed >> 32) ^ 0x534E5253) & 0xFFFFFFFF]
    out = np.empty(frames, dtype=np.float32)
    for i in range(frames):
        f = frame0 + i
        w0 = int(philox4x32_10([0, f & 0xFFFFFFFF, (f >> 32) & 0xFFFFFFFF, 0], key)[0])
        u = ((w0 >> 8) + 0.5) * 2.0 ** -24
        ebn0 = lo + (hi - lo) * u
        out[i] = np.float32(math.sqrt(1.0 / (2.0 * rate * math.pow(10.0, ebn0 / 10.0))))
    return out


def awgn_llr_frames(cw: np.ndarray, frame0: int, seed: int, sigmas) -> np.ndarray:
    """eq. (16)-(17) with a noise level per frame; frame f's LLR scale is
    2 / sigma_f^2 in float32 arithmetic (the square, then the quotient, each
    rounded to float32)."""
    cw = np.ascontiguousarray(cw, dtype=np.uint8)
    out = np.empty(cw.shape, dtype=np.float32)
    for i in range(cw.shape[0]):
        s = np.float32(sigmas[i])
        scale = np.float32(2.0) / (s * s)
        out[i] = awgn_llr(cw[i:i + 1], frame0 + i, seed, float(s), llr_scale=float(scale))[0]
    return out


def mixed_frames(shapes, code_of_frame, ebn0_db=(1.5, 4.5), seed: int = 1,
                 frame_base: int = 0):
    """Info bits and channel LLRs of every frame of a mixed batch, in the
    batch's frame order (lists of uint8[K] and float32[N]): the j-th frame of
    code c has identity synth.mixed_frame_id(c, frame_base + j) for its info
    bits, its Eb/N0 draw (uniform in ebn0_db) and its noise."""
    import synth
    cof = np.asarray(code_of_frame)
    info = [None] * cof.size
    llr = [None] * cof.size
    for ci, s in enumerate(shapes):
        idx = np.nonzero(cof == ci)[0]
        if idx.size == 0:
            continue
        rc = RefCode(s.hbm, s.z)
        f0 = synth.mixed_frame_id(ci, frame_base)
        inf_c = gen_info(seed, f0, idx.size, rc.k)
        sig = snr_sigma(seed, f0, idx.size, ebn0_db[0], ebn0_db[1], rc.k / rc.n)
        x = awgn_llr_frames(rc.encode(inf_c), f0, seed, sig)
        for j, f in enumerate(idx):
            info[f] = inf_c[j]
            llr[f] = x[j]
    return info, llr


def quantize_i8(llr: np.ndarray, scale: float = 4.0, clip: int = 63) -> np.ndarray:
    llr = np.ascontiguousarray(llr, dtype=np.float32)
    out = np.zeros(llr.shape, dtype=np.int8)
    _check(lib().ldpc_ref_quantize_i8(_ptr(llr), _ptr(out), llr.size,
                                      float(scale), int(clip)),
           "ldpc_ref_quantize_i8")
    return out


def unpack_hard(hard: np.ndarray, n: int) -> np.ndarray:
    """[F][ceil(n/32)] LSB-first words -> u8[F][n] bits."""
    hard = np.ascontiguousarray(hard, dtype=np.uint32)
    by = hard.view(np.uint8).reshape(hard.shape[0], -1)
    bits = np.unpackbits(by, axis=1, bitorder="little")
    return bits[:, :n]
