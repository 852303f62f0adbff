"""Seeded synthetic workloads shared by the CUDA path and by the CPU oracle.

This module holds the code *shapes* and the seeded pseudo-random choices that
define them.  It contains none of the decoding or encoding arithmetic: it only
draws base (model) matrices H_bm whose structure follows Section 1 (eq. 2-7)
of Palenik & Szitkey, "High Throughput Open-Source Implementation of Wi-Fi 6
and WiMAX LDPC Encoder and Decoder" (arXiv 2306.12063), with the shapes of
Tab. 1 (IEEE 802.11 codes: Z in {27, 54, 81}) and Tab. 2 (IEEE 802.16 codes:
N = 24 Z, Z = 24..96 step 4).

The standard's own base matrices are not used; these are seeded stand-ins
with the same N, Z, rate and the same h_b / dual-diagonal parity structure
(eq. 3-7), so that the direct encoder of Section 2 applies.

Pseudo-random numbers come from xoshiro256** seeded through splitmix64
(Blackman & Vigna, "Scrambled linear pseudorandom number generators", 2021),
written out below from their published definitions.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Sequence, Tuple

import numpy as np

_M64 = (1 << 64) - 1


def splitmix64_stream(seed: int):
    """splitmix64 (Steele, Lea & Flood 2014): yields 64-bit words."""
    state = seed & _M64
    while True:
        state = (state + 0x9E3779B97F4A7C15) & _M64
        z = state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
        yield z ^ (z >> 31)


def _rotl(x: int, k: int) -> int:
    return ((x << k) | (x >> (64 - k))) & _M64


class Xoshiro256ss:
    """xoshiro256** 1.0, state filled from splitmix64(seed)."""

    def __init__(self, seed: int):
        sm = splitmix64_stream(seed)
        self.s = [next(sm) for _ in range(4)]

    def next_u64(self) -> int:
        s = self.s
        result = (_rotl((s[1] * 5) & _M64, 7) * 9) & _M64
        t = (s[1] << 17) & _M64
        s[2] ^= s[0]
        s[3] ^= s[1]
        s[1] ^= s[2]
        s[0] ^= s[3]
        s[2] ^= t
        s[3] = _rotl(s[3], 45)
        return result

    def below(self, n: int) -> int:
        """Uniform integer in [0, n): modulo with rejection of the biased
        low region (threshold = 2^64 mod n), so every value is equally likely."""
        if n <= 0:
            raise ValueError("n must be positive")
        threshold = ((1 << 64) - n) % n
        while True:
            x = self.next_u64()
            if x >= threshold:
                return x % n

    def uniform01(self) -> float:
        """Uniform double in [0, 1) from the top 53 bits."""
        return (self.next_u64() >> 11) * (1.0 / (1 << 53))

    def sample_without_replacement(self, population: int, k: int) -> List[int]:
        """k distinct values of range(population), in draw order (partial
        Fisher-Yates shuffle)."""
        pool = list(range(population))
        out = []
        for i in range(k):
            j = i + self.below(population - i)
            pool[i], pool[j] = pool[j], pool[i]
            out.append(pool[i])
        return out


@dataclass
class CodeShape:
    """A QC-LDPC code given by its base matrix (eq. 2): H_bm[i][j] = -1 is a
    zero Z x Z block, s >= 0 the identity cyclically shifted by s."""

    name: str
    hbm: np.ndarray  # int16 [mb, nb], row-major
    z: int
    meta: dict = field(default_factory=dict)

    @property
    def mb(self) -> int:
        return int(self.hbm.shape[0])

    @property
    def nb(self) -> int:
        return int(self.hbm.shape[1])

    @property
    def kb(self) -> int:
        return self.nb - self.mb

    @property
    def n(self) -> int:
        return self.nb * self.z

    @property
    def k(self) -> int:
        return self.kb * self.z

    @property
    def m(self) -> int:
        return self.mb * self.z

    @property
    def rate(self) -> float:
        return self.k / self.n


def shaped_base_matrix(
    rng: Xoshiro256ss,
    mb: int,
    nb: int,
    z: int,
    info_weights: Sequence[int],
    hb_shifts: Tuple[int, int, int],
    y: int,
    shift_range: int | None = None,
) -> np.ndarray:
    """Draw a base matrix with the parity structure of eq. (3)-(7).

    * Info columns j = 0..Kb-1 (H_b1, eq. 4), in order: a weight d drawn
      uniformly from ``info_weights``, then d distinct rows drawn uniformly
      without replacement, then for each chosen row (in draw order) a shift.
      With ``shift_range`` None the shift is uniform in [0, z); otherwise s is
      uniform in [0, shift_range) and the entry is floor(s * z / shift_range)
      (the scaling from the largest WiMAX Z to a smaller one).
    * Column Kb (h_b, eq. 5): hb_shifts[0] at row 0, hb_shifts[1] at row y,
      hb_shifts[2] at row mb-1 (paired equal values first and last).
    * Columns Kb+1+t (H_b2', eq. 6), t = 0..mb-2: shift 0 at rows t and t+1
      (the dual diagonal).
    """
    kb = nb - mb
    h = np.full((mb, nb), -1, dtype=np.int16)
    for j in range(kb):
        d = info_weights[rng.below(len(info_weights))]
        rows = rng.sample_without_replacement(mb, d)
        for r in rows:
            if shift_range is None:
                s = rng.below(z)
            else:
                s = (rng.below(shift_range) * z) // shift_range
            h[r, j] = s
    a0, ay, a1 = hb_shifts
    h[0, kb] = a0
    h[y, kb] = ay
    h[mb - 1, kb] = a1
    for t in range(mb - 1):
        h[t, kb + 1 + t] = 0
        h[t + 1, kb + 1 + t] = 0
    return h


def wifi_n648_r12(seed: int = 0) -> CodeShape:
    """Wi-Fi-6-shaped N=648, Z=27, R=1/2 (Tab. 1): 12x24 base matrix, info
    columns of weight 3-4, h_b shifts 1 / 0 / 1 at rows 0 / 6 / 11."""
    rng = Xoshiro256ss(seed)
    h = shaped_base_matrix(rng, 12, 24, 27, (3, 4), (1, 0, 1), 6)
    return CodeShape("wifi_n648_r12", h, 27, {"seed": seed})


def wifi_n1944_r56(seed: int = 2) -> CodeShape:
    """Wi-Fi-6-shaped N=1944, Z=81, R=5/6 (Tab. 1): 4x24 base matrix, info
    columns of weight 2-4, h_b shifts 1 / 0 / 1 at rows 0 / 2 / 3."""
    rng = Xoshiro256ss(seed)
    h = shaped_base_matrix(rng, 4, 24, 81, (2, 3, 4), (1, 0, 1), 2)
    return CodeShape("wifi_n1944_r56", h, 81, {"seed": seed})


WIMAX_Z = tuple(range(24, 97, 4))            # Tab. 2: 19 subblock sizes
WIMAX_RATES = ((1, 2, 12), (2, 3, 8), (3, 4, 6), (5, 6, 4))  # (num, den, Mb)


def wimax_mixed_set(seed: int = 3) -> List[CodeShape]:
    """The 19 x 4 WiMAX-shaped codes (N = 24 Z, Tab. 2) of the mixed-size
    workload, drawn from one xoshiro256** stream in (Z ascending, rate
    ascending) order.  Shifts are floor(s Z / 96) of s uniform in [0, 96);
    h_b = 1 / 0 / 1 at rows 0 / Mb/2 / Mb-1; info weights {3,4} for Mb >= 6,
    {2,3,4} for Mb = 4."""
    rng = Xoshiro256ss(seed)
    out = []
    for z in WIMAX_Z:
        for num, den, mb in WIMAX_RATES:
            weights = (3, 4) if mb >= 6 else (2, 3, 4)
            h = shaped_base_matrix(rng, mb, 24, z, weights, (1, 0, 1), mb // 2,
                                   shift_range=96)
            out.append(CodeShape(f"wimax_n{24 * z}_r{num}{den}", h, z,
                                 {"seed": seed, "rate": (num, den)}))
    return out


def wimax_n2304_r56(seed: int = 3) -> CodeShape:
    """The Z=96, R=5/6 member of the mixed set: the WiMAX N=2304, R=5/6 shape
    on which the paper quotes decoder throughput (Tab. 5)."""
    for c in wimax_mixed_set(seed):
        if c.z == 96 and c.mb == 4:
            return c
    raise AssertionError("unreachable")


def eq7_wimax_r34(seed: int = 5) -> CodeShape:
    """The H_b2 block printed as eq. (7) (WiMAX R=3/4, Z=96: h_b =
    [0,-1,80,-1,-1,0], y = 2, 6x5 dual diagonal) under a seeded H_b1 of
    info-column weight 3-4."""
    rng = Xoshiro256ss(seed)
    h = shaped_base_matrix(rng, 6, 24, 96, (3, 4), (0, 80, 0), 2)
    return CodeShape("eq7_wimax_r34", h, 96, {"seed": seed})


def tiny_z2_code() -> CodeShape:
    """Hand-sized code (Z=2, Mb=3, Nb=5, Kb=2) used for the worked example:
    h_b = [1, 0, 1], y = 1."""
    h = np.array([[0, 1, 1, 0, -1],
                  [1, -1, 0, 0, 0],
                  [-1, 0, 1, -1, 0]], dtype=np.int16)
    return CodeShape("tiny_z2", h, 2)


def tiny_z3_code() -> CodeShape:
    """Z=3 variant of the tiny code (K = 6), small enough for brute-force ML."""
    h = np.array([[0, 2, 1, 0, -1],
                  [1, -1, 0, 0, 0],
                  [-1, 0, 1, -1, 0]], dtype=np.int16)
    return CodeShape("tiny_z3", h, 3)


def random_small_code(seed: int, mb: int, nb: int, z: int) -> CodeShape:
    """A seeded code of arbitrary small shape with the eq. (3)-(7) parity
    structure (y = mb // 2), for tests across many tiles and ragged tails."""
    rng = Xoshiro256ss(seed)
    weights = (2, 3) if mb < 4 else (2, 3, 4)
    a = rng.below(z)
    b = rng.below(z)
    h = shaped_base_matrix(rng, mb, nb, z, weights, (a, b, a), mb // 2)
    return CodeShape(f"rand_s{seed}_{mb}x{nb}_z{z}", h, z, {"seed": seed})


def mixed_frame_assignment(n_codes: int, frames: int, seed: int = 3):
    """Per-frame code index and Eb/N0 (dB, uniform in [1.5, 4.5)) for the
    mixed-size workload, from a stream derived from ``seed``."""
    rng = Xoshiro256ss(seed ^ 0x6D69786564)  # "mixed"
    idx = np.empty(frames, dtype=np.int32)
    ebn0 = np.empty(frames, dtype=np.float64)
    for f in range(frames):
        idx[f] = rng.below(n_codes)
        ebn0[f] = 1.5 + 3.0 * rng.uniform01()
    return idx, ebn0


def mixed_frame_id(code_index: int, j: int) -> int:
    """Identity of the j-th frame of code `code_index` in a mixed batch: the
    counter of its info-bit, noise and Eb/N0 draws (code index in the high
    32 bits, so the codes' streams never overlap)."""
    return (int(code_index) << 32) + int(j)


def ebn0_db_to_sigma(ebn0_db: float, rate: float) -> float:
    """Noise standard deviation for BPSK with unit symbol energy at the given
    Eb/N0 and code rate: sigma^2 = 1 / (2 R 10^(Eb/N0 / 10)).  The paper does
    not print this relation; it is the usual one for eq. (16)."""
    return float(np.sqrt(1.0 / (2.0 * rate * 10.0 ** (ebn0_db / 10.0))))
