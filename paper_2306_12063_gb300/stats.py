"""Frame-error-rate statistics for comparing two decoders on the same frames.

* Wilson score interval of a binomial proportion (Wilson, 1927).
* McNemar's test on paired outcomes (McNemar, 1947), exact form: among the
  frames where exactly one decoder fails, the number b failed only by
  decoder A is Binomial(b + c, 1/2) when both decoders have the same error
  rate.  The one-sided p-value for "A is worse" is P(X >= b).

Host-side arithmetic on a handful of counts; nothing here touches frames.
"""
from __future__ import annotations

import math
from typing import Tuple


def wilson_interval(k: int, n: int, z: float = 1.959963984540054) -> Tuple[float, float]:
    """Two-sided Wilson score interval for k successes in n trials (95 % by
    default)."""
    if n <= 0:
        return (0.0, 1.0)
    p = k / n
    z2 = z * z
    den = 1.0 + z2 / n
    mid = (p + z2 / (2 * n)) / den
    half = z * math.sqrt(p * (1 - p) / n + z2 / (4 * n * n)) / den
    return (max(0.0, mid - half), min(1.0, mid + half))


def binom_sf(b: int, n: int) -> float:
    """P(X >= b) for X ~ Binomial(n, 1/2), summed in log space."""
    if b <= 0:
        return 1.0
    if b > n:
        return 0.0
    ln_half_n = -n * math.log(2.0)
    logs = [math.lgamma(n + 1) - math.lgamma(k + 1) - math.lgamma(n - k + 1) + ln_half_n
            for k in range(b, n + 1)]
    m = max(logs)
    return min(1.0, math.exp(m) * sum(math.exp(x - m) for x in logs))


def mcnemar_one_sided(only_a_wrong: int, only_b_wrong: int) -> float:
    """Exact one-sided McNemar p-value for "decoder A fails more often than
    decoder B", from the discordant frame counts."""
    return binom_sf(int(only_a_wrong), int(only_a_wrong) + int(only_b_wrong))


def compare(counts, frames: int, alpha: float = 0.05) -> dict:
    """Summary of ldpc_paired_frame_errors counts [both right, only B wrong,
    only A wrong, both wrong] for A against B."""
    c = [int(x) for x in counts]
    fa = c[2] + c[3]
    fb = c[1] + c[3]
    p = mcnemar_one_sided(c[2], c[1])
    return {"fer_a": fa / frames, "fer_b": fb / frames,
            "wilson95_a": wilson_interval(fa, frames), "wilson95_b": wilson_interval(fb, frames),
            "only_a_wrong": c[2], "only_b_wrong": c[1],
            "mcnemar_p_a_worse": p, "matched": p >= alpha}
