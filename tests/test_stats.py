"""Host-side FER statistics against closed forms and brute force."""
import math
from fractions import Fraction

import pytest

from paper_2306_12063_gb300 import stats


def test_wilson_known_values():
    # k = 0: upper limit z^2 / (n + z^2)
    z = 1.959963984540054
    lo, hi = stats.wilson_interval(0, 10)
    assert lo == 0.0 and abs(hi - z * z / (10 + z * z)) < 1e-12
    # symmetric case: centred on 1/2
    lo, hi = stats.wilson_interval(50, 100)
    assert abs((lo + hi) / 2 - 0.5) < 1e-12
    # Wilson (1927) limits for 1 of 20 with z = 1.96: (0.0089, 0.2361)
    lo, hi = stats.wilson_interval(1, 20, 1.96)
    assert abs(lo - 0.00889) < 5e-5 and abs(hi - 0.23613) < 5e-5


@pytest.mark.parametrize("b,n", [(0, 0), (3, 5), (7, 7), (10, 18), (0, 4), (12, 30)])
def test_binomial_tail_brute_force(b, n):
    exact = sum(Fraction(math.comb(n, k), 2 ** n) for k in range(b, n + 1)) if b <= n else 0
    assert abs(stats.binom_sf(b, n) - float(exact)) < 1e-12


def test_mcnemar_large_counts_normal_limit():
    # b = c: p ~ 1/2 plus half the central atom
    p = stats.mcnemar_one_sided(5000, 5000)
    assert 0.5 < p < 0.51
    # 3 sigma excess: one-sided p near 1.35e-3
    n = 10000
    b = int(n / 2 + 3 * math.sqrt(n) / 2)
    assert 1e-3 < stats.mcnemar_one_sided(b, n - b) < 1.6e-3


def test_compare_summary():
    s = stats.compare([900, 30, 25, 45], 1000)
    assert s["fer_a"] == 0.07 and s["fer_b"] == 0.075
    assert s["matched"] and s["mcnemar_p_a_worse"] > 0.5
    s = stats.compare([900, 5, 60, 35], 1000)
    assert not s["matched"]
