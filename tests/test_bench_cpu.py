"""The benchmark's reported arithmetic, checked on the host: the algorithmic
operation count behind roofline.frac, the peak it is divided by, and the
committed ncu summaries it reads its DRAM traffic from."""
import os
import re

import numpy as np
import pytest

import bench
import synth


def test_algorithmic_operations_per_frame_iteration():
    # 13 operations per edge and 4 per check row, per frame and iteration;
    # the int8 count is per four-frame word
    assert bench.OPS_PER_EDGE == 13 and bench.OPS_PER_ROW == 4
    s = synth.wifi_n1944_r56()
    E = int((s.hbm >= 0).sum()) * s.z
    M = s.mb * s.z
    assert (E, M) == (5427, 324)
    iters = 1_000_003
    assert bench._alg_ops(E, M, iters, False) == iters * (13 * E + 4 * M)
    assert bench._alg_ops(E, M, iters, True) == iters * (13 * E + 4 * M) / 4


def test_roofline_fraction_from_the_line_fields():
    """frac = (iterations x (13 E + 4 M) / 4) / launch seconds / (152 SMs x 128
    lanes x SM clock): with one launch per step, launch time = ms_per_step
    when nothing else runs in the step."""
    s = synth.wifi_n1944_r56()
    E, M = int((s.hbm >= 0).sum()) * s.z, s.mb * s.z
    frames, mean_iters, ms, mhz = 786432, 5.014, 16.05, 2070.0
    ops = bench._alg_ops(E, M, int(round(frames * mean_iters)), True)
    peak = bench.SMS * bench.LANES_PER_SM * mhz * 1e6
    frac = ops / (ms * 1e-3) / peak
    assert 0.10 < frac < 0.12
    assert bench.SMS * bench.LANES_PER_SM == 19456


@pytest.mark.parametrize("tag,bytes_per_frame", [("ldpc_decode_i8_wifi1944", 1944 + 4 * 61 + 4),
                                                  ("ldpc_decode_f32_wifi1944",
                                                   4 * 1944 + 4 * 61 + 4)])
def test_profile_summaries(tag, bytes_per_frame):
    """Each decoder summary records the digest of the kernel sources it was
    captured on and its DRAM bytes scaled to one benchmark launch (786,432
    frames); when the digest is the current one (the benchmark then reports
    the traffic), the bytes lie within 10 % of the algorithmic bytes."""
    path = os.path.join(bench.ROOT, "profiles", f"{tag}.md")
    txt = open(path).read()
    assert re.search(r"source_sha256_16:\s*[0-9a-f]{16}", txt)
    t = float(re.search(r"traffic_bytes_per_launch:\s*([0-9.e+]+)", txt).group(1))
    alg = 786432 * bytes_per_frame
    traffic = bench._profile_traffic(tag)
    if traffic is None:
        pytest.skip("summary taken on other kernel sources; the benchmark reports no traffic")
    assert traffic == t
    assert abs(traffic / alg - 1.0) < 0.10


def test_kernel_digest_ignores_comments():
    a = "int f(int x) { return x + 1; }  // one\n/* two */\n"
    b = "int f(int x)\n{\n    return x + 1;   // changed comment\n}\n"
    assert bench.code_text(a) == bench.code_text(b)
    assert bench.code_text(a) != bench.code_text(a.replace("+ 1", "+ 2"))
