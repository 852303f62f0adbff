"""Pins for the oracle's code model and direct encoder (Section 1-3,
eq. 2-15).  Nothing here runs the CUDA library."""
import numpy as np
import pytest

import oracle
import synth
from helpers import dense_h, gf2_encode

ALL_SHAPES = [synth.wifi_n648_r12(), synth.wifi_n1944_r56(), synth.eq7_wimax_r34(),
              synth.tiny_z2_code(), synth.tiny_z3_code(), synth.wimax_n2304_r56()]


def test_worked_example_rows(golden_z2):
    c = synth.tiny_z2_code()
    rc = oracle.RefCode(c.hbm, c.z)
    assert rc.y == 1 and rc.encodable == 1
    for r in range(6):
        assert rc.row_vars(r).tolist() == [int(v) for v in golden_z2[f"row{r}"]]


def test_worked_example_codeword(golden_z2):
    c = synth.tiny_z2_code()
    rc = oracle.RefCode(c.hbm, c.z)
    cw = rc.encode(np.array([golden_z2["info"]], dtype=np.uint8))
    assert cw[0].tolist() == [int(v) for v in golden_z2["codeword"]]


def test_tiny_code_closed_form_v0():
    """For the Z=2 code, summing every block row leaves P_0 v0 = sum_i S_i
    (eq. 12 with h_b(y) = 0); working it through gives v0 = [t, t] with t the
    XOR of all four info bits.  Exhaustive over the 16 info words."""
    c = synth.tiny_z2_code()
    rc = oracle.RefCode(c.hbm, c.z)
    infos = ((np.arange(16)[:, None] >> np.arange(4)[None, :]) & 1).astype(np.uint8)
    cw = rc.encode(infos)
    t = infos.sum(axis=1) & 1
    assert (cw[:, 4] == t).all() and (cw[:, 5] == t).all()


@pytest.mark.parametrize("shape", ALL_SHAPES, ids=lambda s: s.name)
def test_parity_checks_hold(shape):
    """H c^T = 0 over a dense H expanded independently from H_bm."""
    rc = oracle.RefCode(shape.hbm, shape.z)
    rng = np.random.default_rng(7)
    info = rng.integers(0, 2, size=(8, rc.k), dtype=np.uint8)
    cw = rc.encode(info)
    H = dense_h(shape.hbm, shape.z).astype(np.int64)
    syn = (cw.astype(np.int64) @ H.T) & 1
    assert not syn.any()
    assert (cw[:, :rc.k] == info).all()          # systematic, eq. (1)
    for w in cw:
        assert rc.syndrome_weight(w) == 0


@pytest.mark.parametrize("shape", ALL_SHAPES[:3], ids=lambda s: s.name)
def test_linearity(shape):
    rc = oracle.RefCode(shape.hbm, shape.z)
    rng = np.random.default_rng(11)
    a = rng.integers(0, 2, size=(4, rc.k), dtype=np.uint8)
    b = rng.integers(0, 2, size=(4, rc.k), dtype=np.uint8)
    assert ((rc.encode(a) ^ rc.encode(b)) == rc.encode(a ^ b)).all()


@pytest.mark.parametrize("shape", [synth.wifi_n648_r12(), synth.tiny_z2_code(),
                                   synth.tiny_z3_code(),
                                   synth.random_small_code(4, 5, 9, 7)],
                         ids=lambda s: s.name)
def test_matches_gaussian_elimination(shape):
    """The parity part is unique (P_{h_b(y)} invertible, dual diagonal
    triangular), so the direct encoder must equal a GF(2) solve of
    H_p p = H_s s."""
    rc = oracle.RefCode(shape.hbm, shape.z)
    rng = np.random.default_rng(3)
    for _ in range(3):
        info = rng.integers(0, 2, size=rc.k, dtype=np.uint8)
        assert (rc.encode(info[None])[0] == gf2_encode(shape.hbm, shape.z, info)).all()


def test_eq7_structure_found():
    """eq. (7): the R=3/4 WiMAX H_b2 block has its middle h_b entry 80 at y=2."""
    c = synth.eq7_wimax_r34()
    assert c.hbm[:, c.kb].tolist() == [0, -1, 80, -1, -1, 0]
    rc = oracle.RefCode(c.hbm, c.z)
    assert rc.y == 2 and rc.encodable == 1


def test_table_shapes():
    """Tab. 1 / Tab. 2 arithmetic: N = Nb Z and K = R N for the stand-ins."""
    a, b = synth.wifi_n648_r12(), synth.wifi_n1944_r56()
    assert (a.n, a.k, a.z) == (648, 324, 27)
    assert (b.n, b.k, b.z) == (1944, 1620, 81)
    mixed = synth.wimax_mixed_set()
    assert len(mixed) == 76
    kbytes = {(1, 2): 36, (2, 3): 48, (3, 4): 54, (5, 6): 60}   # Tab. 2, Z = 24 row
    for c in mixed:
        num, den = c.meta["rate"]
        assert c.n == 24 * c.z
        assert c.k * den == c.n * num
        if c.z == 24:
            assert c.k // 8 == kbytes[(num, den)]
        oracle.RefCode(c.hbm, c.z)   # every member passes the structure check


@pytest.mark.parametrize("bad", ["hb_unpaired", "two_middles", "no_diag", "shift_range"])
def test_structure_rejected(bad):
    c = synth.wifi_n648_r12()
    h = c.hbm.copy()
    kb = c.kb
    if bad == "hb_unpaired":
        h[c.mb - 1, kb] = 2
    elif bad == "two_middles":
        h[3, kb] = 5
    elif bad == "no_diag":
        h[4, kb + 1 + 4] = -1
    elif bad == "shift_range":
        h[0, 0] = c.z
    with pytest.raises(oracle.OracleError):
        oracle.RefCode(h, c.z)
