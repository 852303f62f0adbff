"""The C-ABI library builds, loads and exports every entry point of
include/ldpc.h, and its host-side argument checks answer with the documented
status codes.  None of these calls reaches a GPU."""
import ctypes

import numpy as np
import pytest

import paper_2306_12063_gb300 as ldpc
import synth
from paper_2306_12063_gb300 import _build


@pytest.fixture(scope="module")
def lib():
    _build.build()
    return ldpc.load()


def test_exports_every_declared_symbol(lib):
    names = ldpc.symbols()
    assert len(names) >= 14
    for name in names:
        assert hasattr(lib, name), name


def _create(lib, h, z):
    out = ctypes.c_void_p()
    st = lib.ldpc_code_create(h.ctypes.data_as(ctypes.c_void_p) if h is not None else None,
                              h.shape[0] if h is not None else 0,
                              h.shape[1] if h is not None else 0, z, ctypes.byref(out))
    return st, out


@pytest.mark.parametrize("case,want", [
    ("null", 1), ("mb2", 1), ("nb_big", 1), ("z0", 1), ("z_big", 1),
    ("entry_range", 2), ("hb_unpaired", 2), ("hb_two", 2), ("hb_none", 2), ("diag", 2),
])
def test_create_rejects(lib, case, want):
    c = synth.wifi_n648_r12()
    h, z = c.hbm.copy(), c.z
    kb = c.kb
    if case == "null":
        st, _ = _create(lib, None, z)
        assert st == want
        return
    if case == "mb2":
        h = h[:2]
    elif case == "nb_big":
        h = np.concatenate([h, h[:, :10]], axis=1)
    elif case == "z0":
        z = 0
    elif case == "z_big":
        z = 385
    elif case == "entry_range":
        h[1, 1] = z
    elif case == "hb_unpaired":
        h[c.mb - 1, kb] = 3
    elif case == "hb_two":
        h[2, kb] = 4
    elif case == "hb_none":
        h[6, kb] = -1
    elif case == "diag":
        h[6, kb + 4] = 0   # off the dual diagonal of column kb+4 (rows 3, 4)
    h = np.ascontiguousarray(h)
    st, out = _create(lib, h, z)
    assert st == want
    assert out.value is None
    assert len(lib.ldpc_last_error()) > 0


def test_null_handles_rejected(lib):
    p = ldpc._Params(10, 0.75, 1, 0)
    assert lib.ldpc_decode_layered_minsum(None, 0, None, 4, ctypes.byref(p), None, None,
                                          None, None) == 1
    assert lib.ldpc_encode(None, None, None, 1, None) == 1
    assert lib.ldpc_code_info(None, None, None, None, None, None) == 1
    assert lib.ldpc_frame_stats(None, None, None, None, 1, 10, None, None) == 1
    assert lib.ldpc_sync(None, None, 1.0) == 1
    assert lib.ldpc_decode_host_workspace_bytes(None, 0, 64) == 0
    lib.ldpc_code_destroy(None)


def test_argument_ranges_rejected(lib):
    # clip outside [0, 127] and negative sizes are refused before any launch
    assert lib.ldpc_quantize_pack_i8(None, None, 4, 10, 4.0, 200, None) == 1
    assert lib.ldpc_quantize_pack_i8(None, None, -1, 10, 4.0, 63, None) == 1
    assert lib.ldpc_gen_info(1, 0, -5, 10, None, None) == 1
    assert lib.ldpc_awgn_llr(None, 0, 4, 10, 1, -1.0, 1.0, None, None) == 1
    # zero-sized work is a no-op that needs no buffers
    assert lib.ldpc_quantize_pack_i8(None, None, 0, 10, 4.0, 63, None) == 0
    assert lib.ldpc_gen_info(1, 0, 0, 10, None, None) == 0


def test_symbols_parsed_from_header():
    names = ldpc.symbols()
    for must in ("ldpc_code_create", "ldpc_encode", "ldpc_decode_layered_minsum",
                 "ldpc_quantize_pack_i8", "ldpc_last_error"):
        assert must in names


def test_newer_entry_points_check_arguments_on_the_host(lib):
    """Per-frame Eb/N0 and channel, Adam, learned decoding and training,
    mixed plans, the paper variants, the host pipeline and the bounded-wait
    check refuse bad arguments with LDPC_ERR_INVALID_ARG before any device
    work, and zero-sized work succeeds without buffers."""
    p = ldpc._Params(10, 0.75, 1, 0)
    out = ctypes.c_void_p()
    bad = [
        lib.ldpc_snr_sigma(1, 0, 4, 1.0, 4.0, 0.0, None, None),         # rate 0
        lib.ldpc_snr_sigma(1, 0, 4, 5.0, 4.0, 0.5, None, None),         # lo > hi
        lib.ldpc_snr_sigma(1, 0, -1, 1.0, 4.0, 0.5, None, None),        # negative count
        lib.ldpc_snr_sigma(1, 0, 4, 1.0, 4.0, 0.5, None, None),         # NULL output
        lib.ldpc_awgn_llr_frames(None, 0, 4, 10, 1, None, None, None),
        lib.ldpc_adam_step(None, None, None, None, -1, 1, 1e-3, 0.9, 0.999, 1e-8, None),
        lib.ldpc_adam_step(None, None, None, None, 4, 0, 1e-3, 0.9, 0.999, 1e-8, None),
        lib.ldpc_decode_learned_minsum(None, None, 4, None, 8, 1, None, None, None, None),
        lib.ldpc_learned_train_forward(None, None, None, 4, None, 8, None, None, None, 1.0,
                                       None, None),
        lib.ldpc_codeset_create(None, 0, ctypes.byref(out)),
        lib.ldpc_mixed_plan_create(None, None, 4, ctypes.byref(out)),
        lib.ldpc_decode_mixed(None, 0, None, ctypes.byref(p), None, None, None, None),
        lib.ldpc_mixed_autotune(None, 0, None, ctypes.byref(p), None, None, 3, None),
        lib.ldpc_quantize_i16(None, None, 4, 16.0, 10, None),
        lib.ldpc_encode_bitmap(None, None, None, 4, None),
        lib.ldpc_decode_flooding_minsum(None, None, 4, ctypes.byref(p), None, None, None, None),
        lib.ldpc_decode_host(None, 0, None, 4, ctypes.byref(p), None, None, None, 0, 4, None),
        lib.ldpc_paired_frame_errors(None, None, None, None, 4, None, None),
        lib.ldpc_check_bounded_wait(None, 100, None),
    ]
    assert bad == [1] * len(bad), bad
    assert out.value is None
    assert lib.ldpc_snr_sigma(1, 0, 0, 1.0, 4.0, 0.5, None, None) == 0
    assert lib.ldpc_awgn_llr_frames(None, 0, 0, 10, 1, None, None, None) == 0
    assert lib.ldpc_adam_step(None, None, None, None, 0, 1, 1e-3, 0.9, 0.999, 1e-8, None) == 0
