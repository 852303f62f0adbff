"""The decode entry point for callers that cannot allocate device memory
(ldpc_decode_layered_minsum_noalloc): a real-time thread with a fixed memory
budget, a framework that owns every device allocation, or a steady-state
path where cudaMalloc / cudaFree are not allowed.  Called through the C-ABI
twice in a row, it must give exactly what the oracle and the handle-based
decoder give.  This file is collected last so that a failure here leaves
every other test already run; it also passes on its own in a fresh
process."""
import ctypes

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ldpc():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2306_12063_gb300 import _build
    _build.build()
    import paper_2306_12063_gb300 as m
    m.load()
    return m


def _inputs(shape, frames, ebn0):
    rc = oracle.RefCode(shape.hbm, shape.z)
    info = oracle.gen_info(1, 0, frames, rc.k)
    llr = oracle.awgn_llr(rc.encode(info), 0, 1, synth.ebn0_db_to_sigma(ebn0, rc.k / rc.n))
    return rc, llr


def _noalloc(ldpc, shape, dtype, llr_dev, frames, max_iters, out):
    lib = ldpc.load()
    hbm = np.ascontiguousarray(shape.hbm, dtype=np.int16)
    p = ldpc._Params(max_iters, 0.75, 1, 1)
    hard, iters, post = out
    st = lib.ldpc_decode_layered_minsum_noalloc(
        hbm.ctypes.data_as(ctypes.c_void_p), hbm.shape[0], hbm.shape[1], shape.z, dtype,
        llr_dev.data_ptr(), frames, ctypes.byref(p), hard.data_ptr(), iters.data_ptr(),
        post.data_ptr(), torch.cuda.current_stream().cuda_stream)
    assert st == 0, lib.ldpc_last_error()


@pytest.mark.parametrize("dtype_name", ["f32", "i8"])
@pytest.mark.parametrize("shape_name,frames,ebn0", [("wifi1944", 3001, 4.0),
                                                    ("wifi648", 1001, 2.0)])
def test_noalloc_matches_handle_decoder(ldpc, dtype_name, shape_name, frames, ebn0):
    shape = {"wifi1944": synth.wifi_n1944_r56(), "wifi648": synth.wifi_n648_r12()}[shape_name]
    rc, llr = _inputs(shape, frames, ebn0)
    code = ldpc.Code(shape.hbm, shape.z)
    if dtype_name == "f32":
        dtype = ldpc.F32
        dev_in = torch.from_numpy(llr).cuda()
        post_dtype = torch.float32
        ref_h, ref_i, ref_p = rc.decode_layered_f32(llr, 20, 0.75, True, True)
    else:
        dtype = ldpc.I8X4
        dev_in = ldpc.quantize_pack_i8(torch.from_numpy(llr).cuda())
        post_dtype = torch.int8
        ref_h, ref_i, ref_p, _ = rc.decode_layered_i8(oracle.quantize_i8(llr), 20, True, True)
    want_h, want_i, want_p = code.decode(dev_in, frames=frames, dtype=dtype, max_iters=20,
                                         early_stop=True, want_post=True)
    for call in range(2):   # the second call reuses the static array left by the first
        out = (torch.full((frames, code.nwords), -1, dtype=torch.int32, device="cuda"),
               torch.full((frames,), -1, dtype=torch.int32, device="cuda"),
               torch.zeros((frames, code.n), dtype=post_dtype, device="cuda"))
        _noalloc(ldpc, shape, dtype, dev_in, frames, 20, out)
        torch.cuda.synchronize()
        # against the oracle (posteriors compared with ==, so +0 equals -0)
        assert (out[1].cpu().numpy() == ref_i).all(), f"iterations differ from the oracle ({call})"
        assert (out[0].cpu().numpy().view(np.uint32) == ref_h).all(), \
            f"hard decisions differ from the oracle on call {call}"
        assert (out[2].cpu().numpy() == ref_p).all(), f"posteriors differ from the oracle ({call})"
        # and against the handle-based decoder
        assert torch.equal(out[1], want_i), f"iteration counts differ on call {call}"
        assert torch.equal(out[0], want_h), f"hard decisions differ on call {call}"
        assert torch.equal(out[2], want_p), f"posteriors differ on call {call}"


def test_noalloc_rejects_codes_beyond_the_static_array(ldpc):
    """mb = 12, Z = 384 needs 12 * 12 * 8 * 64 = 73728 table bytes > 65280."""
    lib = ldpc.load()
    h = synth.random_small_code(7, 12, 24, 384).hbm
    h = np.ascontiguousarray(h, dtype=np.int16)
    p = ldpc._Params(10, 0.75, 1, 1)
    st = lib.ldpc_decode_layered_minsum_noalloc(
        h.ctypes.data_as(ctypes.c_void_p), 12, 24, 384, ldpc.F32, None, 4, ctypes.byref(p),
        None, None, None, None)
    assert st == 6
    assert b"static scratch" in lib.ldpc_last_error()
