"""Run by tests/test_gpu_debug_build.py in a process of its own: decodes
with the debug build of the library (edge offsets checked against the
posterior region inside the kernels) and checks that the outputs equal the
oracle's and that no check fired (ldpc_sync raises if one did)."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402
import torch  # noqa: E402

import oracle  # noqa: E402
import synth  # noqa: E402
from paper_2306_12063_gb300 import _build  # noqa: E402

_build.LIB = _build.build(debug=True)
import paper_2306_12063_gb300 as ldpc  # noqa: E402

ldpc.load()


def pack_i8(q):
    F, n = q.shape
    G = (F + 3) // 4
    pad = np.full((4 * G, n), 63, dtype=np.int8)
    pad[:F] = q
    b = pad.reshape(G, 4, n).astype(np.uint8).astype(np.uint32)
    return (b[:, 0] | (b[:, 1] << 8) | (b[:, 2] << 16) | (b[:, 3] << 24)).view(np.int32)


for shape in (synth.wifi_n648_r12(), synth.wifi_n1944_r56(), synth.tiny_z3_code()):
    rc = oracle.RefCode(shape.hbm, shape.z)
    code = ldpc.Code(shape.hbm, shape.z)
    F = 21
    info = oracle.gen_info(1, 0, F, rc.k)
    llr = oracle.awgn_llr(rc.encode(info), 0, 1, synth.ebn0_db_to_sigma(2.5, rc.k / rc.n))
    wh, wi, wp = rc.decode_layered_f32(llr, 12, 0.75, True, True)
    gh, gi, gp = code.decode(torch.from_numpy(llr).cuda(), max_iters=12, early_stop=True,
                             want_post=True)
    code.sync()
    assert (gi.cpu().numpy() == wi).all() and (gp.cpu().numpy() == wp).all()
    q = oracle.quantize_i8(llr)
    wh, wi, wp, _ = rc.decode_layered_i8(q, 12, True, True)
    gh, gi, gp = code.decode(torch.from_numpy(pack_i8(q)).cuda(), frames=F, dtype=ldpc.I8X4,
                             max_iters=12, early_stop=True, want_post=True)
    code.sync()
    assert (gi.cpu().numpy() == wi).all() and (gp.cpu().numpy() == wp).all()
    q16 = oracle.quantize_i16(llr, 16.0, 10)
    wh, wi, wp, _ = rc.decode_layered_i16w(q16, 12, normalise=True, early_stop=True)
    gh, gi, gp = code.decode(torch.from_numpy(q16).cuda(), dtype=ldpc.I16W, max_iters=12,
                             normalise=True, early_stop=True, want_post=True)
    code.sync()
    assert (gi.cpu().numpy() == wi).all() and (gp.cpu().numpy() == wp).all()
    w = np.random.default_rng(2).uniform(0.5, 1.0, (4, rc.nnz_blocks)).astype(np.float32)
    wh, wi, wp = rc.decode_learned_f32(llr, w, max_iters=4, early_stop=True)
    gh, gi, gp = code.decode_learned(torch.from_numpy(llr).cuda(), torch.from_numpy(w).cuda(),
                                     early_stop=True, want_post=True)
    code.sync()
    assert (gi.cpu().numpy() == wi).all() and (gp.cpu().numpy() == wp).all()
# the int8 saturation count against the oracle's, on inputs heavy in +-127
rng = np.random.default_rng(9)
for shape in (synth.wifi_n648_r12(), synth.wifi_n1944_r56()):
    rc = oracle.RefCode(shape.hbm, shape.z)
    code = ldpc.Code(shape.hbm, shape.z)
    F = 37
    q = rng.choice(np.array([-127, -126, -3, -1, 0, 1, 2, 125, 127], dtype=np.int8),
                   size=(F, rc.n))
    code.saturation_count()   # clear
    wh, wi, wp, events = rc.decode_layered_i8(q, 9, True, True)
    gh, gi, gp = code.decode(torch.from_numpy(pack_i8(q)).cuda(), frames=F, dtype=ldpc.I8X4,
                             max_iters=9, early_stop=True, want_post=True)
    code.sync()
    assert (gi.cpu().numpy() == wi).all() and (gp.cpu().numpy() == wp).all()
    got = code.saturation_count()
    assert events > 0 and got == events, (got, events)
print("debug build ok")
