"""Host-side sharding of frames across ranks, run as two gloo processes on
CPU: each rank decodes its share with the oracle and the error counters are
all-reduced; the result must equal one process decoding every frame."""
import os
import socket

import numpy as np
import pytest

import oracle
import synth
from paper_2306_12063_gb300.shard import (frame_offset, mixed_shard, reduce_counters,
                                          shard_range)

FRAMES = 30
EBN0 = 1.5


def _counters(frame0, count):
    s = synth.wifi_n648_r12()
    rc = oracle.RefCode(s.hbm, s.z)
    if count == 0:
        return np.zeros(4, dtype=np.int64)
    info = oracle.gen_info(1, frame0, count, rc.k)
    llr = oracle.awgn_llr(rc.encode(info), frame0, 1, synth.ebn0_db_to_sigma(EBN0, 0.5))
    hard, iters, _ = rc.decode_layered_f32(llr, 8, 0.75, True, True, want_post=False)
    bits = oracle.unpack_hard(hard, rc.n)[:, :rc.k]
    errs = (bits != info).sum(axis=1)
    return np.array([errs.sum(), (errs > 0).sum(), iters.sum(), count], dtype=np.int64)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_path):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        start, count = shard_range(FRAMES, rank, world)
        total = reduce_counters(_counters(start, count))
        mx = reduce_counters([rank], op="max")
        if rank == 0:
            np.save(out_path, np.concatenate([total, mx]))
    finally:
        dist.destroy_process_group()


def test_shard_range_covers_every_frame_once():
    for total in (0, 1, 7, 30, 1001):
        for world in (1, 2, 3, 8):
            seen = []
            for r in range(world):
                s, c = shard_range(total, r, world)
                seen.extend(range(s, s + c))
            assert seen == list(range(total))
    assert frame_offset(0, 0, 100, 3) == 0
    assert frame_offset(1, 2, 100, 3) == 500
    with pytest.raises(ValueError):
        shard_range(5, 2, 2)


def test_two_gloo_ranks_match_one_process(tmp_path):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    out = str(tmp_path / "total.npy")
    mp.spawn(_worker, args=(2, _free_port(), out), nprocs=2, join=True)
    got = np.load(out)
    want = _counters(0, FRAMES)
    assert got[:4].tolist() == want.tolist()
    assert got[4] == 1


MIXED_SHAPES = [synth.tiny_z3_code(), synth.random_small_code(4, 5, 12, 8),
                synth.random_small_code(5, 4, 10, 12)]


def _mixed_counters(first, cof):
    """Frame errors and iteration sum of frames first.. of a mixed batch
    (code cof[i] for frame first + i), decoded by the oracle per code."""
    fe = 0
    it = 0
    for ci, s in enumerate(MIXED_SHAPES):
        idx = np.nonzero(cof == ci)[0]
        if idx.size == 0:
            continue
        rc = oracle.RefCode(s.hbm, s.z)
        for j in idx:
            f = first + int(j)
            info = oracle.gen_info(7, f, 1, rc.k)
            llr = oracle.awgn_llr(rc.encode(info), f, 7, synth.ebn0_db_to_sigma(1.0, rc.k / rc.n))
            hard, iters, _ = rc.decode_layered_f32(llr, 6, 0.75, True, True, want_post=False)
            fe += int((oracle.unpack_hard(hard, rc.n)[0, :rc.k] != info[0]).any())
            it += int(iters[0])
    return np.array([fe, it, cof.size], dtype=np.int64)


def _mixed_worker(rank, world, port, out_path, cof_all):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        first, cof = mixed_shard(cof_all, rank, world)
        total = reduce_counters(_mixed_counters(first, cof))
        if rank == 0:
            np.save(out_path, total)
    finally:
        dist.destroy_process_group()


def test_mixed_shard_splits_in_order():
    cof = np.arange(12) % 5
    parts = [mixed_shard(cof, r, 3) for r in range(3)]
    assert [p[0] for p in parts] == [0, 4, 8]
    assert np.concatenate([p[1] for p in parts]).tolist() == cof.tolist()
    with pytest.raises(ValueError):
        mixed_shard(cof, 0, 5)


def test_two_gloo_ranks_mixed_batch_match_one_process(tmp_path):
    """Weak-scaled mixed batch: two ranks decode their halves of one global
    code assignment; the reduced counters equal one process on all frames."""
    pytest.importorskip("torch")
    import torch.multiprocessing as mp
    cof_all = np.random.default_rng(3).integers(0, len(MIXED_SHAPES), 24).astype(np.int32)
    out = str(tmp_path / "mixed.npy")
    mp.spawn(_mixed_worker, args=(2, _free_port(), out, cof_all), nprocs=2, join=True)
    assert np.load(out).tolist() == _mixed_counters(0, cof_all).tolist()
