"""Block-range sharding across ranks (CPU, gloo): shard streams written with
the exclusive scan of payload sizes form exactly the single-process stream."""
import os
import tempfile

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

import oracle
from paper_2601_20113_gb300 import shard, synth

DIMS = (40, 36, 20, 36)
BLOCK = (16, 16, 8, 16)


def _field():
    return synth.modes3d(*DIMS, seed=31, count=16).numpy()


def _cfg(eb, begin=0, end=-1):
    return oracle.Config(DIMS, BLOCK, oracle.F32, eb=eb, rank_cap=16, block_begin=begin, block_end=end)


def test_block_range_is_the_div_rem_partition():
    for nb in (1, 7, 54, 1000):
        for world in (1, 2, 3, 8):
            rs = [shard.block_range(nb, r, world) for r in range(world)]
            assert rs[0][0] == 0 and rs[-1][1] == nb
            assert all(rs[i][1] == rs[i + 1][0] for i in range(world - 1))
            counts = [e - b for b, e in rs]
            assert max(counts) - min(counts) <= 1
            assert counts == sorted(counts, reverse=True)


@pytest.mark.parametrize("world", [2, 3, 5])
def test_merge_equals_single_stream(world):
    f = _field()
    eb = 1e-3 * float(f.max() - f.min())
    st, full, _ = oracle.compress(_cfg(eb), f)
    nb = oracle.num_blocks(_cfg(eb))
    parts = []
    for r in range(world):
        b, e = shard.block_range(nb, r, world)
        st, s, _ = oracle.compress(_cfg(eb, b, e), f)
        assert st == 0
        parts.append(s.tobytes())
    merged = shard.merge(parts)
    assert merged == full.tobytes()
    st, rec = oracle.decompress(np.frombuffer(merged, np.uint8))
    assert st == 0 and np.abs(rec.astype(np.float64) - f).max() <= eb


def _rank_main(rank, world, port, path, eb):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    f = _field()
    nb = oracle.num_blocks(_cfg(eb))
    b, e = shard.block_range(nb, rank, world)
    st, s, _ = oracle.compress(_cfg(eb, b, e), f, nthreads=1)
    assert st == 0
    shard.write_sharded(path, s, rank, world)
    dist.destroy_process_group()


def test_gloo_ranks_write_one_stream():
    f = _field()
    eb = 1e-3 * float(f.max() - f.min())
    st, full, _ = oracle.compress(_cfg(eb), f)
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "field.dls")
        port = 29500 + (os.getpid() % 1000)
        mp.start_processes(_rank_main, args=(2, port, path, eb), nprocs=2, join=True, start_method="spawn")
        with open(path, "rb") as fh:
            got = fh.read()
    assert got == full.tobytes()
