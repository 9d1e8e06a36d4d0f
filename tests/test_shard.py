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


# ------------------------------------------------------------------ z-slabs
# Two variables on (x, y, z, t) = (40, 36, 44, 20) with 16 x 16 x 8 x 16
# blocks: 5 whole block layers in z and a ragged one (4 of 8), which rides
# with the last whole layer; ragged in x, y and t too.
ZDIMS = (40, 36, 44, 20)


def _field2():
    a = synth.modes3d(*ZDIMS, seed=31, count=16).numpy()
    b = synth.modes3d(*ZDIMS, seed=32, count=12).numpy() * 3.0 + 1.5
    return np.concatenate([a, b], axis=0)


EB = {oracle.EB_ABS: (2e-3, 6e-3), oracle.EB_REL_RANGE: (1e-3, 2e-3), oracle.EB_NRMSE: (0.5, 0.8)}


def _cfg2(dims, eb_type, gstats=None):
    return oracle.Config(dims, BLOCK, oracle.F32, eb=np.array(EB[eb_type]), eb_type=eb_type, rank_cap=16, nvars=2,
                         global_stats=gstats)


def _slab(f, z0, z1):
    return np.ascontiguousarray(f[:, :, z0:z1])


def _own_stats(x):
    """(min, max, sum of squares, points) per variable of a part."""
    x = x.reshape(x.shape[0], -1).astype(np.float64)
    return np.stack([x.min(1), x.max(1), (x * x).sum(1), np.full(x.shape[0], float(x.shape[1]))], axis=1)


def _slab_streams(f, world, eb_type, use_gstats=True):
    nz = ZDIMS[2]
    ranges = [shard.zslab_range(nz, BLOCK[2], r, world) for r in range(world)]
    parts = [_slab(f, z0, z1) for z0, z1 in ranges]
    g = shard.combine_stats([_own_stats(p) for p in parts])
    out = []
    for (z0, z1), p in zip(ranges, parts):
        dims = (ZDIMS[0], ZDIMS[1], z1 - z0, ZDIMS[3])
        st, s, _ = oracle.compress(_cfg2(dims, eb_type, g if use_gstats else None), p)
        assert st == 0
        out.append(s.tobytes())
    return g, out


def test_zslab_range_covers_whole_layers():
    for nz, bz in ((20, 8), (256, 16), (33, 4)):
        for world in range(1, min(nz // bz, 9) + 1):
            rs = [shard.zslab_range(nz, bz, r, world) for r in range(world)]
            assert rs[0][0] == 0 and rs[-1][1] == nz
            assert all(rs[i][1] == rs[i + 1][0] and rs[i][1] % bz == 0 for i in range(world - 1))
            assert all(z1 - z0 >= bz for z0, z1 in rs)
            layers = [(z1 - z0) // bz for z0, z1 in rs]
            assert max(layers) - min(layers) <= 1
    with pytest.raises(ValueError):
        shard.zslab_range(20, 8, 0, 3)


def test_combine_stats_is_the_whole_fields():
    f = _field2()
    parts = [_slab(f, 0, 8), _slab(f, 8, 32), _slab(f, 32, 44)]
    g = shard.combine_stats([_own_stats(p) for p in parts])
    w = _own_stats(f)
    np.testing.assert_array_equal(g[:, [0, 1, 3]], w[:, [0, 1, 3]])      # exact under any grouping
    np.testing.assert_allclose(g[:, 2], w[:, 2], rtol=1e-12)


@pytest.mark.parametrize("world", [2, 3])
@pytest.mark.parametrize("eb_type", [oracle.EB_ABS, oracle.EB_REL_RANGE, oracle.EB_NRMSE])
def test_zslab_merge_equals_whole_stream(eb_type, world):
    """Parts compressed with the whole field's statistics, merged run by run,
    give the whole field's stream byte for byte (compressed with the same
    statistics; for the pointwise bounds also without any, min and max being
    exact under any grouping)."""
    f = _field2()
    g, parts = _slab_streams(f, world, eb_type)
    merged = shard.merge_zslabs(parts)
    st, whole, _ = oracle.compress(_cfg2(ZDIMS, eb_type, g), f)
    assert st == 0 and merged == whole.tobytes()
    if eb_type != oracle.EB_NRMSE:
        st, plain, _ = oracle.compress(_cfg2(ZDIMS, eb_type), f)
        assert st == 0 and merged == plain.tobytes()
    st, rec = oracle.decompress(np.frombuffer(merged, np.uint8))
    assert st == 0 and rec.shape == f.shape
    err = rec.astype(np.float64) - f
    if eb_type == oracle.EB_NRMSE:
        for v in range(2):
            rms = np.sqrt(np.mean(err[v] ** 2)) / np.sqrt(np.mean(f[v].astype(np.float64) ** 2)) * 100
            assert rms <= EB[eb_type][v]
    else:
        _, vars_ = oracle.resolve(_cfg2(ZDIMS, eb_type), f)
        for v in range(2):
            assert np.abs(err[v]).max() <= vars_[v].eb


@pytest.mark.parametrize("eb_type", [oracle.EB_REL_RANGE, oracle.EB_NRMSE])
def test_zslab_parts_on_their_own_statistics_do_not_merge(eb_type):
    """Without the whole field's statistics each part resolves its own range
    or norm and point count, so the parts' bounds differ from each other's
    and merging refuses them: the statistics exchange is needed."""
    f = _field2()
    g, parts = _slab_streams(f, 2, eb_type, use_gstats=False)
    with pytest.raises(ValueError):
        shard.merge_zslabs(parts)


def test_zslab_merge_refuses_mismatched_parts():
    f = _field2()
    _, a = _slab_streams(f, 2, oracle.EB_ABS)
    _, b = _slab_streams(f, 2, oracle.EB_REL_RANGE)
    with pytest.raises(ValueError):
        shard.merge_zslabs([a[0], b[1]])
    with pytest.raises(ValueError):
        shard.merge_zslabs([a[1], a[0]])           # the ragged slab first


def test_oracle_refuses_bad_global_stats():
    f = _field2()
    good = _own_stats(f)
    for i, j, val in ((0, 0, np.nan), (1, 0, 1e9), (0, 2, -1.0), (1, 3, good[1, 3] + 1), (0, 3, 0.5)):
        g = good.copy()
        g[i, j] = val
        st, _, _ = oracle.compress(_cfg2(ZDIMS, oracle.EB_NRMSE, g), f)
        assert st != 0


def _zslab_rank_main(rank, world, port, path, eb_type):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    f = _field2()
    z0, z1 = shard.zslab_range(ZDIMS[2], BLOCK[2], rank, world)
    part = _slab(f, z0, z1)
    g = shard.allreduce_stats(_own_stats(part))
    st, s, _ = oracle.compress(_cfg2((ZDIMS[0], ZDIMS[1], z1 - z0, ZDIMS[3]), eb_type, g), part, nthreads=1)
    assert st == 0
    shard.write_zslabs(path, s, rank, world)
    np.save(path + f".g{rank}.npy", g)
    dist.destroy_process_group()


@pytest.mark.parametrize("eb_type", [oracle.EB_REL_RANGE, oracle.EB_NRMSE])
def test_gloo_zslab_ranks_write_one_stream(eb_type):
    """Two gloo ranks, each with its own z-slab: statistics all-gathered and
    combined, records written at the scanned run positions; the file is the
    whole field's stream."""
    f = _field2()
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "field.dls")
        port = 29500 + (os.getpid() + 7 * eb_type) % 1000 + 1000
        mp.start_processes(_zslab_rank_main, args=(2, port, path, eb_type), nprocs=2, join=True,
                           start_method="spawn")
        with open(path, "rb") as fh:
            got = fh.read()
        g0, g1 = np.load(path + ".g0.npy"), np.load(path + ".g1.npy")
    np.testing.assert_array_equal(g0, g1)
    st, whole, _ = oracle.compress(_cfg2(ZDIMS, eb_type, g0), f)
    assert st == 0 and got == whole.tobytes()
    g, parts = _slab_streams(f, 2, eb_type)
    np.testing.assert_array_equal(g, g0)
    assert got == shard.merge_zslabs(parts)
