"""Block-range sharding across processes (one GPU each) and stream merging.

Blocks are independent (patch-local compression, Sec. 2.5-2.6), so ranks split
the block index range with the balanced partition the paper uses for its rows
(Div/Rem formula of Sec. 2.7.1) and compress their range with no data exchange.
The one collective is an exclusive scan of the shards' payload sizes (the
paper's MPI_Scan for write positions, Sec. 2.7.2); with it every rank knows
where its records land in the merged stream: an addressable header, the
concatenated offset table shifted by the scan, and the concatenated payloads.
The merged stream equals the single-process stream byte for byte.

Z-slab distribution (the data layout of Sec. 2.7.1, where each process owns a
contiguous part of the field): each rank holds the whole block layers
[z0, z1) of every variable and time, compresses that part as a field of its
own and passes the whole field's statistics (an all-gather of each part's
min, max, sum of squares and point count, combined in rank order), so that
the relative and NRMSE bounds, and the NRMSE tolerance of Eq. 4, resolve to
those of the whole field and every part's records are the whole field's.  In
the block order (x fastest, then y, z, t, variable) a part's blocks of one
(variable, time layer) are one contiguous run of the whole field's; the
merged stream interleaves the parts' runs, run by run, and the parallel writer
places them with an exclusive scan of the runs' sizes.

Host-side code only (bytes in, bytes out); works on streams from the GPU
library or from any other writer of the same format.
"""
from __future__ import annotations

import os
import struct
import zlib

import numpy as np

HDR = 128
VARREC = 32


def block_range(nb_total: int, rank: int, world: int):
    """[begin, end) of rank's blocks: Div = nb // P, Rem = nb % P,
    count = Div + (rank < Rem), start = Div * rank + min(rank, Rem)."""
    div, rem = divmod(nb_total, world)
    begin = div * rank + min(rank, rem)
    return begin, begin + div + (1 if rank < rem else 0)


def _align(x, a):
    return (x + a - 1) // a * a


class StreamParts:
    """Header fields, offset table and payload view of one stream."""

    def __init__(self, stream):
        b = bytes(stream) if not isinstance(stream, (bytes, bytearray)) else bytes(stream)
        if len(b) < HDR or b[:4] != b"DLS1":
            raise ValueError("not a DLS stream")
        self.raw = b
        self.nvars = struct.unpack_from("<I", b, 12)[0]
        self.block_begin, self.block_end, self.total_blocks = struct.unpack_from("<qqq", b, 72)
        self.offsets_pos, self.payload_pos, self.total = struct.unpack_from("<QQQ", b, 104)
        if self.total != len(b):
            raise ValueError("stream size does not match its header")
        nb = self.block_end - self.block_begin
        self.offsets = np.frombuffer(b, dtype="<u8", count=nb + 1, offset=self.offsets_pos).astype(np.uint64)
        self.payload = memoryview(b)[self.payload_pos:self.payload_pos + int(self.offsets[-1])]

    @property
    def payload_bytes(self) -> int:
        return int(self.offsets[-1])


def exclusive_scan(sizes):
    out, acc = [], 0
    for s in sizes:
        out.append(acc)
        acc += int(s)
    return out, acc


def merged_header(first: StreamParts, nb_total: int, payload_total: int) -> bytearray:
    """Header + variable table of the merged stream (positions recomputed)."""
    offp = _align(HDR + VARREC * first.nvars, 16)
    payp = _align(offp + 8 * (nb_total + 1), 16)
    h = bytearray(payp)
    h[:offp] = first.raw[:offp]
    struct.pack_into("<qqq", h, 72, 0, nb_total, nb_total)
    struct.pack_into("<QQQQ", h, 96, HDR, offp, payp, payp + payload_total)
    return h


def merge(streams) -> bytes:
    """Concatenates shard streams covering consecutive block ranges (in order)."""
    parts = [StreamParts(s) for s in streams]
    nb_total = parts[0].total_blocks
    pos = 0
    for p in parts:
        if p.block_begin != pos or p.total_blocks != nb_total:
            raise ValueError("shards must cover consecutive block ranges of one field")
        pos = p.block_end
    if pos != nb_total:
        raise ValueError("shards do not cover every block")
    bases, total = exclusive_scan([p.payload_bytes for p in parts])
    h = merged_header(parts[0], nb_total, total)
    offp = struct.unpack_from("<Q", h, 104)[0]
    table = np.empty(nb_total + 1, dtype="<u8")
    for p, base in zip(parts, bases):
        table[p.block_begin:p.block_end] = p.offsets[:-1] + np.uint64(base)
    table[nb_total] = total
    h[offp:offp + 8 * (nb_total + 1)] = table.tobytes()
    return bytes(h) + b"".join(bytes(p.payload) for p in parts)


def write_sharded(path: str, my_stream, rank: int, world: int, group=None) -> int:
    """Every rank writes its records into one file at the position given by the
    exclusive scan of payload sizes (all-gather of one integer per rank), rank 0
    writes the header; returns the file size.  Uses torch.distributed."""
    import torch
    import torch.distributed as dist

    p = StreamParts(my_stream)
    sizes = torch.zeros(world, dtype=torch.int64)
    mine = torch.tensor([p.payload_bytes], dtype=torch.int64)
    gathered = [torch.zeros(1, dtype=torch.int64) for _ in range(world)]
    dist.all_gather(gathered, mine, group=group)
    sizes = [int(t.item()) for t in gathered]
    bases, total = exclusive_scan(sizes)
    nb_total = p.total_blocks
    offp = _align(HDR + VARREC * p.nvars, 16)
    payp = _align(offp + 8 * (nb_total + 1), 16)
    if rank == 0:
        with open(path, "wb") as fh:
            fh.truncate(payp + total)
            fh.seek(0)
            h = merged_header(p, nb_total, total)
            fh.write(bytes(h[:offp]))
            fh.seek(offp + 8 * nb_total)
            fh.write(np.array([total], dtype="<u8").tobytes())
    dist.barrier(group=group)
    fd = os.open(path, os.O_WRONLY)
    try:
        os.pwrite(fd, (p.offsets[:-1] + np.uint64(bases[rank])).astype("<u8").tobytes(), offp + 8 * p.block_begin)
        os.pwrite(fd, bytes(p.payload), payp + bases[rank])
    finally:
        os.close(fd)
    dist.barrier(group=group)
    return payp + total


# ------------------------------------------------------------------ z-slabs

def _cdiv(a, b):
    return -(-a // b)


def zslab_range(nz: int, bz: int, rank: int, world: int):
    """[z0, z1) of rank's z-slab: the Div/Rem partition of the nz // bz whole
    block layers, slab edges on block edges; a ragged last layer (nz % bz
    planes) goes with the last whole one, so that every slab holds at least
    one whole block in z, as a field of its own must."""
    units = nz // bz
    if world > units:
        raise ValueError(f"{world} ranks for {units} whole block layers: every rank needs one")
    b0, b1 = block_range(units, rank, world)
    return b0 * bz, (nz if b1 == units else b1 * bz)


def combine_stats(parts):
    """The whole field's per-variable (min, max, sum of squares, points) from
    the parts' own, in rank order (so every rank combines them alike)."""
    parts = [np.asarray(p, dtype=np.float64).reshape(-1, 4) for p in parts]
    g = parts[0].copy()
    for p in parts[1:]:
        g[:, 0] = np.minimum(g[:, 0], p[:, 0])
        g[:, 1] = np.maximum(g[:, 1], p[:, 1])
        g[:, 2] = g[:, 2] + p[:, 2]
        g[:, 3] = g[:, 3] + p[:, 3]
    return g


def _all_gather_vec(vals, group=None, dtype=None):
    """all_gather of one small vector per rank (CPU tensors on gloo, the
    current CUDA device on NCCL); returns the world's vectors in rank order."""
    import torch
    import torch.distributed as dist

    dev = "cuda" if dist.get_backend(group) == "nccl" else "cpu"
    t = torch.as_tensor(np.asarray(vals), dtype=dtype).reshape(-1).to(dev)
    out = [torch.empty_like(t) for _ in range(dist.get_world_size(group))]
    dist.all_gather(out, t, group=group)
    return [o.cpu().numpy() for o in out]


def allreduce_stats(local, group=None):
    """Every rank's statistics gathered and combined in rank order: the same
    float64 values on every rank (a reduction tree could round differently)."""
    import torch
    return combine_stats([g.reshape(-1, 4) for g in _all_gather_vec(np.asarray(local, np.float64), group,
                                                                     torch.float64)])


class _Slab:
    """One part's stream with its geometry: dims, block, runs of records."""

    def __init__(self, stream):
        self.p = StreamParts(stream)
        b = self.p.raw
        self.dims = struct.unpack_from("<4q", b, 16)
        self.block = struct.unpack_from("<4I", b, 48)
        if self.p.block_begin != 0 or self.p.block_end != self.p.total_blocks:
            raise ValueError("a z-slab stream must hold every block of its slab")
        nbk = [_cdiv(d, k) for d, k in zip(self.dims, self.block)]
        self.nbz = nbk[2]
        self.run = nbk[0] * nbk[1] * nbk[2]            # blocks of one (variable, time layer)
        self.nruns = self.p.total_blocks // self.run
        # everything but the geometry must agree between the parts
        self.key = zlib.crc32(bytes(b[64:72]) + bytes(b[48:64]) + struct.pack("<3q", self.dims[0], self.dims[1],
                                                                              self.dims[3]) +
                              bytes(b[HDR:HDR + VARREC * self.p.nvars]))

    def run_sizes(self):
        o = self.p.offsets
        return np.array([int(o[(r + 1) * self.run]) - int(o[r * self.run]) for r in range(self.nruns)],
                        dtype=np.int64)


def _zslab_plan(nz_list, bz):
    for z in nz_list[:-1]:
        if z % bz:
            raise ValueError("every z-slab but the last must hold whole block layers")
    return sum(nz_list)


def merge_zslabs(streams) -> bytes:
    """The whole field's stream from its z-slabs' streams (in z order)."""
    parts = [_Slab(s) for s in streams]
    a = parts[0]
    if any(q.key != a.key or q.nruns != a.nruns for q in parts):
        raise ValueError("z-slab streams of different fields or bounds")
    nz = _zslab_plan([q.dims[2] for q in parts], a.block[2])
    nb_total = sum(q.p.total_blocks for q in parts)
    sizes, chunks = [], []
    for r in range(a.nruns):
        for q in parts:
            lo, hi = r * q.run, (r + 1) * q.run
            o = q.p.offsets
            sizes.append(np.diff(o[lo:hi + 1].astype(np.int64)))
            chunks.append(bytes(q.p.payload[int(o[lo]):int(o[hi])]))
    sizes = np.concatenate(sizes)
    total = int(sizes.sum())
    h = merged_header(a.p, nb_total, total)
    struct.pack_into("<q", h, 16 + 8 * 2, nz)
    offp = struct.unpack_from("<Q", h, 104)[0]
    table = np.zeros(nb_total + 1, dtype="<u8")
    table[1:] = np.cumsum(sizes).astype(np.uint64)
    h[offp:offp + 8 * (nb_total + 1)] = table.tobytes()
    return bytes(h) + b"".join(chunks)


def write_zslabs(path: str, my_stream, rank: int, world: int, group=None) -> int:
    """Every rank writes its z-slab's records into one file, run by run, at
    the positions an exclusive scan of all runs' sizes (merged order: run of
    the whole field's (variable, time layer), then rank) gives; rank 0 writes
    the header.  One all-gather of (header digest, slab layers, run sizes) per
    rank.  Returns the file size; the file equals merge_zslabs of the parts."""
    import torch
    import torch.distributed as dist

    q = _Slab(my_stream)
    mine = np.concatenate([[q.key, q.dims[2], q.nbz, q.nruns], q.run_sizes()]).astype(np.int64)
    lens = _all_gather_vec([mine.size], group, torch.int64)
    if any(int(l[0]) != mine.size for l in lens):
        raise ValueError("z-slab streams of different fields or bounds")
    allv = _all_gather_vec(mine, group, torch.int64)
    if any(int(v[0]) != q.key or int(v[3]) != q.nruns for v in allv):
        raise ValueError("z-slab streams of different fields or bounds")
    nz_list = [int(v[1]) for v in allv]
    nbz = [int(v[2]) for v in allv]
    sizes = np.stack([v[4:] for v in allv])                 # world x nruns
    nz = _zslab_plan(nz_list, q.block[2])
    nbxy = q.run // q.nbz
    nbz_total = sum(nbz)
    nb_total = nbxy * nbz_total * q.nruns
    # exclusive scan in merged order (run-major, then rank)
    flat = sizes.T.reshape(-1)
    bases = np.concatenate([[0], np.cumsum(flat)[:-1]]).reshape(q.nruns, world)
    total = int(flat.sum())
    offp = _align(HDR + VARREC * q.p.nvars, 16)
    payp = _align(offp + 8 * (nb_total + 1), 16)
    if rank == 0:
        h = merged_header(q.p, nb_total, total)
        struct.pack_into("<q", h, 16 + 8 * 2, nz)
        with open(path, "wb") as fh:
            fh.truncate(payp + total)
            fh.seek(0)
            fh.write(bytes(h[:offp]))
            fh.seek(offp + 8 * nb_total)
            fh.write(np.array([total], dtype="<u8").tobytes())
    dist.barrier(group=group)
    fd = os.open(path, os.O_WRONLY)
    try:
        o = q.p.offsets.astype(np.int64)
        before = sum(nbz[:rank]) * nbxy
        for j in range(q.nruns):
            lo, hi = j * q.run, (j + 1) * q.run
            base = int(bases[j, rank])
            ent = (o[lo:hi] - o[lo] + base).astype("<u8")
            os.pwrite(fd, ent.tobytes(), offp + 8 * (j * nbz_total * nbxy + before))
            os.pwrite(fd, bytes(q.p.payload[int(o[lo]):int(o[hi])]), payp + base)
    finally:
        os.close(fd)
    dist.barrier(group=group)
    return payp + total
