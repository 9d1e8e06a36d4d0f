"""Block-range sharding across processes (one GPU each) and stream merging.

Blocks are independent (patch-local compression, Sec. 2.5-2.6), so ranks split
the block index range with the balanced partition the paper uses for its rows
(Div/Rem formula of Sec. 2.7.1) and compress their range with no data exchange.
The one collective is an exclusive scan of the shards' payload sizes (the
paper's MPI_Scan for write positions, Sec. 2.7.2); with it every rank knows
where its records land in the merged stream: an addressable header, the
concatenated offset table shifted by the scan, and the concatenated payloads.
The merged stream equals the single-process stream byte for byte.

Host-side code only (bytes in, bytes out); works on streams from the GPU
library or from any other writer of the same format.
"""
from __future__ import annotations

import os
import struct

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
