"""Oracle of the global-basis mode (one basis per variable for all patches).

Test infrastructure: only the tests (and the benchmark's CPU baseline) may
import it.  Plain numpy in FP64, one function per definition, no blocking or
fusion; numpy's SVD and matrix-vector product serve as library steps.

What it computes, by definition:
- the modes (Sec. 2.3, Eq. 2-3): the right singular vectors, by decreasing
  singular value, of a sample matrix whose rows are patches of the first
  snapshot (``learn_basis``);
- the per-patch L2 budget eps_l from the global target (Sec. 2.4, Eq. 4;
  ``local_tolerance``);
- the coefficients of a patch on the modes, alpha = Phi^T u (Sec. 2.5, Eq. 5),
  and the smallest set of largest-magnitude coefficients whose reconstruction
  meets eps_l (Eq. 6), the set size found by bisection (``compress_patch``);
- every patch of every snapshot through that map and back (``compress`` /
  ``decompress``).

Readings where the paper is silent or loose:
- G1 patches tile each snapshot from the origin (x fastest within a patch);
  the snapshot's extents must be multiples of the patch, since an edge patch
  would not fit the basis; a 2-D field (nz = 1) uses m x m patches.
- G2 the sample: S patch origins drawn uniformly with replacement over every
  position where a patch fits, handed in by the caller (the method's random
  draws are inputs); Algorithm 1 uses S = 4 m^3.
- G3 mode k is the right singular vector of the k-th largest singular value,
  signed so that its largest-magnitude component is positive (lowest index on
  ties).
- G4 the budget: eps = eps_t ||u|| / 100 over all points of the variable, and
  eps_l^2 = eps^2 M / K for a patch of M points out of K (all snapshots), so
  meeting eps_l on every patch of every snapshot meets the global target.
- G5 coefficients are ranked by decreasing magnitude; equal magnitudes keep
  index order.
- G6 stored values: q = rint(alpha / delta), ties to even, with delta =
  eps / sqrt(K) (the global budget's RMS per point), standing in for
  bit-grooming; the test of a prefix uses the stored values, so it also
  covers their rounding: pass(n) <=> ||u - sum_{s<n} q_s delta phi_s||^2 <=
  eps_l^2 (Algorithm 1 prints <=), the kept modes added in kept order.  With
  every mode kept the error is the rounding alone, at most M delta^2 / 4 <
  eps_l^2, so every patch passes at some n <= M.
"""
from __future__ import annotations

import numpy as np


def patch_shape(dims, m: int):
    """(px, py, pz) of the patches of a field with dims (nx, ny, nz, nt) (G1)."""
    return (int(m), int(m), int(m) if int(dims[2]) > 1 else 1)


def _check_tiling(dims, patch):
    for d, p in zip(dims[:3], patch):
        if int(d) % int(p):
            raise ValueError("the snapshot extents must be multiples of the patch (G1)")


def gather_patch(snap: np.ndarray, origin, patch) -> np.ndarray:
    """The M values of the patch at origin (x0, y0, z0) of a snapshot laid out
    (nz, ny, nx), x fastest."""
    x0, y0, z0 = (int(v) for v in origin)
    px, py, pz = patch
    return np.asarray(snap[z0:z0 + pz, y0:y0 + py, x0:x0 + px], dtype=np.float64).reshape(-1)


def learn_basis(snap0: np.ndarray, origins: np.ndarray, patch):
    """The modes of Sec. 2.3 (Eq. 2-3): Q (S x M) from the sampled patches of
    the first snapshot, Q = U Sigma V^T, Phi = V (M x M, column k = mode k),
    with the singular values (zero beyond the rank of Q) and the sign rule G3."""
    Q = np.stack([gather_patch(snap0, o, patch) for o in origins])
    _, s, vt = np.linalg.svd(Q, full_matrices=True)
    phi = vt.T.copy()
    M = phi.shape[0]
    sv = np.zeros(M)
    sv[:s.size] = s
    for k in range(M):
        col = phi[:, k]
        if col[int(np.argmax(np.abs(col)))] < 0.0:
            phi[:, k] = -col
    return phi, sv


def local_tolerance(field: np.ndarray, eps_t: float, M: int):
    """G4 and G6: (eps_l^2, delta) for a variable (all snapshots) and a target
    NRMSE eps_t in percent."""
    x = np.asarray(field, dtype=np.float64)
    K = x.size
    eps = eps_t * np.sqrt(np.sum(x * x)) / 100.0
    return eps * eps * M / K, eps / np.sqrt(K)


def reconstruct(phi: np.ndarray, idx: np.ndarray, q: np.ndarray, delta: float) -> np.ndarray:
    """sum over the kept modes, in kept order, of q_s delta phi_s."""
    rec = np.zeros(phi.shape[0])
    for s in range(len(idx)):
        rec = rec + (float(q[s]) * delta) * phi[:, int(idx[s])]
    return rec


def compress_patch(u: np.ndarray, phi: np.ndarray, eps_l2: float, delta: float):
    """One patch: alpha = Phi^T u (Eq. 5), the coefficients ranked by
    decreasing magnitude (G5), quantized (G6), and the smallest n with pass(n)
    (Eq. 6) by bisection over [0, M].  Returns (kept mode indices in kept
    order, their q, the squared error at n)."""
    u = np.asarray(u, dtype=np.float64)
    if delta == 0.0:
        # an all-zero variable: eps = 0 and every patch is zero, kept by no mode
        return np.zeros(0, np.int64), np.zeros(0, np.int64), float(np.dot(u, u))
    alpha = phi.T @ u
    order = np.argsort(-np.abs(alpha), kind="stable")
    q_all = np.rint(alpha / delta)

    def err2(n):
        d = u - reconstruct(phi, order[:n], q_all[order[:n]], delta)
        return float(np.dot(d, d))

    lo, hi = 0, phi.shape[0]
    while lo < hi:
        mid = (lo + hi) // 2
        if err2(mid) <= eps_l2:
            hi = mid
        else:
            lo = mid + 1
    idx = order[:lo].copy()
    return idx, q_all[idx].astype(np.int64), err2(lo)


def compress(field: np.ndarray, m: int, eps_t: float, origins: np.ndarray):
    """One variable laid out (nt, nz, ny, nx): the basis from the first
    snapshot's sampled patches, then every patch of every snapshot.  Returns a
    dict with the basis, the singular values, the patch shape, eps_l^2, delta
    and the records (t, origin, kept indices, q, squared error)."""
    f = np.asarray(field, dtype=np.float64)
    nt, nz, ny, nx = f.shape
    dims = (nx, ny, nz, nt)
    patch = patch_shape(dims, m)
    _check_tiling(dims, patch)
    phi, sv = learn_basis(f[0], origins, patch)
    M = phi.shape[0]
    eps_l2, delta = local_tolerance(f, eps_t, M)
    recs = []
    px, py, pz = patch
    for t in range(nt):
        for z0 in range(0, nz, pz):
            for y0 in range(0, ny, py):
                for x0 in range(0, nx, px):
                    u = gather_patch(f[t], (x0, y0, z0), patch)
                    idx, q, e2 = compress_patch(u, phi, eps_l2, delta)
                    recs.append((t, (x0, y0, z0), idx, q, e2))
    return dict(phi=phi, sv=sv, patch=patch, dims=dims, eps_l2=eps_l2, delta=delta, recs=recs)


def decompress(res) -> np.ndarray:
    """The field (nt, nz, ny, nx) from the records: every patch rebuilt from its
    kept modes (Algorithm 2 for the global basis)."""
    nx, ny, nz, nt = res["dims"]
    px, py, pz = res["patch"]
    out = np.zeros((nt, nz, ny, nx))
    for t, (x0, y0, z0), idx, q, _ in res["recs"]:
        rec = reconstruct(res["phi"], idx, q, res["delta"])
        out[t, z0:z0 + pz, y0:y0 + py, x0:x0 + px] = rec.reshape(pz, py, px)
    return out


# ---------------------------------------------------------------- stream
# Readings for the stored form (the paper keeps the DOFs and the basis, then
# gzip, Sec. 2.5-2.6; it gives no layout):
# - header (little-endian): b"DLSG", u32 version 1, u32 M, u32 px, py, pz,
#   u64 nx, ny, nz, nt, f64 eps_l^2, f64 delta, u64 records  (80 bytes);
# - the basis once, M x M float64, mode after mode;
# - (records + 1) u64 byte offsets of the records (a scan of their sizes, so
#   that every record is addressable, Sec. 2.7.2);
# - records in (t, z, y, x) patch order: u32 n, u8 wv, 3 zero bytes, then n
#   mode indices of ib = bit_width(M - 1) bits and n zigzag(q) of wv bits,
#   LSB first in 32-bit words; each record padded to 8 bytes.
_MAGIC = b"DLSG"
_HDR = 80


def _width(x: int) -> int:
    return int(x).bit_length()


def _zz(q):
    q = np.asarray(q, dtype=np.int64)
    return ((q << 1) ^ (q >> 63)).astype(np.uint64)


def _pack_bits(vals, width, nbits_total):
    words = np.zeros(max(1, (nbits_total + 31) // 32), np.uint64)
    pos = 0
    for v in vals:
        v = int(v)
        for i in range(width):
            if (v >> i) & 1:
                words[(pos + i) >> 5] |= np.uint64(1 << ((pos + i) & 31))
        pos += width
    return words.astype(np.uint32), pos


def _record(idx, q, M):
    n = len(idx)
    ib = _width(M - 1)
    z = _zz(q)
    wv = _width(int(z.max())) if n else 0
    nbits = n * (ib + wv)
    w1, p1 = _pack_bits(idx, ib, nbits)
    words = w1.astype(np.uint64)
    pos = p1
    for v in z:                                   # values after the indices
        v = int(v)
        for i in range(wv):
            if (v >> i) & 1:
                words[(pos + i) >> 5] |= np.uint64(1 << ((pos + i) & 31))
        pos += wv
    body = words.astype(np.uint32)[: (nbits + 31) // 32].tobytes()
    rec = np.uint32(n).tobytes() + bytes([wv, 0, 0, 0]) + body
    return rec + bytes((-len(rec)) % 8)


def pack(res) -> bytes:
    """The stream of a compress() result."""
    phi = res["phi"]
    M = phi.shape[0]
    px, py, pz = res["patch"]
    nx, ny, nz, nt = res["dims"]
    recs = [_record(idx, q, M) for _, _, idx, q, _ in res["recs"]]
    offs = np.zeros(len(recs) + 1, np.uint64)
    offs[1:] = np.cumsum([len(r) for r in recs])
    hdr = (_MAGIC + np.array([1, M, px, py, pz], np.uint32).tobytes()
           + np.array([nx, ny, nz, nt], np.uint64).tobytes()
           + np.array([res["eps_l2"], res["delta"]], np.float64).tobytes()
           + np.uint64(len(recs)).tobytes())
    assert len(hdr) == _HDR
    basis = np.ascontiguousarray(phi.T).astype(np.float64).tobytes()   # mode after mode
    return hdr + basis + offs.tobytes() + b"".join(recs)


def _get_bits(words, pos, width):
    v = 0
    for i in range(width):
        p = pos + i
        v |= int((int(words[p >> 5]) >> (p & 31)) & 1) << i
    return v


def unpack(stream: bytes):
    """The compress()-like result of a stream (records without their errors),
    or None when the stream is malformed."""
    b = bytes(stream)
    if len(b) < _HDR or b[:4] != _MAGIC:
        return None
    ver, M, px, py, pz = np.frombuffer(b[4:24], np.uint32)
    nx, ny, nz, nt = (int(v) for v in np.frombuffer(b[24:56], np.uint64))
    eps_l2, delta = np.frombuffer(b[56:72], np.float64)
    nrec = int(np.frombuffer(b[72:80], np.uint64)[0])
    M, px, py, pz = int(M), int(px), int(py), int(pz)
    if ver != 1 or M != px * py * pz or M < 1:
        return None
    if any(d % p for d, p in zip((nx, ny, nz), (px, py, pz))) or nrec != nt * (nx // px) * (ny // py) * (nz // pz):
        return None
    at = _HDR + 8 * M * M
    if len(b) < at + 8 * (nrec + 1):
        return None
    phi = np.frombuffer(b[_HDR:at], np.float64).reshape(M, M).T.copy()
    offs = np.frombuffer(b[at:at + 8 * (nrec + 1)], np.uint64).astype(np.int64)
    base = at + 8 * (nrec + 1)
    if offs[0] != 0 or np.any(np.diff(offs) < 8) or base + offs[-1] != len(b):
        return None
    ib = _width(M - 1)
    recs = []
    i = 0
    for t in range(nt):
        for z0 in range(0, nz, pz):
            for y0 in range(0, ny, py):
                for x0 in range(0, nx, px):
                    r = b[base + offs[i]: base + offs[i + 1]]
                    n = int(np.frombuffer(r[:4], np.uint32)[0])
                    wv = r[4]
                    need = 8 + ((n * (ib + wv) + 31) // 32) * 4
                    if n > M or wv > 63 or need + ((-need) % 8) != len(r):
                        return None
                    words = np.frombuffer(r[8:8 + ((n * (ib + wv) + 31) // 32) * 4], np.uint32)
                    idx = np.array([_get_bits(words, s * ib, ib) for s in range(n)], np.int64)
                    zz = [_get_bits(words, n * ib + s * wv, wv) for s in range(n)]
                    q = np.array([(v >> 1) ^ -(v & 1) for v in zz], np.int64)
                    if np.any(idx >= M):
                        return None
                    recs.append((t, (x0, y0, z0), idx, q, None))
                    i += 1
    return dict(phi=phi, sv=None, patch=(px, py, pz), dims=(nx, ny, nz, nt), eps_l2=float(eps_l2),
                delta=float(delta), recs=recs)
