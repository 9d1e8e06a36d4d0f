"""Plain FP64 CPU oracle for Discontinuous DLS block compression.

TEST INFRASTRUCTURE ONLY: this package is imported by ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` and by
nothing in the product path.  It shares no code with the CUDA library.

The arithmetic lives in ``dls_oracle.c`` (plain C, FP64, OpenMP over blocks);
this module only builds it with gcc and marshals numpy arrays through ctypes.
Each wrapper names the paper passage (arXiv 2601.20113) its C function follows.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dls_oracle.c")
_SO = os.path.join(_HERE, "libdls_oracle.so")
_lock = threading.Lock()
_lib = None

F32, F64 = 0, 1
EB_ABS, EB_REL_RANGE, EB_NRMSE = 0, 1, 2
OK, ERR_INVALID_ARG, ERR_CAPACITY, ERR_NONFINITE, ERR_CORRUPT = 0, -1, -2, -3, -4


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain IEEE FP64: no fast-math, no contraction)."""
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= max(
        os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "dls_oracle.h"))
    ):
        return _SO
    tmp = _SO + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fno-fast-math", "-ffp-contract=off", "-fopenmp",
           "-fPIC", "-shared", "-Wall", "-Wno-unused-function", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True, cwd=_HERE)
    os.replace(tmp, _SO)
    return _SO


class Params(C.Structure):
    _fields_ = [
        ("nvars", C.c_int32),
        ("dims", C.c_int64 * 4),
        ("block", C.c_int32 * 4),
        ("dtype", C.c_int32),
        ("eb_type", C.c_int32),
        ("eb", C.POINTER(C.c_double)),
        ("rank_cap", C.c_int32),
        ("block_begin", C.c_int64),
        ("block_end", C.c_int64),
        ("basis", C.POINTER(C.c_double)),
        ("basis_n", C.c_int32),
        ("corr_codec", C.c_int32),
        ("global_stats", C.POINTER(C.c_double)),
    ]


class Geom(C.Structure):
    _fields_ = [
        ("v", C.c_int32), ("x0", C.c_int64), ("y0", C.c_int64), ("z0", C.c_int64), ("t0", C.c_int64),
        ("sx", C.c_int32), ("sy", C.c_int32), ("sz", C.c_int32), ("st", C.c_int32),
        ("M", C.c_int64), ("T", C.c_int64), ("N", C.c_int64), ("L", C.c_int64),
        ("n", C.c_int32), ("side", C.c_int32),
    ]


class Var(C.Structure):
    _fields_ = [("eb_user", C.c_double), ("eb", C.c_double), ("delta", C.c_double),
                ("step", C.c_double), ("norm2", C.c_double), ("K", C.c_int64)]


class Trace(C.Structure):
    _fields_ = [
        ("n", C.c_int32), ("side", C.c_int32), ("rcap", C.c_int32), ("r", C.c_int32),
        ("raw", C.c_int32), ("sweeps", C.c_int32), ("nprobes", C.c_int32), ("lin_r", C.c_int32),
        ("overflow", C.c_int32), ("wk", C.c_int32), ("ib", C.c_int32), ("dense", C.c_int32),
        ("L", C.c_int64), ("N", C.c_int64), ("n_corr", C.c_int64), ("n_esc", C.c_int64),
        ("nbytes", C.c_int64), ("el2", C.c_double), ("E", C.c_double * 33),
        ("probe_r", C.c_int32 * 8),
    ]


def _p(a, t):
    return a.ctypes.data_as(C.POINTER(t)) if a is not None else None


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(_SO)
            dp, ip, up = C.POINTER(C.c_double), C.POINTER(C.c_int32), C.POINTER(C.c_uint8)
            L.or_num_blocks.restype = C.c_int64
            L.or_num_blocks.argtypes = [C.POINTER(Params)]
            L.or_block_geom.argtypes = [C.POINTER(Params), C.c_int64, C.POINTER(Geom)]
            L.or_validate.argtypes = [C.POINTER(Params)]
            L.or_resolve.argtypes = [C.POINTER(Params), C.c_void_p, C.POINTER(Var)]
            L.or_gather.argtypes = [C.POINTER(Params), C.c_void_p, C.POINTER(Geom), dp]
            L.or_gram.argtypes = [dp, C.c_int64, C.c_int, dp]
            L.or_jacobi.argtypes = [dp, C.c_int, dp, dp]
            L.or_round_basis.argtypes = [dp, C.c_int, C.c_int, C.c_int, dp]
            L.or_project.argtypes = [dp, C.c_int64, C.c_int, dp, C.c_int, dp]
            L.or_quantize.argtypes = [dp, C.c_int64, C.c_double, C.c_int, ip]
            L.or_decode.argtypes = [ip, C.c_int64, C.c_int, C.c_int, dp, C.c_int, C.c_int, C.c_double, dp]
            L.or_block_err.restype = C.c_double
            L.or_block_err.argtypes = [dp, dp, C.c_int64, C.c_int]
            L.or_correct.argtypes = [dp, dp, C.c_int64, C.c_int, C.c_int, C.c_int64, C.c_int,
                                     C.c_double, C.c_double, ip, up]
            L.or_block_compress.restype = C.c_int64
            L.or_block_compress.argtypes = [C.POINTER(Params), C.c_void_p, C.c_int64, C.POINTER(Var),
                                            up, C.c_int64, C.POINTER(Trace), dp, dp, dp, dp, ip, ip, C.c_int]
            L.or_max_record_bytes.restype = C.c_int64
            L.or_max_record_bytes.argtypes = [C.POINTER(Params), C.c_int64]
            L.or_compress_bound.restype = C.c_int64
            L.or_compress_bound.argtypes = [C.POINTER(Params)]
            L.or_compress.argtypes = [C.POINTER(Params), C.c_void_p, C.c_void_p, C.c_int64,
                                      C.POINTER(C.c_int64), C.POINTER(Trace), C.c_int]
            L.or_decompress.argtypes = [C.c_void_p, C.c_int64, C.c_void_p, C.c_int64, C.c_int]
            i32p = C.POINTER(C.c_int32)
            u32p = C.POINTER(C.c_uint32)
            L.or_rice_bits.restype = C.c_int64
            L.or_rice_bits.argtypes = [i32p, C.c_int64, C.c_int, C.c_int, C.c_int]
            L.or_rice_choose.restype = None
            L.or_rice_choose.argtypes = [i32p, C.c_int64, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int)]
            L.or_rice_encode.restype = C.c_int64
            L.or_rice_encode.argtypes = [i32p, C.c_int64, C.c_int, C.c_int, C.c_int, u32p, C.c_int64, u32p]
            L.or_rice_decode.restype = C.c_int
            L.or_rice_decode.argtypes = [u32p, C.c_int64, u32p, C.c_int64, C.c_int, C.c_int, C.c_int, i32p]
            L.or_parse_record.restype = C.c_int
            L.or_parse_record.argtypes = [up, C.c_int64, C.c_int, C.c_int, C.c_int64, C.c_int64, C.c_int,
                                          C.POINTER(C.c_int), C.POINTER(C.c_int), dp, ip, ip, up, dp]
            L.or_project_f32.restype = None
            L.or_project_f32.argtypes = [dp, C.c_int64, C.c_int, dp, C.c_int, dp]
            L.or_pack_record.restype = C.c_int64
            L.or_pack_record.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int64, C.c_int64, C.c_int,
                                         dp, ip, ip, up, dp, up, C.c_int64, C.c_int]
            _lib = L
    return _lib


class Config:
    """Compression parameters, mirroring the paper's problem statement
    (snapshots, patch size, target error; Algorithm 1 inputs) plus block shape,
    bound type and rank cap."""

    def __init__(self, dims, block, dtype, eb, eb_type=EB_ABS, rank_cap=32, nvars=1,
                 block_begin=0, block_end=-1, basis=None, corr_codec=0, global_stats=None):
        self.dims = tuple(int(d) for d in dims)
        self.block = tuple(int(b) for b in block)
        self.dtype = int(dtype)
        self.eb = np.ascontiguousarray(np.broadcast_to(np.asarray(eb, dtype=np.float64), (nvars,)))
        self.eb_type = int(eb_type)
        self.rank_cap = int(rank_cap)
        self.nvars = int(nvars)
        self.block_begin = int(block_begin)
        self.block_end = int(block_end)
        # fixed basis (Sec. 4): n x n, column k = mode k, for blocks of Gram order n
        self.corr_codec = int(corr_codec)   # 1: Rice-coded corrections where smaller (proposed format)
        self.basis = None if basis is None else np.ascontiguousarray(basis, dtype=np.float64)
        if self.basis is not None and (self.basis.ndim != 2 or self.basis.shape[0] != self.basis.shape[1]):
            raise ValueError("basis must be a square matrix")
        # whole-field statistics (nvars x 4: min, max, sum of squares, points)
        # when the field passed is one part of it (Sec. 2.7.1 data distribution)
        self.global_stats = (None if global_stats is None else
                             np.ascontiguousarray(np.asarray(global_stats, dtype=np.float64).reshape(self.nvars, 4)))

    def c(self) -> Params:
        p = Params()
        p.nvars = self.nvars
        for a in range(4):
            p.dims[a] = self.dims[a]
            p.block[a] = self.block[a]
        p.dtype = self.dtype
        p.eb_type = self.eb_type
        p.eb = _p(self.eb, C.c_double)
        p.rank_cap = self.rank_cap
        p.block_begin = self.block_begin
        p.block_end = self.block_end
        if self.basis is not None:
            p.basis = _p(self.basis, C.c_double)
            p.basis_n = self.basis.shape[0]
        p.corr_codec = self.corr_codec
        if self.global_stats is not None:
            p.global_stats = _p(self.global_stats, C.c_double)
        return p


def _np_dtype(dt):
    return np.float32 if dt == F32 else np.float64


def num_blocks(cfg: Config) -> int:
    return lib().or_num_blocks(C.byref(cfg.c()))


def block_geom(cfg: Config, b: int) -> Geom:
    g = Geom()
    lib().or_block_geom(C.byref(cfg.c()), b, C.byref(g))
    return g


def validate(cfg: Config) -> int:
    return lib().or_validate(C.byref(cfg.c()))


def resolve(cfg: Config, field: np.ndarray):
    """Bound resolution per variable (Sec. 2.4, Eq. 4)."""
    f = np.ascontiguousarray(field, dtype=_np_dtype(cfg.dtype))
    vars_ = (Var * cfg.nvars)()
    st = lib().or_resolve(C.byref(cfg.c()), f.ctypes.data, vars_)
    return st, [vars_[i] for i in range(cfg.nvars)]


def gather(cfg: Config, field: np.ndarray, b: int) -> np.ndarray:
    f = np.ascontiguousarray(field, dtype=_np_dtype(cfg.dtype))
    g = block_geom(cfg, b)
    A = np.zeros((g.L, g.n), np.float64)
    lib().or_gather(C.byref(cfg.c()), f.ctypes.data, C.byref(g), _p(A, C.c_double))
    return A


def gram(A: np.ndarray) -> np.ndarray:
    """G = A^T A, sequential fma sums (cross-product SVD, Sec. 2.7.1)."""
    A = np.ascontiguousarray(A, np.float64)
    L, n = A.shape
    G = np.zeros((n, n), np.float64)
    lib().or_gram(_p(A, C.c_double), L, n, _p(G, C.c_double))
    return G


def jacobi(G: np.ndarray):
    """Eigenpairs of a symmetric G (<= 32x32): (lambda desc, V columns, sweeps)."""
    G = np.ascontiguousarray(G, np.float64)
    n = G.shape[0]
    lam = np.zeros(n, np.float64)
    V = np.zeros((n, n), np.float64)
    sw = lib().or_jacobi(_p(G, C.c_double), n, _p(lam, C.c_double), _p(V, C.c_double))
    return lam, V, sw


def round_basis(V: np.ndarray, r: int, dtype: int) -> np.ndarray:
    V = np.ascontiguousarray(V, np.float64)
    n = V.shape[0]
    Vst = np.zeros((n, r), np.float64)
    lib().or_round_basis(_p(V, C.c_double), n, r, dtype, _p(Vst, C.c_double))
    return Vst


def project(A: np.ndarray, Vst: np.ndarray) -> np.ndarray:
    """C = A Vst, sequential fma over the basis components (Sec. 2.5, Eq. 5)."""
    A = np.ascontiguousarray(A, np.float64)
    Vst = np.ascontiguousarray(Vst, np.float64)
    L, n = A.shape
    r = Vst.shape[1]
    Cm = np.zeros((L, r), np.float64)
    lib().or_project(_p(A, C.c_double), L, n, _p(Vst, C.c_double), r, _p(Cm, C.c_double))
    return Cm


def quantize(Cm: np.ndarray, delta: float, dtype: int):
    Cm = np.ascontiguousarray(Cm, np.float64)
    q = np.zeros(Cm.shape, np.int32)
    ovf = lib().or_quantize(_p(Cm, C.c_double), Cm.size, float(delta), dtype, _p(q, C.c_int32))
    return q, bool(ovf)


def decode(q: np.ndarray, r: int, Vst: np.ndarray, dtype: int, delta: float) -> np.ndarray:
    """Reconstruction with the first r modes (Sec. 2.6, Algorithm 2), fma chain in dtype."""
    q = np.ascontiguousarray(q, np.int32)
    Vst = np.ascontiguousarray(Vst, np.float64)
    L, rq = q.shape
    n = Vst.shape[0]
    assert Vst.shape[1] == rq
    D = np.zeros((L, n), np.float64)
    lib().or_decode(_p(q, C.c_int32), L, rq, r, _p(Vst, C.c_double), n, dtype, float(delta), _p(D, C.c_double))
    return D


def block_err(A: np.ndarray, D: np.ndarray) -> float:
    A = np.ascontiguousarray(A, np.float64)
    D = np.ascontiguousarray(D, np.float64)
    return lib().or_block_err(_p(A, C.c_double), _p(D, C.c_double), A.shape[0], A.shape[1])


def correct(A, D, side, M, dtype, eb, step):
    A = np.ascontiguousarray(A, np.float64)
    D = np.ascontiguousarray(D, np.float64)
    L, n = A.shape
    k = np.zeros(L * n, np.int32)
    esc = np.zeros(L * n, np.uint8)
    lib().or_correct(_p(A, C.c_double), _p(D, C.c_double), L, n, side, M, dtype, float(eb), float(step),
                     _p(k, C.c_int32), _p(esc, C.c_uint8))
    return k, esc


def pack_record(r, side, n, L, M, dtype, Vst, q, k, esc, A, corr_codec=0) -> bytes:
    Vst = np.ascontiguousarray(Vst, np.float64)
    q = np.ascontiguousarray(q, np.int32)
    k = np.ascontiguousarray(k, np.int32)
    esc = np.ascontiguousarray(esc, np.uint8)
    A = np.ascontiguousarray(A, np.float64)
    cap = 64 + 16 * L * n + 64 * n * n + 4096
    buf = np.zeros(cap, np.uint8)
    sz = lib().or_pack_record(r, side, n, L, M, dtype, _p(Vst, C.c_double), _p(q, C.c_int32),
                              _p(k, C.c_int32), _p(esc, C.c_uint8), _p(A, C.c_double),
                              _p(buf, C.c_uint8), cap, int(corr_codec))
    if sz < 0:
        raise RuntimeError(f"or_pack_record failed: {sz}")
    return buf[:sz].tobytes()


def parse_record(rec, side, n, L, M, dtype):
    """Inverse of pack_record for one record of the given block geometry
    (the record layout of Sec. 2.7.2).  Returns None for a record that does
    not follow the layout exactly, else a dict with r, flags, Vst (n x r),
    q (L x r), k and esc (element order) and escval (the raw values of
    escaped points; all values for a raw record)."""
    rec = np.ascontiguousarray(np.frombuffer(bytes(rec), np.uint8))
    N = L * n
    r, fl = C.c_int(0), C.c_int(0)
    Vst = np.zeros(n * n, np.float64)
    q = np.zeros(L * n, np.int32)
    k = np.zeros(N, np.int32)
    esc = np.zeros(N, np.uint8)
    ev = np.zeros(N, np.float64)
    st = lib().or_parse_record(_p(rec, C.c_uint8), rec.size, side, n, L, M, dtype, C.byref(r), C.byref(fl),
                               _p(Vst, C.c_double), _p(q, C.c_int32), _p(k, C.c_int32), _p(esc, C.c_uint8),
                               _p(ev, C.c_double))
    if st != OK:
        return None
    rr = r.value
    return dict(r=rr, flags=fl.value, Vst=Vst[: n * rr].reshape(n, rr), q=q[: L * rr].reshape(L, rr), k=k,
                esc=esc.astype(bool), escval=ev)


def project_f32(A: np.ndarray, Vst: np.ndarray) -> np.ndarray:
    """Coefficients as the FP32 form defines them (shifted binary32
    projection in a fixed order; Sec. 2.5 Eq. 5 evaluated in that precision)."""
    A = np.ascontiguousarray(A, np.float64)
    Vst = np.ascontiguousarray(Vst, np.float64)
    L, n = A.shape
    r = Vst.shape[1]
    Cm = np.zeros((L, max(r, 1)), np.float64)
    lib().or_project_f32(_p(A, C.c_double), L, n, _p(Vst, C.c_double), r, _p(Cm, C.c_double))
    return Cm[:, :r]


def block_compress(cfg: Config, field: np.ndarray, b: int, want_linear=False):
    """One block end to end with every intermediate (Algorithm 1 step 3)."""
    f = np.ascontiguousarray(field, dtype=_np_dtype(cfg.dtype))
    st, vars_ = resolve(cfg, f)
    if st != OK:
        raise RuntimeError(f"resolve failed: {st}")
    vv = (Var * cfg.nvars)(*vars_)
    g = block_geom(cfg, b)
    n, L = g.n, g.L
    rcap = min(cfg.rank_cap, n)
    cap = lib().or_max_record_bytes(C.byref(cfg.c()), b)
    rec = np.zeros(cap, np.uint8)
    tr = Trace()
    G = np.zeros((n, n)); lam = np.zeros(n); V = np.zeros((n, n)); Vst = np.zeros((n, max(rcap, 1)))
    q = np.zeros((L, max(rcap, 1)), np.int32)
    k = np.zeros(g.N, np.int32)
    sz = lib().or_block_compress(C.byref(cfg.c()), f.ctypes.data, b, vv, _p(rec, C.c_uint8), cap,
                                 C.byref(tr), _p(G, C.c_double), _p(lam, C.c_double), _p(V, C.c_double),
                                 _p(Vst, C.c_double), _p(q, C.c_int32), _p(k, C.c_int32),
                                 1 if want_linear else 0)
    if sz < 0:
        raise RuntimeError(f"or_block_compress failed: {sz}")
    return dict(record=rec[:sz].tobytes(), trace=tr, G=G, lam=lam, V=V, Vst=Vst[:, :rcap],
                q=q[:, :rcap], k=k, geom=g, var=vars_[g.v])


def compress_bound(cfg: Config) -> int:
    return lib().or_compress_bound(C.byref(cfg.c()))


def compress(cfg: Config, field: np.ndarray, traces: bool = False, nthreads: int = 0):
    """Whole-field compression; returns (status, stream bytes as np.uint8, traces)."""
    f = np.ascontiguousarray(field, dtype=_np_dtype(cfg.dtype))
    bound = compress_bound(cfg)
    if bound < 0:
        return ERR_INVALID_ARG, None, None
    out = np.zeros(bound, np.uint8)
    nb_total = num_blocks(cfg)
    e = nb_total if cfg.block_end < 0 else cfg.block_end
    nb = e - cfg.block_begin
    trs = (Trace * max(nb, 1))() if traces else None
    ob = C.c_int64(0)
    st = lib().or_compress(C.byref(cfg.c()), f.ctypes.data, out.ctypes.data, bound, C.byref(ob),
                           trs, nthreads)
    if st != OK:
        return st, None, None
    return st, out[: ob.value].copy(), ([trs[i] for i in range(nb)] if traces else None)


def decompress(stream: np.ndarray, nthreads: int = 0):
    """Returns (status, field array (nvars, nt, nz, ny, nx))."""
    s = np.ascontiguousarray(np.frombuffer(bytes(stream), np.uint8) if not isinstance(stream, np.ndarray) else stream,
                             np.uint8)
    if s.size < 128:
        return ERR_CORRUPT, None
    hdr = s[:128].tobytes()
    nvars = int.from_bytes(hdr[12:16], "little")
    dims = [int.from_bytes(hdr[16 + 8 * a: 24 + 8 * a], "little", signed=True) for a in range(4)]
    dtype = hdr[64]
    if nvars < 1 or nvars > 64 or dtype not in (0, 1) or min(dims) < 1 or np.prod(dims) * nvars > (1 << 34):
        return ERR_CORRUPT, None
    out = np.zeros((nvars, dims[3], dims[2], dims[1], dims[0]), _np_dtype(dtype))
    st = lib().or_decompress(s.ctypes.data, s.size, out.ctypes.data, out.nbytes, nthreads)
    return st, out


# ---------------------------------------------------------------- Rice-coded corrections
def rice_bits(k: np.ndarray, chunk: int, kr: int, wv: int) -> int:
    """Exact size in bits of the Rice-coded correction section (a proposed
    record section; see dls_oracle.c)."""
    k = np.ascontiguousarray(k, dtype=np.int32)
    return int(lib().or_rice_bits(_p(k, C.c_int32), k.size, chunk, kr, wv))


def rice_choose(k: np.ndarray, chunk: int):
    """(kr, wv) with the fewest bits."""
    k = np.ascontiguousarray(k, dtype=np.int32)
    kr, wv = C.c_int(0), C.c_int(0)
    lib().or_rice_choose(_p(k, C.c_int32), k.size, chunk, C.byref(kr), C.byref(wv))
    return kr.value, wv.value


def rice_encode(k: np.ndarray, chunk: int, kr: int, wv: int):
    """(words, chunk bit offsets, bits)."""
    k = np.ascontiguousarray(k, dtype=np.int32)
    nbits = rice_bits(k, chunk, kr, wv)
    words = np.zeros(max(1, (nbits + 31) // 32), np.uint32)
    off = np.zeros(max(1, -(-k.size // chunk)), np.uint32)
    got = lib().or_rice_encode(_p(k, C.c_int32), k.size, chunk, kr, wv, _p(words, C.c_uint32), words.size,
                               _p(off, C.c_uint32))
    if got < 0:
        raise RuntimeError("or_rice_encode: capacity")
    return words, off, int(got)


def rice_decode(words: np.ndarray, off: np.ndarray, N: int, chunk: int, kr: int, wv: int):
    """The corrections, or None for a malformed section."""
    words = np.ascontiguousarray(words, dtype=np.uint32)
    off = np.ascontiguousarray(off, dtype=np.uint32)
    k = np.zeros(max(1, N), np.int32)
    st = lib().or_rice_decode(_p(words, C.c_uint32), words.size, _p(off, C.c_uint32), N, chunk, kr, wv,
                              _p(k, C.c_int32))
    return None if st != 0 else k[:N]
