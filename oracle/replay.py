"""Replay of a compressed stream through the oracle's steps (TEST INFRASTRUCTURE).

Only ``tests/`` and ``__graft_entry__.smoke()`` use this module.  It shares no
code with the CUDA library: it parses a stream with the oracle's record parser
and recomputes, with the oracle's functions, everything a record holds from the
block's data and the record's own stored modes.

A block's stored modes V^st are the one part of a record that the FP32
(mixed-precision) form computes differently from the FP64 oracle: its Gram
matrix is summed in binary32 (Sec. 2.7.1 cross-product SVD), so its
eigenvectors, rounded to the field dtype (the stored basis of Sec. 2.3), can
differ from the oracle's in the last bits.  Given V^st, every further step is a
definition the oracle evaluates exactly:

  1. coefficients (Sec. 2.5 Eq. 5): the FP32 form's shifted binary32
     projection (``project_f32``), quantized with FP64 semantics
     (``quantize``): the codes must be equal, code for code.  Independently of
     that definition, every code must be a correct rounding of the FP64
     projection within the binary32 evaluation error bound;
  2. rank (Sec. 2.5 Eq. 6, Algorithm 1 bisection): with E(r) in the fixed FP64
     order, r == rank cap or pass(r), and r == 0 or not pass(r - 1) -- the
     property every bisection result and every accepted prediction has;
  3. reconstruction (Sec. 2.6, Algorithm 2): the decode contract in binary32;
  4. pointwise corrections and escapes: equal, element for element;
  5. the record (Sec. 2.7.2 layout): the oracle's packer given (r, V^st, q, k,
     escapes, the block's raw values) and the configuration's correction codec
     (Rice-coded sections where smaller, when asked) must write the same bytes.

The stored modes themselves are checked against the oracle's FP64 eigenproblem
of the same block: orthonormal to binary32 rounding, and their Rayleigh
quotients on the FP64 Gram matrix within the perturbation bound of a
binary32-summed Gram matrix of the eigenvalues the oracle's Jacobi solver finds.
"""
from __future__ import annotations

import numpy as np

from . import (F32, F64, EB_NRMSE, Config, block_err, block_geom, correct, decode, gather, gram, jacobi,
               pack_record, parse_record, project, project_f32, quantize)

U32 = 2.0 ** -24                 # unit roundoff of binary32


def parse_stream(stream):
    """Header, per-variable table and offset table of a stream (Sec. 2.7.2)."""
    s = np.ascontiguousarray(np.frombuffer(bytes(stream), np.uint8) if not isinstance(stream, np.ndarray)
                             else stream, np.uint8)
    u32 = lambda o: int(s[o:o + 4].view(np.uint32)[0])
    i64 = lambda o: int(s[o:o + 8].view(np.int64)[0])
    h = dict(magic=u32(0), version=u32(4), nvars=u32(12), dims=tuple(i64(16 + 8 * a) for a in range(4)),
             block=tuple(u32(48 + 4 * a) for a in range(4)), dtype=int(s[64]), eb_type=int(s[65]),
             precision=int(s[66]), rank_mode=int(s[67]), rank_cap=u32(68), block_begin=i64(72),
             block_end=i64(80), total_blocks=i64(88), offp=i64(104), payp=i64(112), total=i64(120))
    vt = s[128:128 + 32 * h["nvars"]].view(np.float64).reshape(h["nvars"], 4)
    h["eb_user"], h["eb"], h["delta"], h["step"] = (vt[:, i].copy() for i in range(4))
    nb = h["block_end"] - h["block_begin"]
    h["offsets"] = s[h["offp"]:h["offp"] + 8 * (nb + 1)].view(np.uint64).astype(np.int64)
    return s, h


def record_of(s, h, i):
    o0, o1 = int(h["offsets"][i]), int(h["offsets"][i + 1])
    return s[h["payp"] + o0:h["payp"] + o1]


def check_modes(A, Vst, u_prod=0.0):
    """Orthonormality of the stored modes and their Rayleigh quotients on the
    block's FP64 Gram matrix against the oracle's eigenvalues.  u_prod: the
    relative error of each Gram product's operands (0 for binary32 operands;
    2^-21, 2^-11, 2^-16, 2^-9 for the 3xTF32, TF32, BF16x3 and BF16 tensor-core
    Grams).  Returns (orthonormality error, worst eigenvalue error / bound)."""
    L, n = A.shape
    r = Vst.shape[1]
    if r == 0:
        return 0.0, 0.0
    G = gram(A)
    lam, _, _ = jacobi(G)
    orth = float(np.abs(Vst.T @ Vst - np.eye(r)).max())
    # A binary32 Gram summed along chains of at most L + 32 terms is G + dG with
    # |dG_ij| <= gamma sqrt(G_ii G_jj), gamma = (L + 32) u (+ 2 u_prod when the
    # products' operands carry a relative error u_prod): ||dG||_2 <= gamma
    # trace(G).  An exact eigenvector v of G + dG then has
    # |v^T G v - lambda_k| <= 2 ||dG||_2 (Weyl), and rounding v to binary32
    # moves the quotient by at most 4 n u lambda_0 more.
    gamma = (L + 32) * U32 + 2.0 * u_prod
    bound = 2.0 * gamma * float(np.trace(G)) + 4.0 * n * U32 * float(lam[0]) + 1e-300
    rq = np.einsum("jk,ji,ik->k", Vst, G, Vst)
    return orth, float(np.abs(rq - lam[:r]).max() / bound)


def replay_block(cfg: Config, field, b: int, rec, eb: float, delta: float, step: float, coeff: str = "f32",
                 u_prod: float = 0.0):
    """Checks one record; returns a dict of findings (empty 'errors' when
    everything holds).  coeff: 'f32' (the FP32 form's coefficient definition,
    codes compared exactly) or 'f64' (the oracle's own FP64 projection)."""
    g = block_geom(cfg, b)
    n, L, M, N = g.n, g.L, g.M, g.N
    out = dict(block=b, errors=[], raw=False, r=0, dense=False, sparse=False, nesc=0)
    p = parse_record(rec, g.side, n, L, M, cfg.dtype)
    if p is None:
        out["errors"].append("record does not parse")
        return out
    A = gather(cfg, field, b)
    el = A.reshape(L, n)
    xe = (el.T.reshape(-1) if g.side == 0 else el.reshape(-1))     # element order e = t M + s
    if p["flags"] & 1:
        out["raw"] = True
        if not np.array_equal(p["escval"], xe):
            out["errors"].append("raw record values differ from the block")
        return out
    r, Vst, q = p["r"], p["Vst"], p["q"]
    out["r"] = r
    rcap = min(cfg.rank_cap, n)
    # 1. codes
    Cm = project_f32(A, Vst) if coeff == "f32" else project(A, Vst)
    qo, ovf = quantize(Cm, delta, cfg.dtype)
    if ovf or not np.array_equal(qo, q):
        out["errors"].append(f"codes differ in {int(np.count_nonzero(qo != q))} of {q.size}")
    C64 = project(A, Vst)
    d = np.abs(A - A[:, :1])
    tol = 2 * (n + 3) * U32 * (d @ np.abs(Vst) + np.abs(A[:, :1]) * np.abs(Vst).sum(0)[None, :])
    if cfg.dtype == F64:
        tol = tol * 0.0 + 1e-12 * (np.abs(A) @ np.abs(Vst))
    if np.any(np.abs(q * delta - C64) > delta / 2 + tol + 1e-12 * delta):
        out["errors"].append("a code is not a rounding of the FP64 projection within the evaluation bound")
    # 2. rank
    # local tolerance (Sec. 2.4 Eq. 4): eb^2 N pointwise, eps^2 N / K for NRMSE
    el2 = eb * eb * N / float(np.prod(cfg.dims)) if cfg.eb_type == EB_NRMSE else eb * eb * N
    D = decode(q, r, Vst, cfg.dtype, delta)
    E_r = block_err(A, D)
    if not (r == rcap or E_r <= el2):
        out["errors"].append(f"pass(r) fails at r = {r}")
    if r > 0:
        Dm = decode(q[:, :r - 1], r - 1, Vst[:, :r - 1], cfg.dtype, delta)
        if block_err(A, Dm) <= el2:
            out["errors"].append(f"pass(r - 1) holds at r = {r}")
    # 4. corrections
    if cfg.eb_type == EB_NRMSE:
        k = np.zeros(N, np.int32)
        esc = np.zeros(N, np.uint8)
    else:
        k, esc = correct(A, D, g.side, M, cfg.dtype, eb, step)
    if not np.array_equal(k, p["k"]):
        out["errors"].append(f"corrections differ in {int(np.count_nonzero(k != p['k']))} elements")
    if not np.array_equal(esc.astype(bool), p["esc"]):
        out["errors"].append("escape sets differ")
    if np.any(p["esc"]) and not np.array_equal(p["escval"][p["esc"]], xe[p["esc"]]):
        out["errors"].append("escaped values are not the raw values")
    out["nesc"] = int(p["esc"].sum())
    out["dense"] = bool(p["flags"] & 4)
    out["sparse"] = (not out["dense"]) and bool(np.any(p["k"] != 0))
    # 5. the record, repacked by the oracle
    rec_o = pack_record(r, g.side, n, L, M, cfg.dtype, Vst, q, k, esc, A, cfg.corr_codec)
    if rec_o != bytes(rec):
        out["errors"].append("record bytes differ from the oracle packer's")
    # the stored modes against the oracle's eigenproblem
    orth, lam_err = check_modes(A, Vst, u_prod)
    out["orth"], out["lam_err"] = orth, lam_err
    # modes orthonormal in exact arithmetic, each component rounded once to the
    # dtype (relative error u): |v_i^T v_j - delta_ij| <= 2u + u^2 by
    # Cauchy-Schwarz; 4u leaves room for an FP64 residual far below u
    # (float64 modes: the 1e-12 of the FP64 eigensolver's own pin)
    if orth > (4 * U32 if cfg.dtype == F32 else 1e-12):
        out["errors"].append(f"stored modes not orthonormal: {orth:.3e}")
    if lam_err > 1.0:
        out["errors"].append(f"Rayleigh quotient off by {lam_err:.3f} x its bound")
    return out


def replay_stream(cfg: Config, field, stream, blocks=None, coeff: str = "f32", u_prod: float = 0.0):
    """Replays the records of `blocks` (all by default).  Returns (findings,
    stream-level errors)."""
    s, h = parse_stream(stream)
    errs = []
    if h["total"] != s.size:
        errs.append("stream size differs from the header's")
    sizes = np.diff(h["offsets"])
    if h["offsets"][0] != 0 or np.any(sizes <= 0) or np.any(sizes % 16):
        errs.append("offset table is not an exclusive scan of 16-byte aligned record sizes")
    nb = len(sizes)
    idx = range(nb) if blocks is None else blocks
    out = []
    for i in idx:
        rec = record_of(s, h, i)
        if int(rec[12:16].view(np.uint32)[0]) != sizes[i]:
            errs.append(f"record {i}: size field differs from the offset table")
        b = h["block_begin"] + i
        v = block_geom(cfg, b).v
        out.append(replay_block(cfg, field, b, rec, float(h["eb"][v]), float(h["delta"][v]), float(h["step"][v]),
                                coeff, u_prod))
    return out, errs
