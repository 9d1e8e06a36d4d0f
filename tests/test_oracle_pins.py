"""Pins of the CPU oracle against what the paper and the mathematics fix.

None of these compare the oracle with itself: they use textbook results
(numpy/LAPACK SVD and eigh, Eckart-Young, Pythagoras), closed forms, brute
force on tiny inputs, invariants the paper states (full-basis exactness,
orthonormal bases, NRMSE below the target, pointwise bound) and a
hand-derived packed record.  Paper: arXiv 2601.20113.
"""
import os

import numpy as np
import pytest
import torch

import oracle
from paper_2601_20113_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _psd(n, seed, cond=1e8, rank=None):
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    lam = np.logspace(0, -np.log10(cond), n)
    if rank is not None:
        lam[rank:] = 0.0
    return (Q * lam) @ Q.T


# ---------------------------------------------------------------- Gram / eigensolve

@pytest.mark.parametrize("L,n", [(64, 16), (7, 3), (300, 32), (5, 1), (33, 17)])
def test_gram_is_AtA(L, n):
    """Cross-product matrix G = A^T A (Sec. 2.7.1): a transposed operand fails."""
    A = np.random.default_rng(L * 100 + n).standard_normal((L, n))
    G = oracle.gram(A)
    assert G.shape == (n, n)
    np.testing.assert_allclose(G, A.T @ A, rtol=1e-13, atol=1e-13 * np.abs(A.T @ A).max())


@pytest.mark.parametrize("n,seed,cond,rank", [(16, 1, 1e6, None), (32, 2, 1e12, None), (16, 3, 1e3, 5),
                                              (7, 4, 1e4, None), (2, 5, 10, None), (1, 6, 1, None),
                                              (31, 7, 1e10, 12)])
def test_jacobi_matches_lapack(n, seed, cond, rank):
    """Eigenvalues agree with LAPACK (eigh) within 1e-12 of lambda_max, the
    basis is orthonormal within 1e-12 (Sec. 2.3: SVD bases are orthonormal),
    G V = V Lambda, eigenvalues descending, and each column's largest
    component is positive."""
    G = _psd(n, seed, cond, rank)
    lam, V, sweeps = oracle.jacobi(G)
    w = np.linalg.eigh(G)[0][::-1]
    w = np.maximum(w, 0)
    scale = max(w[0], 1e-300)
    assert np.abs(lam - w).max() <= 1e-12 * scale
    assert np.abs(V.T @ V - np.eye(n)).max() <= 1e-12
    assert np.abs(G @ V - V * lam).max() <= 1e-12 * scale
    assert np.all(np.diff(lam) <= 0)
    for k in range(n):
        i = int(np.argmax(np.abs(V[:, k])))
        assert V[i, k] > 0
    assert (1 if n > 1 else 0) <= sweeps <= 30


def test_jacobi_is_svd_of_block():
    """Brute force on a tiny block: lambda_i = sigma_i^2 of A and the basis
    equals the right singular vectors (Eq. 2-3, Phi = V) up to sign."""
    rng = np.random.default_rng(11)
    A = rng.standard_normal((12, 5)) @ np.diag([5, 3, 2, 1, 0.5])
    lam, V, _ = oracle.jacobi(oracle.gram(A))
    U, s, Vt = np.linalg.svd(A, full_matrices=False)
    np.testing.assert_allclose(lam, s ** 2, rtol=1e-12)
    for k in range(5):
        v = Vt[k] * np.sign(Vt[k][np.argmax(np.abs(Vt[k]))])
        np.testing.assert_allclose(V[:, k], v, atol=1e-12)


def test_full_basis_is_exact():
    """Retaining every mode represents the block exactly before coefficient
    approximation (Sec. 2.3, no truncation; full-basis exactness)."""
    f = synth.vortex2d(nt=32).numpy()
    cfg = oracle.Config((64, 64, 1, 32), (8, 8, 1, 32), oracle.F64, eb=1e-3)
    for b in (0, 17, 63):
        A = oracle.gather(cfg, f, b)
        lam, V, _ = oracle.jacobi(oracle.gram(A))
        Cm = oracle.project(A, V)
        rec = Cm @ V.T
        assert np.linalg.norm(rec - A) <= 1e-12 * np.linalg.norm(A)


def test_known_rank_recovery():
    """A = P Q^T of rank k: eigenvalues beyond k vanish (Eckart-Young) and a
    tight tolerance selects exactly k modes."""
    for k in (1, 3, 6):
        A = synth.lowrank(200, 16, k, seed=k)
        lam, V, _ = oracle.jacobi(oracle.gram(A))
        assert lam[k - 1] > 1e-3 * lam[0]
        assert lam[k:].max(initial=0) <= 1e-13 * lam[0]
    f = synth.field_lowrank(16, 16, 8, 32, rank=3, seed=5)
    cfg = oracle.Config((16, 16, 8, 32), (8, 8, 4, 16), oracle.F64, eb=1e-6, rank_cap=16)
    st, s, trs = oracle.compress(cfg, f.numpy(), traces=True)
    assert st == 0
    assert all(t.r == 3 for t in trs)


def test_pythagoras_and_error_metric():
    """With an FP64 basis, e_r^2 = sum_{i>=r} lambda_i + ||C_r - Chat_r||^2
    (orthogonal projection, Pythagoras).  Pins projection, quantizer,
    dequantization, decode and the block error together."""
    rng = np.random.default_rng(3)
    A = rng.standard_normal((256, 16)) @ np.diag(np.logspace(0, -3, 16))
    lam, V, _ = oracle.jacobi(oracle.gram(A))
    delta = 1e-3
    Cm = oracle.project(A, V)
    q, ovf = oracle.quantize(Cm, delta, oracle.F64)
    assert not ovf
    for r in (0, 1, 4, 9, 16):
        D = oracle.decode(q, r, V, oracle.F64, delta)
        e2 = oracle.block_err(A, D)
        np.testing.assert_allclose(e2, np.sum((A - D) ** 2), rtol=1e-13)
        expect = lam[r:].sum() + np.sum((Cm[:, :r] - q[:, :r] * delta) ** 2)
        np.testing.assert_allclose(e2, expect, rtol=1e-10, atol=1e-14 * lam[0])


def test_decode_matches_matrix_product():
    """Reconstruction u = sum_s alpha_s phi_s (Sec. 2.6): f64 equals the matrix
    product to rounding; f32 is the fma chain in float (within a few ulp)."""
    rng = np.random.default_rng(4)
    q = rng.integers(-1000, 1000, size=(100, 6)).astype(np.int32)
    V = np.linalg.qr(rng.standard_normal((12, 12)))[0][:, :6]
    delta = 0.01
    D = oracle.decode(q, 6, V, oracle.F64, delta)
    np.testing.assert_allclose(D, (q * delta) @ V.T, rtol=1e-12, atol=1e-12)
    Vf = V.astype(np.float32).astype(np.float64)
    Df = oracle.decode(q, 6, Vf, oracle.F32, delta)
    ref = (q.astype(np.float32) * np.float32(delta)).astype(np.float64) @ Vf.T
    assert np.all(Df.astype(np.float32).astype(np.float64) == Df)
    np.testing.assert_allclose(Df, ref, rtol=1e-5, atol=1e-5)
    D3 = oracle.decode(q, 3, V, oracle.F64, delta)
    np.testing.assert_allclose(D3, (q[:, :3] * delta) @ V[:, :3].T, rtol=1e-12, atol=1e-12)


# ---------------------------------------------------------------- quantizer / correction

def test_quantizer_rounds_half_to_even_and_flags_overflow():
    Cm = np.array([0.5, 1.5, 2.5, -0.5, -1.5, 0.49999999999999994, 3.0, -7.2]) * 0.25
    q, ovf = oracle.quantize(Cm, 0.25, oracle.F64)
    assert q.tolist() == [0, 2, 2, 0, -2, 0, 3, -7]
    assert not ovf
    _, ovf = oracle.quantize(np.array([2.0 ** 24 * 0.1]), 0.1, oracle.F32)
    assert ovf
    q, ovf = oracle.quantize(np.array([(2.0 ** 24 - 1) * 0.1]), 0.1, oracle.F32)
    assert not ovf and q[0] == 2 ** 24 - 1


def test_correction_brute_force():
    """Pointwise correction on a tiny block, against the definition written
    out independently: k = rint((x - xhat)/(2eb)), xtilde = xhat + 2eb k."""
    rng = np.random.default_rng(8)
    A = rng.standard_normal((6, 3))
    D = A + rng.uniform(-0.5, 0.5, size=A.shape)
    eb = 0.05
    k, esc = oracle.correct(A, D, 0, 6, oracle.F64, eb, 2 * eb)
    for l in range(6):
        for j in range(3):
            e = j * 6 + l
            kk = np.rint((A[l, j] - D[l, j]) / (2 * eb))
            assert k[e] == kk and esc[e] == 0
            assert abs(A[l, j] - (D[l, j] + 2 * eb * kk)) <= eb * (1 + 1e-12)


# ---------------------------------------------------------------- rank search / tolerance

def test_bisection_equals_linear_scan_and_picks_smallest():
    """The retained set is the smallest prefix meeting eps_l (Sec. 2.5, Eq. 6,
    bisection of Algorithm 1).  Where pass(r) is monotone, bisection equals the
    linear scan."""
    f = synth.modes3d(32, 32, 16, 32, seed=9, count=16).numpy()
    rngv = float(f.max() - f.min())
    cfg = oracle.Config((32, 32, 16, 32), (16, 16, 8, 16), oracle.F32, eb=1e-3 * rngv, rank_cap=16)
    nb = oracle.num_blocks(cfg)
    agree = 0
    for b in range(nb):
        out = oracle.block_compress(cfg, f, b, want_linear=True)
        t = out["trace"]
        assert t.lin_r == t.r
        agree += 1
        if t.r > 0:
            assert t.E[t.r - 1] != t.E[t.r - 1] or t.E[t.r - 1] > t.el2   # probed r-1 failed if probed
    assert agree == nb


def test_local_tolerance_budget_sums_to_global():
    """eps_l^2 summed over the blocks of a variable equals eps^2 (Sec. 2.4,
    Eq. 4 with patch size = block points, coarsened elements = all points)."""
    f = synth.modes3d(24, 20, 12, 20, seed=3, count=8).numpy()
    cfg = oracle.Config((24, 20, 12, 20), (8, 8, 8, 8), oracle.F32, eb=0.5, eb_type=oracle.EB_NRMSE)
    st, s, trs = oracle.compress(cfg, f, traces=True)
    _, vars_ = oracle.resolve(cfg, f)
    eps = vars_[0].eb
    np.testing.assert_allclose(eps, 0.5 * np.sqrt(np.sum(f.astype(np.float64) ** 2)) / 100, rtol=1e-12)
    np.testing.assert_allclose(sum(t.el2 for t in trs), eps ** 2, rtol=1e-12)
    cfg2 = oracle.Config((24, 20, 12, 20), (8, 8, 8, 8), oracle.F32, eb=0.01)
    st, s, trs = oracle.compress(cfg2, f, traces=True)
    np.testing.assert_allclose(sum(t.el2 for t in trs), 0.01 ** 2 * f.size, rtol=1e-12)


@pytest.mark.parametrize("eps_t", [0.1, 1.0, 5.0])
def test_nrmse_mode_meets_global_target(eps_t):
    """Achieved NRMSE stays below the target (Sec. 4-5 report it; the local
    tolerance makes it a guarantee)."""
    f = synth.modes3d(32, 32, 16, 32, seed=12, count=24).numpy()
    cfg = oracle.Config((32, 32, 16, 32), (16, 16, 8, 16), oracle.F32, eb=eps_t, eb_type=oracle.EB_NRMSE)
    st, s, _ = oracle.compress(cfg, f)
    assert st == 0
    st, g = oracle.decompress(s)
    assert st == 0
    x = f.astype(np.float64)
    nrmse = 100 * np.linalg.norm(g - x) / np.linalg.norm(x)
    assert nrmse <= eps_t


@pytest.mark.parametrize("dtype,eb_type,ebv", [(oracle.F64, oracle.EB_ABS, 1e-3), (oracle.F32, oracle.EB_ABS, 1e-2),
                                              (oracle.F32, oracle.EB_REL_RANGE, 1e-4), (oracle.F64, oracle.EB_REL_RANGE, 1e-5)])
def test_pointwise_bound_everywhere(dtype, eb_type, ebv):
    """|x - xtilde| <= eb at every point (the pointwise guarantee)."""
    td = torch.float32 if dtype == oracle.F32 else torch.float64
    f = synth.modes3d(30, 22, 10, 20, seed=5, count=16, dtype=td).numpy()
    cfg = oracle.Config((30, 22, 10, 20), (8, 8, 4, 8), dtype, eb=ebv, eb_type=eb_type, rank_cap=8)
    st, s, trs = oracle.compress(cfg, f, traces=True)
    assert st == 0
    st, g = oracle.decompress(s)
    assert st == 0
    x = f.astype(np.float64)
    eb = ebv if eb_type == oracle.EB_ABS else ebv * (x.max() - x.min())
    assert np.abs(g.astype(np.float64) - x).max() <= eb
    assert s.size < f.nbytes


# ---------------------------------------------------------------- tiling / format

def test_block_tiling_covers_every_point_once():
    cfg = oracle.Config((13, 7, 5, 9), (4, 3, 2, 4), oracle.F32, eb=1.0, nvars=2)
    nb = oracle.num_blocks(cfg)
    assert nb == 2 * 4 * 3 * 3 * 3
    cover = np.zeros((2, 9, 5, 7, 13), np.int32)
    for b in range(nb):
        g = oracle.block_geom(cfg, b)
        cover[g.v, g.t0:g.t0 + g.st, g.z0:g.z0 + g.sz, g.y0:g.y0 + g.sy, g.x0:g.x0 + g.sx] += 1
        assert g.N == g.sx * g.sy * g.sz * g.st
        assert g.n == min(g.M, g.T) and (g.side == 0) == (g.T <= g.M)
    assert np.all(cover == 1)


def test_gather_layout():
    """Block matrix rows are spatial points (x fastest), columns timesteps; the
    spatial side transposes."""
    f = np.arange(2 * 5 * 4 * 3 * 6, dtype=np.float64).reshape(2, 5, 4, 3, 6)  # (v,t,z,y,x)
    cfg = oracle.Config((6, 3, 4, 5), (2, 3, 2, 5), oracle.F64, eb=1.0, nvars=2)
    g = oracle.block_geom(cfg, 7)
    A = oracle.gather(cfg, f, 7)
    blk = f[g.v, g.t0:g.t0 + g.st, g.z0:g.z0 + g.sz, g.y0:g.y0 + g.sy, g.x0:g.x0 + g.sx]
    X = blk.reshape(g.st, -1).T      # (M, T)
    assert g.side == 0
    np.testing.assert_array_equal(A, X)
    cfg2 = oracle.Config((6, 3, 4, 5), (1, 1, 2, 5), oracle.F64, eb=1.0, nvars=2)
    g2 = oracle.block_geom(cfg2, 3)
    A2 = oracle.gather(cfg2, f, 3)
    blk2 = f[g2.v, g2.t0:g2.t0 + g2.st, g2.z0:g2.z0 + g2.sz, g2.y0:g2.y0 + g2.sy, g2.x0:g2.x0 + g2.sx]
    assert g2.side == 1
    np.testing.assert_array_equal(A2, blk2.reshape(g2.st, -1))


def _golden_record():
    d = {"bytes": []}
    with open(os.path.join(GOLDEN, "record_2x2x2x2.txt")) as fh:
        for line in fh:
            if not line.strip() or line.startswith("#"):
                continue
            key, *vals = line.split()
            if key == "bytes":
                d["bytes"] += [int(v, 16) for v in vals]
            else:
                d[key] = vals
    return d


def test_packed_record_matches_hand_derived_golden():
    g = _golden_record()
    L, n, M = int(g["L"][0]), int(g["n"][0]), int(g["M"][0])
    q = np.array([int(v) for v in g["q"]], np.int32).reshape(L, 1)
    k = np.array([int(v) for v in g["k"]], np.int32)
    esc = np.zeros(L * n, np.uint8)
    esc[int(g["esc"][0])] = 1
    Vst = np.array([float(np.float32(v)) for v in g["vst"]]).reshape(n, 1)
    A = np.zeros((L, n))
    A[7, 0] = float(g["a7"][0])
    rec = oracle.pack_record(1, 0, n, L, M, oracle.F32, Vst, q, k, esc, A)
    assert list(rec) == g["bytes"]


def test_stream_header_and_corruption():
    """Addressable header + offset table (Sec. 2.7.2); corrupt or truncated
    streams are rejected."""
    f = synth.vortex2d(32, 32, 16, seed=2).numpy()
    cfg = oracle.Config((32, 32, 1, 16), (8, 8, 1, 16), oracle.F64, eb=1e-3, rank_cap=8)
    st, s, trs = oracle.compress(cfg, f, traces=True)
    b = s.tobytes()
    assert b[:4] == b"DLS1"
    nb = oracle.num_blocks(cfg)
    offp = int.from_bytes(b[104:112], "little")
    payp = int.from_bytes(b[112:120], "little")
    assert int.from_bytes(b[120:128], "little") == len(b)
    offs = np.frombuffer(b[offp:offp + 8 * (nb + 1)], np.uint64)
    assert offs[0] == 0 and np.all(np.diff(offs.astype(np.int64)) == [t.nbytes for t in trs])
    assert payp + int(offs[-1]) == len(b)
    assert oracle.decompress(s[:-16])[0] == oracle.ERR_CORRUPT
    bad = s.copy(); bad[0] ^= 1
    assert oracle.decompress(bad)[0] == oracle.ERR_CORRUPT
    bad = s.copy(); bad[offp + 8] ^= 0x10
    assert oracle.decompress(bad)[0] == oracle.ERR_CORRUPT


def test_invalid_and_nonfinite_inputs():
    f = np.zeros((1, 8, 1, 8, 8))
    assert oracle.validate(oracle.Config((8, 8, 1, 8), (4, 4, 1, 8), oracle.F64, eb=0.0)) == oracle.ERR_INVALID_ARG
    assert oracle.validate(oracle.Config((8, 8, 1, 8), (4, 4, 1, 8), oracle.F64, eb=1.0, rank_cap=-1)) == oracle.ERR_INVALID_ARG
    assert oracle.validate(oracle.Config((8, 8, 1, 8), (16, 4, 1, 8), oracle.F64, eb=1.0)) == oracle.ERR_INVALID_ARG
    assert oracle.validate(oracle.Config((64, 64, 1, 64), (64, 64, 1, 64), oracle.F64, eb=1.0)) == oracle.ERR_INVALID_ARG
    f[0, 3, 0, 2, 2] = np.nan
    st, _, _ = oracle.compress(oracle.Config((8, 8, 1, 8), (4, 4, 1, 8), oracle.F64, eb=1.0), f)
    assert st == oracle.ERR_NONFINITE


def test_degenerate_blocks():
    """Zero field -> rank 0, no corrections; rank cap 0 -> corrections only;
    T = 1 and M = 1 blocks; a block larger than its edge remainder."""
    z = np.zeros((1, 4, 3, 5, 7), np.float32)
    cfg = oracle.Config((7, 5, 3, 4), (4, 4, 2, 4), oracle.F32, eb=1e-3)
    st, s, trs = oracle.compress(cfg, z, traces=True)
    assert st == 0 and all(t.r == 0 and t.n_corr == 0 and not t.raw for t in trs)
    assert np.all(oracle.decompress(s)[1] == 0)
    f = synth.modes3d(7, 5, 3, 4, seed=1, count=4).numpy()
    for block, cap in (((4, 4, 2, 4), 0), ((1, 1, 1, 4), 4), ((7, 5, 3, 1), 4), ((3, 2, 1, 4), 3)):
        cfg = oracle.Config((7, 5, 3, 4), block, oracle.F32, eb=1e-2, rank_cap=cap)
        st, s, trs = oracle.compress(cfg, f, traces=True)
        assert st == 0
        g = oracle.decompress(s)[1]
        assert np.abs(g.astype(np.float64) - f).max() <= 1e-2
        if cap == 0:
            assert all(t.r == 0 for t in trs)
