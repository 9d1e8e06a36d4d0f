"""Pins of the global-basis oracle (the global-basis mode: one basis per
variable from random patches of the first snapshot; per patch, the smallest
magnitude-ordered prefix of its coefficients meeting the local tolerance).

The pins use facts fixed outside the oracle: a fixed quadratic form plus
varying linear parts puts every window in the 5-dimensional span of
{1, x, y, z, the form}; for an orthonormal basis the best n-term subset is the
n largest coefficients (checked by brute force with least squares); bisection
on a monotone error equals the linear scan; meeting every local tolerance
meets the global NRMSE target."""
import itertools

import numpy as np
import pytest

from oracle import global_basis as gb
from paper_2601_20113_gb300 import synth


_QC = (0.02, -0.03, 0.015, 0.01, -0.02, 0.025)   # xx, yy, zz, xy, xz, yz


def _quad(x, y, z):
    a, b, c, d, e, f = _QC
    return a * x * x + b * y * y + c * z * z + d * x * y + e * x * z + f * y * z


def _quadratic_field(nt, n, seed):
    """(nt, n, n, n): snapshot t = a_t + b_t x + c_t y + d_t z + Q(x, y, z), one
    fixed quadratic form Q, random linear parts.  Any m^3 window of any
    snapshot, in local coordinates, lies in span{1, x, y, z, Q}: the window's
    quadratic part is Q itself, its linear and constant parts vary."""
    rng = np.random.default_rng(seed)
    z, y, x = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    out = np.empty((nt, n, n, n))
    for t in range(nt):
        a, b, c, d = rng.standard_normal(4) * [5.0, 1.0, 1.0, 1.0]
        out[t] = a + b * x + c * y + d * z + _quad(x, y, z)
    return out


def _window_span(m):
    """Orthonormal basis (numpy QR) of {1, x, y, z, Q} on an m^3 patch, x fastest."""
    z, y, x = np.meshgrid(np.arange(m), np.arange(m), np.arange(m), indexing="ij")
    A = np.stack([np.ones(m ** 3), x.ravel(), y.ravel(), z.ravel(), _quad(x, y, z).ravel()], axis=1)
    return np.linalg.qr(A.astype(np.float64))[0]


def test_learned_modes_lead_with_the_span_of_the_data():
    m, n = 4, 16
    f = _quadratic_field(6, n, seed=1)
    origins = synth.patch_origins((n, n, n), (m, m, m), 4 * m ** 3, seed=2)
    phi, sv = gb.learn_basis(f[0], origins, (m, m, m))
    np.testing.assert_allclose(phi.T @ phi, np.eye(m ** 3), atol=1e-12)
    B = _window_span(m)
    assert abs(np.sum((B.T @ phi[:, :5]) ** 2) - 5.0) < 1e-9        # the first 5 modes span the windows
    assert sv[4] > 1e-8 * sv[0] and sv[5] <= 1e-10 * sv[0]
    assert np.all(np.diff(sv) <= 1e-9 * sv[0])
    for k in range(m ** 3):                                          # sign rule
        col = phi[:, k]
        assert col[int(np.argmax(np.abs(col)))] > 0
    res = gb.compress(f, m, 0.1, origins)
    assert max(len(r[2]) for r in res["recs"]) <= 5                 # every snapshot's patches: <= 5 modes


def test_magnitude_prefix_is_the_best_subset():
    """For an orthonormal basis the n largest coefficients give the smallest
    n-term error: brute force over all subsets with least squares."""
    M = 8
    rng = np.random.default_rng(3)
    phi = np.linalg.qr(rng.standard_normal((M, M)))[0]
    for trial in range(5):
        u = rng.standard_normal(M) * np.logspace(0, -3, M)[rng.permutation(M)]
        best = np.zeros(M + 1)
        for n in range(M + 1):
            e = np.inf
            for A in itertools.combinations(range(M), n):
                if n == 0:
                    r = u
                else:
                    c = np.linalg.lstsq(phi[:, A], u, rcond=None)[0]
                    r = u - phi[:, A] @ c
                e = min(e, float(r @ r))
            best[n] = e
        for tol in (best[2] * 1.000001, best[5] * 1.000001, best[M - 1] * 1.000001):
            idx, q, e2 = gb.compress_patch(u, phi, tol, 1e-12)
            n_star = int(np.argmax(best <= tol))                    # smallest n with some subset meeting tol
            assert len(idx) == n_star
            np.testing.assert_allclose(e2, best[n_star], rtol=1e-6, atol=1e-18)


def test_bisection_equals_the_linear_scan():
    rng = np.random.default_rng(4)
    M = 27
    phi = np.linalg.qr(rng.standard_normal((M, M)))[0]
    for _ in range(20):
        u = rng.standard_normal(M) * np.logspace(0, -4, M)[rng.permutation(M)]
        tol = float(u @ u) * 10 ** rng.uniform(-6, -1)
        idx, _, _ = gb.compress_patch(u, phi, tol, 1e-13)
        alpha = np.linalg.solve(phi, u)                             # coefficients without Phi^T
        tail = np.sort(alpha ** 2)                                  # ascending: energy left after n terms
        left = [float(np.sum(tail[:M - n])) for n in range(M + 1)]
        assert len(idx) == next(n for n in range(M + 1) if left[n] <= tol)


@pytest.mark.parametrize("eps_t", [0.1, 1.0, 5.0])
def test_global_nrmse_meets_the_target(eps_t):
    f = synth.modes3d(16, 16, 16, 8, seed=5, count=24).numpy()[0].astype(np.float64)   # (nt, nz, ny, nx)
    m = 4
    origins = synth.patch_origins((16, 16, 16), (m, m, m), 4 * m ** 3, seed=6)
    res = gb.compress(f, m, eps_t, origins)
    rec = gb.decompress(res)
    nrmse = 100.0 * np.linalg.norm(rec - f) / np.linalg.norm(f)
    assert nrmse <= eps_t
    for t, (x0, y0, z0), idx, q, e2 in res["recs"]:
        u = f[t, z0:z0 + m, y0:y0 + m, x0:x0 + m].ravel()
        d = u - rec[t, z0:z0 + m, y0:y0 + m, x0:x0 + m].ravel()
        assert e2 <= res["eps_l2"] and abs(float(d @ d) - e2) <= 1e-9 * max(e2, res["eps_l2"])
        assert len(set(idx.tolist())) == len(idx)
    dofs = sum(len(r[2]) for r in res["recs"])
    assert 0 < dofs < f.size                                        # fewer DOFs than values


def test_two_dimensional_patches_and_zero_field():
    f = np.zeros((3, 1, 8, 8))
    origins = synth.patch_origins((8, 8, 1), (4, 4, 1), 64, seed=7)
    res = gb.compress(f, 4, 1.0, origins)
    assert res["patch"] == (4, 4, 1) and res["phi"].shape == (16, 16)
    assert all(len(r[2]) == 0 for r in res["recs"])
    assert np.array_equal(gb.decompress(res), f)


def test_tiling_rule_and_origins():
    with pytest.raises(ValueError):
        gb.compress(np.zeros((2, 6, 6, 6)), 4, 1.0, np.zeros((4, 3), np.int64))
    o1 = synth.patch_origins((20, 12, 9), (4, 4, 4), 500, seed=8)
    o2 = synth.patch_origins((20, 12, 9), (4, 4, 4), 500, seed=8)
    assert np.array_equal(o1, o2) and o1.min() >= 0
    assert o1[:, 0].max() <= 16 and o1[:, 1].max() <= 8 and o1[:, 2].max() <= 5


def _small_result(eps_t=1.0):
    f = synth.modes3d(16, 16, 16, 8, seed=5, count=24).numpy()[0].astype(np.float64)
    origins = synth.patch_origins((16, 16, 16), (4, 4, 4), 256, seed=6)
    return f, gb.compress(f, 4, eps_t, origins)


def test_stream_round_trip_and_size():
    """pack/unpack keep every record's kept modes and values; the size is the
    header, the basis, the offsets and the records as laid out."""
    f, res = _small_result()
    s = gb.pack(res)
    back = gb.unpack(s)
    assert back is not None and len(back["recs"]) == len(res["recs"])
    for a, b in zip(res["recs"], back["recs"]):
        assert a[0] == b[0] and a[1] == b[1]
        assert np.array_equal(a[2], b[2]) and np.array_equal(a[3], b[3])
    assert np.array_equal(gb.decompress(back), gb.decompress(res))
    M = res["phi"].shape[0]
    ib = (M - 1).bit_length()
    size = 80 + 8 * M * M + 8 * (len(res["recs"]) + 1)
    for _, _, idx, q, _ in res["recs"]:
        wv = max((int(abs(2 * v) - (v < 0)) for v in q), default=0).bit_length()
        body = 8 + 4 * ((len(idx) * (ib + wv) + 31) // 32)
        size += body + (-body) % 8
    assert len(s) == size


def test_malformed_streams_are_rejected():
    _, res = _small_result()
    s = gb.pack(res)
    assert gb.unpack(s[:100]) is None                      # truncated
    assert gb.unpack(b"XXXX" + s[4:]) is None              # magic
    bad = bytearray(s)
    at = 80 + 8 * 64 * 64 + 8                              # second offset
    bad[at:at + 8] = np.uint64(3).tobytes()                # a record shorter than its header
    assert gb.unpack(bytes(bad)) is None
