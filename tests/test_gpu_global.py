"""The global-basis mode on the GPU (dls_gb_compress / dls_gb_decompress)
against the oracle's global-basis mode (oracle/global_basis.py).

The basis is the one part the GPU computes differently (eigenvectors of the
FP64 Gram matrix by Jacobi, against the oracle's SVD of the sample matrix), so
it is checked against the oracle's: orthonormal to 1e-12, the sign rule, and
its Rayleigh quotients on Q^T Q equal to the oracle's squared singular values
within the Gram matrix's rounding.  Given the stream's basis and tolerance,
every record must be the one the oracle's per-patch step writes (kept modes in
kept order, their values), the tolerance must be the oracle's, and the GPU
decoder must rebuild the oracle decoder's field bit for bit.
"""
import numpy as np
import pytest
import torch

from oracle import global_basis as gb
from paper_2601_20113_gb300 import dls, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2601_20113_gb300 import build
    build.build()


def _run(f32, m, eps_t, seed=6):
    nt, nz, ny, nx = f32.shape
    patch = gb.patch_shape((nx, ny, nz, nt), m)
    origins = synth.patch_origins((nx, ny, nz), patch, 4 * int(np.prod(patch)), seed=seed)
    comp = dls.gb_compress(torch.from_numpy(np.ascontiguousarray(f32)).cuda(), m, eps_t, origins)
    return comp, origins, patch


def _check(f32, m, eps_t, seed=6):
    comp, origins, patch = _run(f32, m, eps_t, seed)
    f = f32.astype(np.float64)
    s = comp.cpu().numpy().tobytes()
    res = gb.unpack(s)
    assert res is not None and res["patch"] == patch
    phi = res["phi"]
    M = phi.shape[0]
    # the basis against the oracle's SVD
    assert np.abs(phi.T @ phi - np.eye(M)).max() <= 1e-12
    for k in range(M):
        col = phi[:, k]
        assert col[int(np.argmax(np.abs(col)))] > 0
    _, sv = gb.learn_basis(f[0], origins, patch)
    Q = np.stack([gb.gather_patch(f[0], o, patch) for o in origins])
    G = Q.T @ Q
    rq = np.einsum("ik,ij,jk->k", phi, G, phi)
    assert np.abs(rq - sv ** 2).max() <= 1e-12 * M * max(float(sv[0]) ** 2, 1e-300)
    # the tolerance
    el2, delta = gb.local_tolerance(f, eps_t, M)
    assert abs(res["eps_l2"] - el2) <= 1e-13 * el2 and abs(res["delta"] - delta) <= 1e-13 * delta
    # every record, through the oracle's per-patch step with the stream's basis
    bad = []
    for t, (x0, y0, z0), idx, q, _ in res["recs"]:
        u = gb.gather_patch(f[t], (x0, y0, z0), patch)
        io, qo, _ = gb.compress_patch(u, phi, res["eps_l2"], res["delta"])
        if not (np.array_equal(io, idx) and np.array_equal(qo, q)):
            bad.append((t, (x0, y0, z0), len(io), len(idx)))
    assert not bad, bad[:5]
    # the stream is the oracle's packing of those records
    assert gb.pack(res) == s
    # the decoder
    rec = dls.gb_decompress(comp).cpu().numpy()
    ref = gb.decompress(res)
    assert np.array_equal(rec, ref)
    nrmse = 100.0 * np.linalg.norm(rec - f) / np.linalg.norm(f)
    assert nrmse <= eps_t
    return res


@pytest.mark.parametrize("eps_t", [0.1, 1.0, 5.0])
def test_modes3d_patches_of_4(eps_t):
    f = synth.modes3d(16, 16, 16, 8, seed=5, count=24).numpy()[0]
    res = _check(f, 4, eps_t)
    assert 0 < sum(len(r[2]) for r in res["recs"]) < f.size


def test_patches_of_5_the_papers_smallest():
    """m = 5: M = 125 modes (odd order: the Jacobi pads to 126)."""
    f = synth.modes3d(20, 20, 20, 4, seed=7, count=24).numpy()[0]
    _check(f, 5, 1.0, seed=8)


def test_two_dimensional_patches():
    f = synth.modes3d(32, 32, 1, 6, seed=9, count=16).numpy()[0]
    res = _check(f, 8, 0.5, seed=10)
    assert res["patch"] == (8, 8, 1)


def test_quadratic_field_keeps_at_most_five_modes():
    """Every 4^3 window of a field with one fixed quadratic form and varying
    linear parts lies in a 5-dimensional span: no patch keeps more than 5."""
    n, m = 16, 4
    rng = np.random.default_rng(1)
    z, y, x = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    quad = 0.02 * x * x - 0.03 * y * y + 0.015 * z * z + 0.01 * x * y - 0.02 * x * z + 0.025 * y * z
    f = np.stack([rng.standard_normal() * 5 + rng.standard_normal() * x + rng.standard_normal() * y +
                  rng.standard_normal() * z + quad for _ in range(4)]).astype(np.float32)
    comp, _, _ = _run(f, m, 0.5)
    res = gb.unpack(comp.cpu().numpy().tobytes())
    assert max(len(r[2]) for r in res["recs"]) <= 5


def test_zero_field_and_errors():
    z = np.zeros((3, 8, 8, 8), np.float32)
    comp, _, _ = _run(z, 4, 1.0)
    res = gb.unpack(comp.cpu().numpy().tobytes())
    assert all(len(r[2]) == 0 for r in res["recs"])
    assert np.array_equal(dls.gb_decompress(comp).cpu().numpy(), np.zeros(z.shape))
    f = torch.from_numpy(synth.modes3d(8, 8, 8, 2, seed=3, count=4).numpy()[0]).cuda()
    with pytest.raises(dls.DlsError):                       # an origin outside the snapshot
        dls.gb_compress(f, 4, 1.0, np.array([[5, 0, 0]], np.int64))
    bad = f.clone()
    bad[1, 2, 3, 4] = float("nan")
    with pytest.raises(dls.DlsError):
        dls.gb_compress(bad, 4, 1.0, np.zeros((4, 3), np.int64))
    with pytest.raises(dls.DlsError):                       # extents not multiples of the patch
        dls.gb_compress(f[:, :, :, :6].contiguous(), 4, 1.0, np.zeros((4, 3), np.int64))
    comp = dls.gb_compress(f, 4, 1.0, np.zeros((4, 3), np.int64))
    out = torch.empty(f.shape, dtype=torch.float64, device="cuda")
    assert dls.gb_decompress_into(comp[:-8], out) == dls.ERR_CORRUPT
    c2 = comp.clone()
    c2[0] ^= 1
    assert dls.gb_decompress_into(c2, out) == dls.ERR_CORRUPT
    assert dls.gb_decompress_into(comp, out) == dls.OK
