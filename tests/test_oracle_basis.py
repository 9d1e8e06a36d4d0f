"""Fixed bases (Sec. 4: data-adaptive SVD modes against fixed cosine and random
modes).  The oracle's basis option is pinned on cases whose answer follows
from the construction (data built from chosen modes, the block's own
eigenvectors handed back as a fixed basis, blocks of another Gram order), and
the paper's finding is reproduced on a synthetic field: SVD modes compress
best, cosine modes less, random modes least.  The library's host-side checks
of a basis run here too (no GPU call)."""
import numpy as np
import pytest

import oracle
from paper_2601_20113_gb300 import synth


@pytest.fixture(scope="module", autouse=True)
def _oracle():
    oracle.build()


def _field_from_modes(B, modes, eb, seed, dims=(8, 8, 4, 16)):
    """One float64 block whose rows are sum_k c_lk B[:, k] over the given modes
    (time side, n = nt = B's order), c_lk integer multiples of eb in [-50, 50] eb."""
    nx, ny, nz, nt = dims
    M = nx * ny * nz
    rng = np.random.default_rng(seed)
    C = rng.integers(-50, 51, size=(M, len(modes))).astype(np.float64) * eb
    X = C @ B[:, modes].T                                       # M x nt, row l = x + nx (y + ny z)
    return np.ascontiguousarray(X.T.reshape(1, nt, nz, ny, nx))


def _block(cfg, f, b=0):
    return oracle.block_compress(cfg, f, b)


def test_dct_and_random_bases_are_orthonormal():
    """The two fixed bases are orthonormal; the cosine modes are the DCT-II
    closed form (mode 0 constant, mode k with k sign changes)."""
    for n in (1, 2, 8, 16, 32):
        for B in (synth.dct_basis(n), synth.random_basis(n, 5)):
            np.testing.assert_allclose(B.T @ B, np.eye(n), atol=1e-13)
    D = synth.dct_basis(16)
    np.testing.assert_allclose(D[:, 0], np.full(16, 0.25), rtol=0, atol=1e-15)
    for k in range(16):
        assert np.count_nonzero(np.diff(np.sign(D[:, k])) != 0) == k


def test_modes_are_used_in_the_given_order():
    """Data in cosine modes 0 and 2 only: with the cosine basis the rank is 3
    (mode 1, empty, comes first), nothing needs a correction, and the stored
    modes are the given columns; sorted by captured energy it would be 2.  The
    block's own SVD basis spans exactly those two modes: rank 2."""
    eb = 0.5
    D = synth.dct_basis(16)
    f = _field_from_modes(D, [0, 2], eb, seed=3)
    fixed = _block(oracle.Config((8, 8, 4, 16), (8, 8, 4, 16), oracle.F64, eb=eb, rank_cap=16, basis=D), f)
    assert fixed["trace"].r == 3 and fixed["trace"].sweeps == 0
    assert fixed["trace"].n_corr == 0 and fixed["trace"].n_esc == 0
    np.testing.assert_array_equal(fixed["Vst"], D)
    own = _block(oracle.Config((8, 8, 4, 16), (8, 8, 4, 16), oracle.F64, eb=eb, rank_cap=16), f)
    assert own["trace"].r == 2
    # a random basis does not see the two-mode structure
    rnd = _block(oracle.Config((8, 8, 4, 16), (8, 8, 4, 16), oracle.F64, eb=eb, rank_cap=16,
                               basis=synth.random_basis(16, 11)), f)
    assert rnd["trace"].r > 3


def test_own_eigenvectors_as_fixed_basis_give_the_same_stream():
    """Handing a block its own (sorted, sign-normalised) eigenvectors as the
    fixed basis changes nothing: the fixed path and the adaptive path meet."""
    dims = (16, 16, 16, 16)
    f = synth.modes3d(*dims, seed=4, count=24).numpy()
    eb = 1e-3 * float(f.max() - f.min())
    cfg = oracle.Config(dims, (16, 16, 16, 16), oracle.F32, eb=eb, rank_cap=16)
    V = _block(cfg, f)["V"]
    st0, s0, _ = oracle.compress(cfg, f)
    st1, s1, _ = oracle.compress(oracle.Config(dims, (16, 16, 16, 16), oracle.F32, eb=eb, rank_cap=16, basis=V), f)
    assert st0 == 0 and st1 == 0
    np.testing.assert_array_equal(s0, s1)


def test_blocks_of_another_gram_order_keep_their_own_basis():
    """A ragged time edge gives blocks of Gram order 8 beside order 16: a
    16-mode basis changes only the order-16 blocks."""
    dims = (16, 16, 16, 24)
    f = synth.modes3d(*dims, seed=6, count=24).numpy()
    eb = 1e-3 * float(f.max() - f.min())
    a = oracle.Config(dims, (16, 16, 16, 16), oracle.F32, eb=eb, rank_cap=16)
    b = oracle.Config(dims, (16, 16, 16, 16), oracle.F32, eb=eb, rank_cap=16, basis=synth.dct_basis(16))
    assert oracle.block_geom(a, 0).n == 16 and oracle.block_geom(a, 1).n == 8
    assert _block(a, f, 0)["record"] != _block(b, f, 0)["record"]
    assert _block(a, f, 1)["record"] == _block(b, f, 1)["record"]


@pytest.mark.parametrize("bad", ["scaled", "nan", "order0", "order33", "rect"])
def test_invalid_bases_are_rejected(bad):
    dims = (16, 16, 16, 16)
    f = np.zeros((1, 16, 16, 16, 16), np.float32)
    B = {"scaled": 2.0 * np.eye(16), "nan": np.where(np.eye(16) > 0, np.nan, 0.0),
         "order0": np.zeros((0, 0)), "order33": np.eye(33), "rect": np.eye(16)[:, :8]}[bad]
    if bad == "rect":
        with pytest.raises(ValueError):
            oracle.Config(dims, (16, 16, 16, 16), oracle.F32, eb=1.0, basis=B)
        return
    cfg = oracle.Config(dims, (16, 16, 16, 16), oracle.F32, eb=1.0, basis=B)
    st, _, _ = oracle.compress(cfg, f)
    assert st != 0


@pytest.mark.parametrize("rel,eb_type", [(1e-3, oracle.EB_ABS), (1e-2, oracle.EB_NRMSE)])
def test_svd_beats_cosine_beats_random(rel, eb_type):
    """Sec. 4: at the same bound the data-adaptive modes give the highest
    ratio, the cosine modes less, random modes the least; the bound holds for
    every basis (pointwise for ABS, the global NRMSE target for NRMSE)."""
    dims = (32, 32, 32, 32)
    f = synth.modes3d(*dims, seed=2, count=64).numpy()
    rng = float(f.max() - f.min())
    eb = rel * rng if eb_type == oracle.EB_ABS else rel * 100.0
    cr = {}
    for name, B in (("svd", None), ("cosine", synth.dct_basis(16)), ("random", synth.random_basis(16, 7))):
        cfg = oracle.Config(dims, (16, 16, 16, 16), oracle.F32, eb=eb, eb_type=eb_type, rank_cap=16, basis=B)
        st, s, _ = oracle.compress(cfg, f)
        assert st == 0
        st, rec = oracle.decompress(s)
        assert st == 0
        err = rec.astype(np.float64) - f.astype(np.float64)
        if eb_type == oracle.EB_ABS:
            assert np.abs(err).max() <= eb
        else:
            assert np.sqrt((err ** 2).sum() / (f.astype(np.float64) ** 2).sum()) * 100 <= rel * 100 * (1 + 1e-9)
        cr[name] = f.nbytes / s.size
    assert cr["svd"] > 1.2 * cr["cosine"] > 1.2 * cr["random"], cr


def test_library_checks_a_basis_on_the_host():
    """The library's size queries apply the same rules (no GPU call): a basis
    needs the plain form and the bisection, an order in [1, 32] and
    orthonormal columns; a valid one adds its bytes to the workspace."""
    from paper_2601_20113_gb300 import dls
    shape, blk = (1, 32, 32, 32, 32), (16, 16, 16, 16)
    base = dls.workspace_size(dls.make_params(shape, dls.F32, blk, 1e-3))
    ok = dls.make_params(shape, dls.F32, blk, 1e-3, basis=synth.dct_basis(16))
    assert dls.compress_bound(ok) > 0 and dls.workspace_size(ok) >= base + 16 * 16 * 8
    for kw in (dict(basis=2.0 * np.eye(16)), dict(basis=np.eye(33)),
               dict(basis=synth.dct_basis(16), precision=dls.PREC_FP32),
               dict(basis=synth.dct_basis(16), rank_mode=dls.RANK_LEARNED)):
        assert dls.compress_bound(dls.make_params(shape, dls.F32, blk, 1e-3, **kw)) == 0, kw
