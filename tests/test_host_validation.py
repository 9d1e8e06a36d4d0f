"""Parameter validation of the C ABI, on the host (no GPU): the size queries
run the same checks as the compressions, so an invalid parameter set reports
size 0, and the global-basis entry points reject bad arguments before any
device work."""
import ctypes as C

import numpy as np
import pytest
import torch

SHAPE = (2, 32, 32, 32, 32)          # nvars, nt, nz, ny, nx
BLOCK = (16, 16, 16, 16)
POINTS = float(32 ** 4)


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2601_20113_gb300 import build
    build.build()


def _bound(**kw):
    from paper_2601_20113_gb300 import dls
    p = dls.make_params(SHAPE, torch.float32, BLOCK, [1e-3, 2e-3], kw.pop("eb_type", dls.EB_REL_RANGE), 16,
                        precision=dls.PREC_FP32, **kw)
    return dls.compress_bound(p), dls.workspace_size(p)


def _stats(over=None):
    g = np.array([[-1.0, 2.0, 10.0, POINTS], [0.5, 0.75, 3.0, POINTS]])
    for (i, j), v in (over or {}).items():
        g[i, j] = v
    return g


def test_corr_codec_values():
    ok0, ws0 = _bound(corr_codec=0)
    ok1, ws1 = _bound(corr_codec=1)
    assert ok0 > 0 and ok1 == ok0                   # the bound does not change
    assert ws1 >= ws0 + ok0                         # the stage's staging stream lives in the workspace
    for bad in (2, -1, 7):
        assert _bound(corr_codec=bad) == (0, 0)


def test_global_stats_validation():
    assert _bound(global_stats=_stats())[0] > 0
    bad = [
        {(0, 0): np.nan},                    # not finite
        {(1, 2): np.inf},
        {(0, 0): 3.0},                       # min > max
        {(1, 2): -1.0},                      # negative sum of squares
        {(0, 3): 0.5, (1, 3): 0.5},          # fewer than one point
        {(1, 3): POINTS + 1},                # point counts differ between variables
        {(0, 3): 10.5, (1, 3): 10.5},        # not an integral count
    ]
    for over in bad:
        assert _bound(global_stats=_stats(over)) == (0, 0), over
    from paper_2601_20113_gb300 import dls
    with pytest.raises(ValueError):          # the binding checks the shape
        dls.make_params(SHAPE, torch.float32, BLOCK, 1e-3, dls.EB_ABS, 16, global_stats=np.zeros((3, 4)))


def _gb(dims, m, eps_t=1.0, nsample=256):
    from paper_2601_20113_gb300 import dls
    p = dls.gb_params(dims, m, eps_t, nsample)
    return dls.lib().dls_gb_bound(C.byref(p)), dls.lib().dls_gb_workspace_size(C.byref(p)), p


def test_global_basis_sizes_and_validation():
    # the bound: header, basis, offsets, and every record at its largest
    b, ws, _ = _gb((8, 16, 16, 16), 4)
    M, nrec = 64, 8 * 4 * 4 * 4
    rec_max = 8 + 4 * ((M * (6 + 63) + 31) // 32)
    assert b == 80 + 8 * M * M + 8 * (nrec + 1) + nrec * (-(-rec_max // 8) * 8)
    assert ws > 0
    assert _gb((4, 1, 33, 33), 11)[0] > 0         # 2-D patches: M = 121
    assert _gb((8, 16, 16, 15), 4)[0] == 0        # extents not multiples of the patch
    assert _gb((8, 18, 18, 18), 6)[0] == 0        # M = 216 > 128
    assert _gb((8, 16, 16, 16), 4, eps_t=0.0)[0] == 0
    assert _gb((8, 16, 16, 16), 4, eps_t=float("nan"))[0] == 0
    assert _gb((8, 16, 16, 16), 4, nsample=0)[0] == 0


def test_global_basis_rejects_null_buffers_before_device_work():
    from paper_2601_20113_gb300 import dls
    _, _, p = _gb((8, 16, 16, 16), 4)
    nb = C.c_size_t(0)
    st = dls.lib().dls_gb_compress(C.byref(p), None, None, None, 0, C.byref(nb), None, 0, None)
    assert st == -1
    assert dls.lib().dls_gb_decompress(None, 0, None, 0, None) == -1


def test_pitched_copy_in_the_workspace():
    """A float32 field whose x extent is not a multiple of 4 floats, compressed
    whole by the staged kernels, has a copy with x lines padded to a multiple of
    4 floats in its workspace; a block range of it, and a field whose lines are
    already whole multiples of 16 bytes, have none."""
    from paper_2601_20113_gb300 import dls

    def ws(shape, **kw):
        p = dls.make_params(shape, torch.float32, BLOCK, 1e-3, dls.EB_ABS, 16, precision=dls.PREC_FP32, **kw)
        return dls.workspace_size(p)

    nb = 2 * 2 * 2 * 3 * 4                       # 2 variables, 2 x 2 x 3 x 4 blocks of 16^4 each
    slack = 16384                                # the last block's per-block entries and alignments
    for nx, pitched in ((50, 2 * 18 * 26 * 38 * 52 * 4), (52, 0)):
        shape = (2, 18, 26, 38, nx)
        diff = ws(shape) - ws(shape, block_end=nb - 1)
        assert pitched <= diff <= pitched + slack, (nx, diff)
