"""Z-slab distribution on the GPU library (Sec. 2.7.1 data layout): each part
of the field compressed on its own with the whole field's statistics, its
records merged run by run, gives the whole field's stream byte for byte.

One GPU plays the ranks one after another (the parts share nothing but the
statistics, combined on the host in rank order as the all-gather of the
multi-process writer does).  The statistics pass itself is checked against
plain definitions: min and max exact, the point count exact, the sum of
squares within FP64 rounding; and the whole field's own statistics given back
as the global statistics resolve the bounds the library resolves alone.
"""
import numpy as np
import pytest
import torch

from paper_2601_20113_gb300 import dls, shard, synth, train_rank

pytestmark = pytest.mark.gpu

BLOCK = (16, 16, 16, 16)
DIMS = (64, 48, 88, 40)            # x, y, z, t: 5 whole z layers and a ragged one; ragged in t
EB = {dls.EB_ABS: (2e-3, 7e-3), dls.EB_REL_RANGE: (1e-3, 3e-4), dls.EB_NRMSE: (0.4, 0.9)}
FORMS = [(dls.PREC_FP64, dls.RANK_SEARCH), (dls.PREC_FP32, dls.RANK_LEARNED), (dls.PREC_FP32, dls.RANK_TAIL)]


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2601_20113_gb300 import build
    build.build()
    dls.set_rank_model(train_rank.load_model())


@pytest.fixture(scope="module")
def field():
    a = synth.modes3d(*DIMS, seed=41, count=40, device="cuda")
    b = synth.modes3d(*DIMS, seed=42, count=20, device="cuda") * 2.5 - 0.75
    return torch.cat([a, b], dim=0).contiguous()


def _params(x, eb_type, form, gstats=None, codec=0):
    return dls.make_params(tuple(x.shape), x.dtype, BLOCK, EB[eb_type], eb_type, 16, precision=form[0],
                           rank_mode=form[1], global_stats=gstats, corr_codec=codec)


def _compress(x, eb_type, form, gstats=None, plan=False, codec=0):
    p = _params(x, eb_type, form, gstats, codec)
    out = torch.empty(dls.compress_bound(p), dtype=torch.uint8, device="cuda")
    ws = torch.empty(dls.workspace_size(p), dtype=torch.uint8, device="cuda")
    if plan:
        pl = dls.CompressPlan(p, x, out, ws)
        nb = pl.execute()
        pl.close()
    else:
        st, nb = dls.compress_into(p, x, out, ws)
        assert st == dls.OK, dls.status_string(st)
    return out[:nb].cpu().numpy().tobytes()


def _stats(x):
    p = _params(x, dls.EB_ABS, FORMS[0])
    return dls.field_stats(p, x)


def test_field_stats_against_definitions(field):
    g = _stats(field)
    f = field.double().reshape(field.shape[0], -1)
    np.testing.assert_array_equal(g[:, 0], f.min(1).values.cpu().numpy())
    np.testing.assert_array_equal(g[:, 1], f.max(1).values.cpu().numpy())
    np.testing.assert_allclose(g[:, 2], (f * f).sum(1).cpu().numpy(), rtol=1e-13)
    np.testing.assert_array_equal(g[:, 3], np.full(2, float(f.shape[1])))
    bad = field.clone()
    bad[1, 3, 5, 7, 11] = float("nan")
    with pytest.raises(dls.DlsError):
        _stats(bad)


@pytest.mark.parametrize("eb_type", [dls.EB_REL_RANGE, dls.EB_NRMSE])
def test_own_statistics_given_back_resolve_alike(field, eb_type):
    """A field's own statistics as global statistics: the same stream as the
    library's own resolution (same pass, same summation order)."""
    form = FORMS[1]
    assert _compress(field, eb_type, form, _stats(field)) == _compress(field, eb_type, form)


@pytest.mark.parametrize("form", FORMS, ids=["fp64-search", "fp32-learned", "fp32-tail"])
@pytest.mark.parametrize("eb_type", [dls.EB_ABS, dls.EB_REL_RANGE, dls.EB_NRMSE])
@pytest.mark.parametrize("world", [2, 3])
def test_zslab_parts_merge_into_the_whole_stream(field, eb_type, form, world):
    ranges = [shard.zslab_range(DIMS[2], BLOCK[2], r, world) for r in range(world)]
    parts = [field[:, :, z0:z1].contiguous() for z0, z1 in ranges]
    g = shard.combine_stats([_stats(x) for x in parts])
    streams = [_compress(x, eb_type, form, g, plan=(form == FORMS[1] and i == 0)) for i, x in enumerate(parts)]
    merged = shard.merge_zslabs(streams)
    whole = _compress(field, eb_type, form, g)
    assert merged == whole
    if eb_type != dls.EB_NRMSE:
        assert merged == _compress(field, eb_type, form)
    rec = dls.decompress(torch.from_numpy(np.frombuffer(merged, np.uint8).copy()).cuda())
    err = (rec.double() - field.double()).reshape(2, -1)
    info = dls.stream_info(torch.from_numpy(np.frombuffer(merged, np.uint8).copy()).cuda())
    for v in range(2):
        if eb_type == dls.EB_NRMSE:
            nrmse = err[v].norm().item() / field[v].double().norm().item() * 100
            assert nrmse <= EB[eb_type][v]
        else:
            assert err[v].abs().max().item() <= info.eb[v]


@pytest.mark.parametrize("eb_type", [dls.EB_ABS, dls.EB_REL_RANGE])
def test_zslab_parts_with_rice_coded_corrections(field, eb_type):
    """The lossless stage changes records, not their order: parts compressed
    with Rice-coded corrections merge into the whole field's stream with them."""
    form = FORMS[1]
    ranges = [shard.zslab_range(DIMS[2], BLOCK[2], r, 2) for r in range(2)]
    parts = [field[:, :, z0:z1].contiguous() for z0, z1 in ranges]
    g = shard.combine_stats([_stats(x) for x in parts])
    merged = shard.merge_zslabs([_compress(x, eb_type, form, g, codec=1) for x in parts])
    assert merged == _compress(field, eb_type, form, g, codec=1)
    plain = _compress(field, eb_type, form, g)
    assert len(merged) <= len(plain)
    a = dls.decompress(torch.from_numpy(np.frombuffer(merged, np.uint8).copy()).cuda())
    b = dls.decompress(torch.from_numpy(np.frombuffer(plain, np.uint8).copy()).cuda())
    assert torch.equal(a.view(torch.int32), b.view(torch.int32))
