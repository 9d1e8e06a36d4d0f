"""Plans: the autotuned, graph-captured compression of fixed buffers gives the
same stream as dls_compress, call after call, on an uneven multi-variable field;
the tuner picks and caches an occupancy form per shape class of the blocks."""
import json
import os

import numpy as np
import pytest
import torch

import oracle
from paper_2601_20113_gb300 import dls, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2601_20113_gb300 import build
    build.build()


def _buffers(p, field):
    out = torch.empty(dls.compress_bound(p), dtype=torch.uint8, device="cuda")
    ws = torch.empty(dls.workspace_size(p), dtype=torch.uint8, device="cuda")
    return out, ws


def _uneven():
    f = synth.multivar(50, 38, 26, 18).cuda()
    ebs = [1e-3, 1e-3, 1e-3, 1e-4, 1e-4]
    p = dls.make_params(tuple(f.shape), f.dtype, (16, 16, 16, 16), ebs, dls.EB_REL_RANGE, 16,
                        precision=dls.PREC_FP32, rank_mode=dls.RANK_TAIL)
    return f, p


def _key_class(line):
    return line["key"].rsplit("|", 1)[1]


def test_plan_matches_compress_on_uneven_multivariable_field(tmp_path, monkeypatch):
    cache = tmp_path / "tune.jsonl"
    monkeypatch.setenv("DLS_AUTOTUNE_CACHE", str(cache))
    f, p = _uneven()
    out, ws = _buffers(p, f)
    st, nb = dls.compress_into(p, f, out, ws)
    assert st == 0
    ref = out[:nb].cpu().clone()
    plan = dls.CompressPlan(p, f, out, ws)
    variant, ms = plan.info()
    tu = plan.tuning()
    assert variant == tu["whole"] and min(ms) > 0
    # both classes have work here (whole blocks, and edge blocks on every axis),
    # and each class keeps its faster form
    for c in ("whole", "rest"):
        a, b = tu["ms"][c]
        assert min(a, b) > 0 and tu[c] == (1 if a < b else 2)
    for _ in range(3):
        n = plan.execute()
        assert n == nb and torch.equal(out[:n].cpu(), ref)
    plan.close()
    lines = [json.loads(l) for l in cache.read_text().splitlines()]
    assert sorted(_key_class(l) for l in lines) == ["rest", "whole"]
    assert {_key_class(l): l["variant"] for l in lines} == {"whole": tu["whole"], "rest": tu["rest"]}
    plan2 = dls.CompressPlan(p, f, out, ws)      # second creation reads the cache
    t2 = plan2.tuning()
    assert (t2["whole"], t2["rest"]) == (tu["whole"], tu["rest"]) and plan2.info()[1] == (0.0, 0.0)
    assert t2["ms"] == {"whole": (0.0, 0.0), "rest": (0.0, 0.0)}
    assert plan2.execute() == nb
    plan2.close()


@pytest.mark.parametrize("forms", [(1, 2), (2, 1)])
def test_plan_takes_each_shape_class_form_from_the_cache(tmp_path, monkeypatch, forms):
    """Different cached forms for the two shape classes are each honoured, and
    the stream does not depend on them."""
    cache = tmp_path / "tune.jsonl"
    monkeypatch.setenv("DLS_AUTOTUNE_CACHE", str(cache))
    f, p = _uneven()
    out, ws = _buffers(p, f)
    st, nb = dls.compress_into(p, f, out, ws)
    assert st == 0
    ref = out[:nb].cpu().clone()
    dls.CompressPlan(p, f, out, ws).close()      # tunes and writes one line per class
    lines = [json.loads(l) for l in cache.read_text().splitlines()]
    want = dict(zip(("whole", "rest"), forms))
    with open(cache, "a") as fh:                 # later lines for a key win
        for l in lines:
            fh.write(json.dumps({"key": l["key"], "variant": want[_key_class(l)], "ms": [0, 0]}) + "\n")
    plan = dls.CompressPlan(p, f, out, ws)
    tu = plan.tuning()
    assert (tu["whole"], tu["rest"]) == forms
    for _ in range(2):
        n = plan.execute()
        assert n == nb and torch.equal(out[:n].cpu(), ref)
    plan.close()


def test_plan_plain_form_equals_oracle():
    f = synth.vortex2d(64, 64, 32, seed=1)
    eb = 1e-3 * float(f.max() - f.min())
    fd = f.cuda()
    p = dls.make_params(tuple(fd.shape), fd.dtype, (8, 8, 1, 32), eb, rank_cap=16)
    out, ws = _buffers(p, fd)
    plan = dls.CompressPlan(p, fd, out, ws)
    n = plan.execute()
    st, ref, _ = oracle.compress(oracle.Config((64, 64, 1, 32), (8, 8, 1, 32), oracle.F64, eb=eb, rank_cap=16),
                                 f.numpy())
    assert np.array_equal(out[:n].cpu().numpy(), ref)
    plan.close()


def test_plan_reports_capacity():
    f = synth.modes3d(32, 32, 16, 16, seed=3, count=8).cuda()
    p = dls.make_params(tuple(f.shape), f.dtype, (16, 16, 16, 16), 1e-3, precision=dls.PREC_FP32,
                        rank_mode=dls.RANK_TAIL)
    out = torch.empty(256, dtype=torch.uint8, device="cuda")
    ws = torch.empty(dls.workspace_size(p), dtype=torch.uint8, device="cuda")
    plan = dls.CompressPlan(p, f, out, ws)
    with pytest.raises(dls.DlsError) as e:
        plan.execute()
    assert e.value.status == -2
    plan.close()
