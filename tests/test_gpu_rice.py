"""The lossless stage on the corrections: Rice-coded correction sections
(record flag 8, corr_codec = 1) on the GPU, against the oracle's coder.

- The plain FP64 form writes the oracle's stream byte for byte with the codec
  on, over block shapes that cover ragged edges, the spatial Gram side, the
  relative and NRMSE bounds and several variables.
- The headline form (FP32 products, learned rank, captured plan) replays
  through the oracle with the codec: every record, Rice-coded or not, is the
  oracle packer's record of the same codes, corrections and escapes.
- The GPU decoder reads the oracle's Rice-coded streams into the oracle
  decoder's field, and the stage changes no decoded value.
- Damaged sections are refused.
"""
import numpy as np
import pytest
import torch

import oracle
from oracle import replay
from paper_2601_20113_gb300 import dls, synth, train_rank

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2601_20113_gb300 import build
    build.build()
    oracle.build()
    dls.set_rank_model(train_rank.load_model())


def _gpu(fd, block, eb, eb_type=dls.EB_ABS, codec=1, precision=dls.PREC_FP64, rank_mode=dls.RANK_SEARCH,
         plan=False, rank_cap=16, gstats=None):
    p = dls.make_params(tuple(fd.shape), fd.dtype, block, eb, eb_type, rank_cap, precision=precision,
                        rank_mode=rank_mode, corr_codec=codec, global_stats=gstats)
    out = torch.empty(dls.compress_bound(p), dtype=torch.uint8, device="cuda")
    ws = torch.empty(dls.workspace_size(p), dtype=torch.uint8, device="cuda")
    if plan:
        pl = dls.CompressPlan(p, fd, out, ws)
        nb = pl.execute()
        pl.close()
    else:
        st, nb = dls.compress_into(p, fd, out, ws)
        assert st == dls.OK, dls.status_string(st)
    return out[:nb].clone()


def _rice_records(stream):
    s, h = replay.parse_stream(stream)
    return sum(int(replay.record_of(s, h, i)[1]) & 8 != 0 for i in range(len(h["offsets"]) - 1))


CASES = [
    # dims (x, y, z, t), block, bound, bound type, variables
    ((48, 48, 32, 32), (16, 16, 16, 16), 1e-3, dls.EB_ABS, 1),      # entry lists smaller: no Rice record
    ((48, 48, 32, 32), (16, 16, 16, 16), 5e-4, dls.EB_ABS, 1),
    ((40, 36, 20, 36), (16, 16, 8, 16), 1e-4, dls.EB_ABS, 1),       # ragged in every axis
    ((24, 20, 2, 40), (4, 4, 2, 40), 3e-3, dls.EB_ABS, 1),          # spatial Gram side (32 < 40)
    ((32, 32, 16, 32), (16, 16, 16, 16), 2e-3, dls.EB_REL_RANGE, 2),
    ((32, 32, 16, 32), (16, 16, 16, 16), 0.3, dls.EB_NRMSE, 1),
]


@pytest.mark.parametrize("dims,block,rel,eb_type,nvars", CASES)
def test_plain_form_stream_equals_the_oracles(dims, block, rel, eb_type, nvars):
    fs = [synth.modes3d(*dims, seed=21 + v, count=24).numpy() * (1.0 + v) for v in range(nvars)]
    f = np.concatenate(fs, axis=0)
    eb = rel * float(f.max() - f.min()) if eb_type == dls.EB_ABS else rel
    fd = torch.from_numpy(f).cuda()
    # both sides resolve the bound from the same statistics (the field's norm
    # is a sum whose order differs between them)
    x = f.reshape(nvars, -1).astype(np.float64)
    g = np.stack([x.min(1), x.max(1), (x * x).sum(1), np.full(nvars, float(x.shape[1]))], axis=1)
    comp = _gpu(fd, block, eb, eb_type, gstats=g)
    cfg = oracle.Config(dims, block, oracle.F64 if f.dtype == np.float64 else oracle.F32, eb=eb, eb_type=eb_type,
                        rank_cap=16, nvars=nvars, corr_codec=1, global_stats=g)
    st, ref, _ = oracle.compress(cfg, f)
    assert st == oracle.OK
    got = comp.cpu().numpy()
    assert got.size == ref.size and np.array_equal(got, ref), (got.size, ref.size)
    # NRMSE blocks carry no corrections; at 1e-3 this field's entry lists win
    assert (_rice_records(got) > 0) == (eb_type != dls.EB_NRMSE and rel != 1e-3)
    # the stage changes no decoded value
    plain = _gpu(fd, block, eb, eb_type, codec=0, gstats=g)
    assert plain.numel() >= comp.numel()
    a, b = dls.decompress(comp), dls.decompress(plain)
    assert torch.equal(a.view(torch.int32), b.view(torch.int32))


def test_decoder_reads_the_oracles_rice_stream():
    dims = (32, 32, 16, 16)
    f = synth.modes3d(*dims, seed=12, count=16).numpy()
    eb = 1e-4 * float(f.max() - f.min())
    cfg = oracle.Config(dims, (16, 16, 16, 16), oracle.F32, eb=eb, rank_cap=16, corr_codec=1)
    st, s, _ = oracle.compress(cfg, f)
    assert st == oracle.OK and _rice_records(s) > 0
    st, ref = oracle.decompress(s)
    assert st == oracle.OK
    rec = dls.decompress(torch.from_numpy(s).cuda()).cpu().numpy()
    assert np.array_equal(rec, ref.astype(np.float32))


@pytest.mark.parametrize("rel", [1e-3, 1e-4])
def test_headline_plan_with_the_codec_replays_through_the_oracle(rel):
    dims = (128, 128, 160, 32)
    fd = synth.modes3d(*dims, seed=31, count=64, device="cuda")
    f = fd.cpu().numpy()
    eb = rel * float(f.max() - f.min())
    comp = _gpu(fd, (16, 16, 16, 16), eb, precision=dls.PREC_FP32, rank_mode=dls.RANK_LEARNED, plan=True)
    plain = _gpu(fd, (16, 16, 16, 16), eb, codec=0, precision=dls.PREC_FP32, rank_mode=dls.RANK_LEARNED)
    s = comp.cpu().numpy()
    nr = _rice_records(s)
    assert nr > 0 and comp.numel() < plain.numel()
    cfg = oracle.Config(dims, (16, 16, 16, 16), oracle.F32, eb=eb, rank_cap=16, corr_codec=1)
    res, errs = replay.replay_stream(cfg, f, s)
    assert errs == [], errs
    bad = [(r["block"], r["errors"]) for r in res if r["errors"]]
    assert not bad, bad[:5]
    a, b = dls.decompress(comp), dls.decompress(plain)
    assert torch.equal(a.view(torch.int32), b.view(torch.int32))
    assert (a.double() - fd.double()).abs().max().item() <= eb
    st, rref = oracle.decompress(s)
    assert st == oracle.OK and np.array_equal(rref.astype(np.float32), a.cpu().numpy())
    print(f"rel {rel}: {nr} of {len(res)} records Rice-coded, stream {plain.numel()} -> {comp.numel()} B "
          f"(x{plain.numel() / comp.numel():.3f})")


def test_host_path_with_the_codec_equals_the_device_path():
    dims = (64, 64, 32, 32)
    fd = synth.modes3d(*dims, seed=5, count=32, device="cuda")
    eb = 1e-3 * float(fd.max() - fd.min())
    dev = _gpu(fd, (16, 16, 16, 16), eb, precision=dls.PREC_FP32, rank_mode=dls.RANK_TAIL)
    p = dls.make_params(tuple(fd.shape), fd.dtype, (16, 16, 16, 16), eb, dls.EB_ABS, 16, precision=dls.PREC_FP32,
                        rank_mode=dls.RANK_TAIL, corr_codec=1)
    h_in = fd.cpu().pin_memory()
    h_out = torch.empty(dls.compress_bound(p), dtype=torch.uint8).pin_memory()
    staging = torch.empty(dls.host_staging_size(p), dtype=torch.uint8, device="cuda")
    st, nb = dls.compress_host_into(p, h_in, h_out, staging)
    assert st == dls.OK and np.array_equal(h_out[:nb].numpy(), dev.cpu().numpy())


def _corrupt_status(s):
    info = dls.stream_info(torch.from_numpy(s).cuda())
    out = torch.zeros((info.nvars, info.dims[3], info.dims[2], info.dims[1], info.dims[0]), dtype=torch.float32,
                      device="cuda")
    return dls.decompress_into(torch.from_numpy(s).cuda(), out)


def test_damaged_rice_sections_are_refused():
    dims = (32, 32, 16, 16)
    fd = synth.modes3d(*dims, seed=12, count=16, device="cuda")
    eb = 1e-4 * float(fd.max() - fd.min())
    s = _gpu(fd, (16, 16, 16, 16), eb).cpu().numpy()
    assert _corrupt_status(s.copy()) == dls.OK
    sb, h = replay.parse_stream(s)
    i = next(j for j in range(len(h["offsets"]) - 1) if replay.record_of(sb, h, j)[1] & 8)
    o = h["payp"] + int(h["offsets"][i])
    r = int(s[o])
    g_n, L = 16, 16 * 16 * 16
    wq = s[o + 16:o + 16 + r].astype(np.int64)
    al = lambda x, a: (x + a - 1) // a * a
    off_c = al(al(16 + al(r, 8), 8) + g_n * r * 4, 8) + al(int(sum((L * w + 31) // 32 for w in wq)) * 4, 8)
    c = o + off_c
    for mutate in (lambda b: b[c:c + 4].view(np.uint32).__iadd__(4),          # word count vs record size
                   lambda b: b[c + 4:c + 8].view(np.uint32).__setitem__(0, 21),  # kr beyond 20
                   lambda b: b[c + 8:c + 12].view(np.uint32).__setitem__(0, 0xFFFFFF)):  # chunk offset past the words
        b = s.copy()
        mutate(b)
        assert _corrupt_status(b) == dls.ERR_CORRUPT
