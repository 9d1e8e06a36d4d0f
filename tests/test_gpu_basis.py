"""Fixed bases (Sec. 4) through the C ABI on the GPU: the plain form with
cosine or random modes writes the oracle's stream byte for byte (blocks of
another Gram order keep their own modes), through dls_compress, a captured
plan and the host-buffer entry point; the decoder needs nothing more; the
library refuses what the host checks refuse."""
import numpy as np
import pytest
import torch

import oracle
from paper_2601_20113_gb300 import dls, synth

pytestmark = pytest.mark.gpu

BLOCK = (16, 16, 16, 16)


@pytest.fixture(scope="module", autouse=True)
def _build():
    from paper_2601_20113_gb300 import build
    build.build()
    oracle.build()


def _basis(which, n=16):
    return synth.dct_basis(n) if which == "cosine" else synth.random_basis(n, 21)


def _field(dims, dtype):
    # ragged time edge: blocks of Gram order 16 and 8
    return synth.modes3d(*dims, seed=8, count=32, dtype=dtype)


@pytest.mark.parametrize("which", ["cosine", "random"])
@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
def test_fixed_basis_stream_identical(which, dtype):
    dims = (32, 32, 16, 24)
    f = _field(dims, dtype)
    f_np = f.numpy()
    eb = 1e-3 * float(f.max() - f.min())
    B = _basis(which)
    cfg = oracle.Config(dims, BLOCK, oracle.F32 if dtype == torch.float32 else oracle.F64, eb=eb, rank_cap=16,
                        basis=B)
    st, ref, _ = oracle.compress(cfg, f_np)
    assert st == 0
    fd = f.cuda()
    comp = dls.compress(fd, block=BLOCK, eb=eb, rank_cap=16, basis=B)
    got = comp.cpu().numpy()
    assert got.size == ref.size and np.array_equal(got, ref)
    # the modes travel in the records: the plain decoder restores the field within eb
    rec = dls.decompress(comp)
    assert float((rec.double() - fd.double()).abs().max()) <= eb
    # and the adaptive modes give a different, smaller stream on this field
    own = dls.compress(fd, block=BLOCK, eb=eb, rank_cap=16)
    assert own.numel() < comp.numel()


def test_fixed_basis_plan_and_host_entry():
    dims = (32, 32, 16, 32)
    f = synth.modes3d(*dims, seed=9, count=32)
    eb = 1e-3 * float(f.max() - f.min())
    B = _basis("cosine")
    cfg = oracle.Config(dims, BLOCK, oracle.F32, eb=eb, rank_cap=16, basis=B)
    st, ref, _ = oracle.compress(cfg, f.numpy())
    assert st == 0
    fd = f.cuda()
    p = dls.make_params(tuple(f.shape), torch.float32, BLOCK, eb, rank_cap=16, basis=B)
    out = torch.empty(dls.compress_bound(p), dtype=torch.uint8, device="cuda")
    ws = torch.empty(dls.workspace_size(p), dtype=torch.uint8, device="cuda")
    plan = dls.CompressPlan(p, fd, out, ws)
    for _ in range(2):
        nb = plan.execute()
        assert np.array_equal(out[:nb].cpu().numpy(), ref)
    plan.close()
    h_in = f.contiguous().pin_memory()
    h_out = torch.empty(dls.compress_bound(p), dtype=torch.uint8).pin_memory()
    staging = torch.empty(dls.host_staging_size(p), dtype=torch.uint8, device="cuda")
    st, nb = dls.compress_host_into(p, h_in, h_out, staging)
    assert st == 0 and np.array_equal(h_out[:nb].numpy(), ref)


@pytest.mark.parametrize("kw", [dict(precision=dls.PREC_FP32), dict(rank_mode=dls.RANK_LEARNED)])
def test_fixed_basis_needs_the_plain_search(kw):
    f = synth.modes3d(16, 16, 16, 16, seed=1, count=8).cuda()
    with pytest.raises(dls.DlsError):
        dls.compress(f, block=BLOCK, eb=1e-3, rank_cap=16, basis=_basis("cosine"), **kw)
