"""The allocation-free compression entry point, called through the C ABI.

Callers that cannot allocate device memory (an in-situ hook inside a
simulation that already owns the device memory, code where CUDA allocation is
not allowed) use dls_compress_noalloc, whose workspace is a fixed 64 MiB device
array inside the library.  Its streams must equal dls_compress's on the same
input, also on a second call that finds the first call's leftovers in the
shared array.  This file is named to run after every other test.
"""
import ctypes

import pytest
import torch

from paper_2601_20113_gb300 import dls, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2601_20113_gb300 import build
    build.build()


def _reference_stream(p, field):
    out = torch.empty(dls.compress_bound(p), dtype=torch.uint8, device="cuda")
    ws = torch.empty(dls.workspace_size(p), dtype=torch.uint8, device="cuda")
    st, nb = dls.compress_into(p, field, out, ws)
    assert st == 0
    return out[:nb].cpu()


def _noalloc_stream(p, field):
    L = dls.lib()
    out = torch.empty(dls.compress_bound(p), dtype=torch.uint8, device="cuda")
    nb = ctypes.c_size_t(0)
    st = L.dls_compress_noalloc(ctypes.byref(p), ctypes.c_void_p(field.data_ptr()),
                                ctypes.c_void_p(out.data_ptr()), out.numel(), ctypes.byref(nb),
                                ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 0, dls.status_string(st)
    return out[:nb.value].cpu()


def test_noalloc_matches_dls_compress_on_two_calls():
    # Two different fields back to back: the second call runs on the array the
    # first one left behind.
    cases = [
        (synth.modes3d(64, 48, 32, 16, seed=21, count=32).cuda(), (16, 16, 16, 16), 1e-3),
        (synth.modes3d(40, 36, 20, 36, seed=22, count=24).cuda(), (16, 16, 8, 16), 1e-2),
    ]
    for field, block, rel in cases:
        eb = rel * float(field.max() - field.min())
        p = dls.make_params(tuple(field.shape), field.dtype, block, eb, rank_cap=16)
        assert dls.workspace_size(p) <= 64 << 20
        ref = _reference_stream(p, field)
        got = _noalloc_stream(p, field)
        assert got.numel() == ref.numel() and torch.equal(got, ref)
        rec = dls.decompress(got.cuda())
        assert (rec.double() - field.double()).abs().max().item() <= eb


def test_noalloc_rejects_fields_beyond_its_workspace():
    # 256^3 x 16 float32 needs far more than 64 MiB of workspace; the check is
    # made on the host before any device work.
    field = torch.zeros((1, 16, 256, 256, 256), dtype=torch.float32, device="cuda")
    p = dls.make_params(tuple(field.shape), field.dtype, (16, 16, 16, 16), 1e-3)
    out = torch.empty(1024, dtype=torch.uint8, device="cuda")
    st, _ = dls.compress_noalloc_into(p, field, out)
    assert st == -8
