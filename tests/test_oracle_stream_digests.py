"""The oracle's stream bytes for fixed configurations match the digests stored
in tests/golden/stream_digests.txt (written by make_stream_digests.py beside
it).  The plain FP64 form on the GPU writes these same bytes, so a change
here is a change of the stream format: the CUDA packers and decoder must move
with it, and the digests are rewritten only together with that change."""
import importlib.util
import os

import oracle

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _gen():
    spec = importlib.util.spec_from_file_location("make_stream_digests", os.path.join(GOLDEN, "make_stream_digests.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_stream_digests():
    oracle.build()
    want = {}
    for line in open(os.path.join(GOLDEN, "stream_digests.txt")):
        if line.strip() and not line.startswith("#"):
            name, size, h = line.split()
            want[name] = (h, int(size))
    got = _gen().digests()
    assert set(got) == set(want)
    for name in want:
        assert got[name] == want[name], name
