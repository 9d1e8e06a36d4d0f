"""Host-side checks of the C ABI that need no GPU: the library builds for
sm_103a, loads, and exports every function include/dls.h declares."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", fn)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"\b(dls_[a-z0-9_]+)\s*\(", src):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def libpath():
    from paper_2601_20113_gb300 import build
    return build.build()


def test_library_exports_every_declared_symbol(libpath):
    L = ctypes.CDLL(libpath)
    declared = _declared_functions()
    assert "dls_compress" in declared and "dls_decompress" in declared and "dls_verify" in declared
    missing = [n for n in sorted(declared) if not hasattr(L, n)]
    assert not missing, missing


def test_binding_declares_every_symbol(libpath):
    from paper_2601_20113_gb300 import dls
    assert _declared_functions() <= set(dls._SIGS)


def test_host_only_entry_points(libpath):
    """Size queries and status strings run without touching the GPU."""
    from paper_2601_20113_gb300 import dls
    p = dls.make_params((1, 64, 256, 256, 256), dls.F32, (16, 16, 16, 16), 1e-3)
    assert dls.compress_bound(p) >= 4 * 256 ** 3 * 64
    assert dls.workspace_size(p) > 0
    bad = dls.make_params((1, 8, 1, 8, 8), dls.F32, (16, 8, 1, 8), 1e-3)
    assert dls.compress_bound(bad) == 0 and dls.workspace_size(bad) == 0
    bad = dls.make_params((1, 64, 1, 64, 64), dls.F32, (64, 64, 1, 64), 1e-3)
    assert dls.compress_bound(bad) == 0
    assert dls.status_string(0) == "ok"
    assert "corrupt" in dls.status_string(-4)


def test_compress_bound_matches_oracle(libpath):
    import oracle
    from paper_2601_20113_gb300 import dls
    for dims, block, nv, dt in [((64, 64, 1, 32), (8, 8, 1, 32), 1, oracle.F64),
                                ((250, 190, 130, 50), (16, 16, 16, 16), 5, oracle.F32),
                                ((13, 7, 5, 9), (4, 3, 2, 4), 2, oracle.F32)]:
        cfg = oracle.Config(dims, block, dt, eb=1.0, nvars=nv)
        p = dls.make_params((nv, dims[3], dims[2], dims[1], dims[0]), dt, block, 1.0)
        assert dls.compress_bound(p) == oracle.compress_bound(cfg)


def test_struct_layouts_match_the_header(tmp_path):
    """Every struct the ABI passes (parameters, verification report, stream
    information) has the same size and field offsets in include/dls.h, as
    compiled by the host C compiler, as in its ctypes mirror in the binding;
    the oracle's own parameter struct likewise matches its header."""
    import shutil
    import subprocess
    import oracle
    from paper_2601_20113_gb300 import dls
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    cases = [("dls_params", dls.Params, "dls.h", os.path.join(ROOT, "include")),
             ("dls_report", dls.Report, "dls.h", os.path.join(ROOT, "include")),
             ("dls_stream_info", dls.StreamInfo, "dls.h", os.path.join(ROOT, "include")),
             ("dls_gb_params", dls.GbParams, "dls.h", os.path.join(ROOT, "include")),
             ("or_params", oracle.Params, "dls_oracle.h", os.path.join(ROOT, "oracle"))]
    for cname, py, hdr, inc in cases:
        lines = [f'#include "{hdr}"', "#include <stdio.h>", "#include <stddef.h>", "int main(void) {",
                 f'  printf("%zu\\n", sizeof({cname}));']
        for name, _ in py._fields_:
            lines.append(f'  printf("%zu\\n", offsetof({cname}, {name}));')
        lines += ["  return 0;", "}"]
        src = tmp_path / f"{cname}.c"
        src.write_text("\n".join(lines) + "\n")
        exe = tmp_path / cname
        subprocess.run([cc, "-I", inc, str(src), "-o", str(exe)], check=True, capture_output=True)
        got = [int(v) for v in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()]
        want = [ctypes.sizeof(py)] + [getattr(py, name).offset for name, _ in py._fields_]
        assert got == want, (cname, got, want)
