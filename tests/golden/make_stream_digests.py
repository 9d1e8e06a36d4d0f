"""Writes tests/golden/stream_digests.txt: the SHA-256 of the oracle's stream
for a few fixed configurations (exactly computed fields, every bound type,
both dtypes, ragged edges, several variables).  Calls only the oracle.  A change to these digests is a change to the stream
format, which the CUDA packers and decoder must follow.

    python tests/golden/make_stream_digests.py
"""
import hashlib
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle  # noqa: E402


def exact_field(nvars, nt, nz, ny, nx, seed, dtype=np.float32):
    """(nvars, nt, nz, ny, nx): a smooth integer polynomial in (x, y, z, t) times
    2^-6 plus a hashed integer noise times 2^-14 -- exact dyadic values, no libm,
    so the field's bits are the same on every platform."""
    t, z, y, x = np.meshgrid(np.arange(nt), np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    out = np.empty((nvars, nt, nz, ny, nx))
    for v in range(nvars):
        s = seed + 7 * v
        h = ((x * 73856093) ^ (y * 19349663) ^ (z * 83492791) ^ (t * 2654435761) ^ (s * 97)) % 4096
        smooth = x * (t + 3) - 2 * y * z + 3 * (x - y) * (t % 7) + (s % 5) * z * z + (s % 3) * x * y
        out[v] = smooth * 2.0 ** -6 + h * 2.0 ** -14
    return out.astype(dtype)


def cases():
    """(name, field (nvars, nt, nz, ny, nx) numpy, Config)."""
    a = exact_field(1, 32, 1, 64, 64, seed=1, dtype=np.float64)
    yield "exact2d_f64_abs", a, oracle.Config((64, 64, 1, 32), (8, 8, 1, 32), oracle.F64,
                                              eb=1e-3 * float(a.max() - a.min()), rank_cap=16)
    m = exact_field(1, 24, 20, 24, 40, seed=2)
    yield "exact3d_f32_ragged_abs", m, oracle.Config((40, 24, 20, 24), (16, 16, 16, 16), oracle.F32,
                                                     eb=1e-3 * float(m.max() - m.min()), rank_cap=16)
    yield "exact3d_f32_rel", m, oracle.Config((40, 24, 20, 24), (16, 16, 16, 16), oracle.F32, eb=1e-4,
                                              eb_type=oracle.EB_REL_RANGE, rank_cap=8)
    yield "exact3d_f32_nrmse", m, oracle.Config((40, 24, 20, 24), (16, 16, 16, 16), oracle.F32, eb=0.05,
                                                eb_type=oracle.EB_NRMSE, rank_cap=16)
    mv = exact_field(3, 10, 18, 20, 30, seed=3)
    yield "exact3d_f32_multivar", mv, oracle.Config((30, 20, 18, 10), (8, 8, 8, 8), oracle.F32,
                                                    eb=[1e-1, 1e-2, 1e-3], rank_cap=16, nvars=3)


def digests():
    out = {}
    for name, f, cfg in cases():
        st, s, _ = oracle.compress(cfg, f)
        if st != 0:
            raise RuntimeError(f"{name}: oracle status {st}")
        out[name] = (hashlib.sha256(s.tobytes()).hexdigest(), int(s.size))
    return out


if __name__ == "__main__":
    oracle.build()
    with open(os.path.join(HERE, "stream_digests.txt"), "w") as fh:
        fh.write("# SHA-256 of the oracle's stream per configuration (tests/golden/make_stream_digests.py)\n")
        for name, (h, n) in digests().items():
            fh.write(f"{name} {n} {h}\n")
    print(open(os.path.join(HERE, "stream_digests.txt")).read())
