"""CPU measurements of stored forms, from oracle streams (test infrastructure).

    python -m oracle.measure_formats

Prints, for modes3d fields:
- the ratio of the current records, with the Rice-coded correction section, and
  with deflate (zlib 1 / 6 / 9) over the whole stream; the share of each record
  section and how much deflate shrinks it (the plain form's GPU streams are
  byte-identical to these);
- the global-basis form (one basis per variable, m = 4) against the block-local
  NRMSE form at the same NRMSE targets.
"""
from __future__ import annotations

import zlib

import numpy as np

from . import Config, EB_ABS, EB_NRMSE, F32, build, compress, decompress
from . import global_basis as gb


def _sections(s: bytes):
    """Bytes of each record section of a stream of 16^3 x 16 float32 blocks."""
    al = lambda x, a: (x + a - 1) // a * a
    u64 = np.frombuffer(s[:128], np.uint64)
    nb, offp, payp = int(u64[11]), int(u64[13]), int(u64[14])
    offs = np.frombuffer(s[offp:offp + 8 * (nb + 1)], np.uint64)
    sec = {k: bytearray() for k in ("header", "basis", "coefficients", "corrections", "escapes")}
    n, L, N, es = 16, 4096, 65536, 4
    for i in range(nb):
        rec = s[payp + int(offs[i]): payp + int(offs[i + 1])]
        r, flags, wk, ib = rec[0], rec[1], rec[2], rec[3]
        if flags & 1:
            sec["escapes"] += rec
            continue
        ncorr = int(np.frombuffer(rec[4:8], np.uint32)[0])
        off_v = 16 + al(r, 8)
        off_q = off_v + al(n * r * es, 8)
        off_c = off_q + al(sum((L * w + 31) // 32 for w in rec[16:16 + r]) * 4, 8)
        if flags & 8:
            cw = 2 + (N + 1023) // 1024 + int(np.frombuffer(rec[off_c:off_c + 4], np.uint32)[0])
        elif wk == 0:
            cw = 0
        elif flags & 4:
            cw = (N * wk + 31) // 32
        else:
            cw = (ncorr * (ib + wk) + 31) // 32
        off_ei = off_c + al(cw * 4, 8)
        sec["header"] += rec[:off_v]
        sec["basis"] += rec[off_v:off_q]
        sec["coefficients"] += rec[off_q:off_c]
        sec["corrections"] += rec[off_c:off_ei]
        sec["escapes"] += rec[off_ei:]
    return sec


def lossless(dims=(64, 64, 64, 32), bounds=(1e-2, 1e-3, 1e-4)):
    from paper_2601_20113_gb300 import synth
    f = synth.modes3d(*dims, seed=2, count=64).numpy()
    rng = float(f.max() - f.min())
    for rel in bounds:
        ratios = []
        for codec in (0, 1):
            st, s, _ = compress(Config(dims, (16, 16, 16, 16), F32, eb=rel * rng, eb_type=EB_ABS, rank_cap=16,
                                       corr_codec=codec), f)
            ratios.append(f.nbytes / s.size)
            if codec == 0:
                b = s.tobytes()
        z = [f.nbytes / len(zlib.compress(b, lvl)) for lvl in (1, 6, 9)]
        sec = _sections(b)
        tot = sum(len(v) for v in sec.values())
        parts = "; ".join(f"{k} {100 * len(v) / tot:.0f}% deflate x{len(v) / max(1, len(zlib.compress(bytes(v), 6))):.2f}"
                          for k, v in sec.items() if len(v))
        print(f"abs {rel:g} x range: ratio {ratios[0]:.3f}, Rice corrections {ratios[1]:.3f}, "
              f"deflate 1/6/9 {z[0]:.2f}/{z[1]:.2f}/{z[2]:.2f} | {parts}", flush=True)


def global_vs_local(dims=(32, 32, 32, 32), targets=(1.0, 0.1), m=4):
    from paper_2601_20113_gb300 import synth
    f = synth.modes3d(*dims, seed=2, count=64).numpy()
    origins = synth.patch_origins(dims[:3], (m, m, m), 4 * m ** 3, seed=3)
    for eps_t in targets:
        res = gb.compress(f[0].astype(np.float64), m, eps_t, origins)
        s = gb.pack(res)
        rec = gb.decompress(res)
        nr = 100 * np.linalg.norm(rec - f[0]) / np.linalg.norm(f[0])
        dofs = sum(len(r[2]) for r in res["recs"]) / f.size
        st, sl, _ = compress(Config(dims, (16, 16, 16, 16), F32, eb=eps_t, eb_type=EB_NRMSE, rank_cap=16), f)
        st, rl = decompress(sl)
        nrl = 100 * np.linalg.norm(rl.astype(np.float64) - f) / np.linalg.norm(f.astype(np.float64))
        print(f"NRMSE target {eps_t}%: global m={m} ratio {f.nbytes / len(s):.2f} ({nr:.3f}%, {dofs:.3f} DOFs "
              f"per point) | block-local 16^3x16 ratio {f.nbytes / sl.size:.2f} ({nrl:.3f}%)", flush=True)


if __name__ == "__main__":
    build()
    lossless()
    global_vs_local()
