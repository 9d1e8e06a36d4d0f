"""Compression ratio against error for three bases (Sec. 4): the blocks' own
SVD modes (the method), fixed cosine (DCT-II) modes and seeded random
orthonormal modes, on a seeded modes3d field, through the plain FP64 form of
the library.  Prints one JSON line per (basis, bound).

    python -m paper_2601_20113_gb300.basis_compare [--dims 256,256,64,64] [--rel 1e-2,1e-3,1e-4]
"""
from __future__ import annotations

import argparse
import json

import torch

from . import build, dls, synth


def run(dims, rels, steps=3, seed=2):
    build.build()
    f = synth.modes3d(*dims, seed=seed, count=64, device="cuda")
    rng = float(f.max() - f.min())
    in_bytes = f.numel() * f.element_size()
    block = (16, 16, 16, 16)
    bases = (("svd", None), ("cosine", synth.dct_basis(16)), ("random", synth.random_basis(16, 7)))
    rows = []
    for rel in rels:
        eb = rel * rng
        for name, B in bases:
            p = dls.make_params(tuple(f.shape), torch.float32, block, eb, rank_cap=16, basis=B)
            out = torch.empty(dls.compress_bound(p), dtype=torch.uint8, device="cuda")
            ws = torch.empty(dls.workspace_size(p), dtype=torch.uint8, device="cuda")
            st, nb = dls.compress_into(p, f, out, ws)
            if st != dls.OK:
                raise dls.DlsError(st, "dls_compress")
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(steps):
                st, nb = dls.compress_into(p, f, out, ws)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / steps
            rec = dls.decompress(out[:nb])
            rep = dls.verify(f, rec, out[:nb])
            row = {"basis": name, "rel_bound": rel, "ratio": in_bytes / nb, "nrmse": rep["nrmse"],
                   "max_abs_err_over_eb": rep["max_abs_err"] / eb, "n_over_bound": rep["n_over_bound"],
                   "mean_rank": rep["mean_rank"], "compress_gbs": in_bytes / (ms * 1e-3) / 1e9,
                   "dims": list(dims), "block": list(block)}
            rows.append(row)
            print(json.dumps(row), flush=True)
            del out, ws, rec
    return rows


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--dims", default="256,256,64,64", help="nx,ny,nz,nt")
    ap.add_argument("--rel", default="1e-2,1e-3,1e-4", help="bounds as fractions of the value range")
    ap.add_argument("--steps", type=int, default=3)
    a = ap.parse_args()
    run(tuple(int(x) for x in a.dims.split(",")), [float(x) for x in a.rel.split(",")], a.steps)


if __name__ == "__main__":
    main()
