"""Trains the block-rank MLP on the GPU with the library's own kernels.

Training data: for seeded synthetic fields of the modes3d kind (64^3 x 32
float32, 128 blocks of 16^3 x 16 each, with the mode count, noise level and
absolute bound drawn per field), the per-block features and the rank the
bisection of Algorithm 1 chose (dls_block_features, FP32 mode).  The network
(dls_mlp_train: minibatch Adam on the squared error of the rank) learns to
predict that rank, so the learned rank mode can test one candidate instead of
bisecting.  The saved model is a little-endian float32 file: magic "DLSM",
u32 count, then DLS_MLP_NPARAM values.

    python -m paper_2601_20113_gb300.train_rank --fields 2000 --out rank_model.bin
"""
from __future__ import annotations

import argparse
import json
import os
import struct
import sys
import time

import numpy as np
import torch

from . import dls, synth

HERE = os.path.dirname(os.path.abspath(__file__))
DEFAULT_MODEL = os.path.join(HERE, "rank_model.bin")
F, H = dls.MLP_NFEAT, 64
OFF_MU, OFF_SIG, OFF_W1 = 0, F, 2 * F
OFF_B1 = OFF_W1 + H * F
OFF_W2 = OFF_B1 + H
OFF_B2 = OFF_W2 + H * H
OFF_W3 = OFF_B2 + H
OFF_B3 = OFF_W3 + H


def save_model(path: str, params: np.ndarray) -> None:
    params = np.ascontiguousarray(params, dtype="<f4")
    with open(path, "wb") as fh:
        fh.write(b"DLSM" + struct.pack("<I", params.size) + params.tobytes())


def load_model(path: str = DEFAULT_MODEL) -> np.ndarray:
    with open(path, "rb") as fh:
        blob = fh.read()
    if blob[:4] != b"DLSM":
        raise ValueError(f"{path}: not a rank model")
    n = struct.unpack("<I", blob[4:8])[0]
    p = np.frombuffer(blob[8:8 + 4 * n], dtype="<f4").astype(np.float32)
    if p.size != dls.MLP_NPARAM:
        raise ValueError(f"{path}: {p.size} parameters, expected {dls.MLP_NPARAM}")
    return p


def collect(nfields: int, seed0: int, dims=(64, 64, 64, 32), device="cuda"):
    """Features and exact ranks of every block of `nfields` seeded fields."""
    rng = np.random.Generator(np.random.Philox(seed0))
    feats, ranks = [], []
    for i in range(nfields):
        count = int(rng.integers(16, 97))
        noise = float(10.0 ** rng.uniform(-4, -2))
        rel = float(10.0 ** rng.uniform(-5, -2))
        f = synth.modes3d(*dims, seed=seed0 + i, count=count, noise=noise, device=device)
        eb = rel * float(f.max() - f.min())
        fe, r = dls.block_features(f, (16, 16, 16, 16), eb, rank_cap=16)
        keep = r >= 0
        feats.append(fe[keep])
        ranks.append(r[keep].float())
    return torch.cat(feats), torch.cat(ranks)


def init_params(seed: int, mu: np.ndarray, sig: np.ndarray) -> np.ndarray:
    rng = np.random.Generator(np.random.Philox(seed))
    p = np.zeros(dls.MLP_NPARAM, np.float32)
    p[OFF_MU:OFF_SIG] = mu
    p[OFF_SIG:OFF_W1] = sig
    p[OFF_W1:OFF_B1] = rng.standard_normal(H * F) * np.sqrt(2.0 / F)
    p[OFF_W2:OFF_B2] = rng.standard_normal(H * H) * np.sqrt(2.0 / H)
    p[OFF_W3:OFF_B3] = rng.standard_normal(H) * np.sqrt(1.0 / H)
    p[OFF_B3] = 4.0
    return p


def accuracy(params: torch.Tensor, feat: torch.Tensor, rank: torch.Tensor) -> float:
    y = dls.mlp_forward(params, feat)
    pred = torch.clamp(torch.round(y), 0, 16)
    return float((pred == rank).float().mean().item())


def train(feat: torch.Tensor, rank: torch.Tensor, epochs: int = 12, batch: int = 128, lr: float = 2e-3,
          seed: int = 7):
    fe = feat.cpu().numpy()
    mu = fe.mean(0).astype(np.float32)
    sig = (fe.std(0) + 1e-3).astype(np.float32)
    P = torch.from_numpy(init_params(seed, mu, sig)).to(feat.device)
    A = torch.zeros(2 * dls.MLP_NPARAM, dtype=torch.float32, device=feat.device)
    n = feat.shape[0]
    rng = np.random.Generator(np.random.Philox(seed + 1))
    steps_per_epoch = max(1, n // batch)
    step = 0
    log = []
    for ep in range(epochs):
        order = torch.from_numpy(rng.permutation(n).astype(np.int32)).to(feat.device)
        lr_ep = lr * (0.5 ** (ep // 4))
        losses = dls.mlp_train(P, A, feat, rank, order, steps_per_epoch, batch, lr_ep, step)
        step += steps_per_epoch
        log.append(float(losses[-min(200, steps_per_epoch):].mean().item()))
    return P, log


def main(argv=None) -> int:
    ap = argparse.ArgumentParser()
    ap.add_argument("--fields", type=int, default=2000)
    ap.add_argument("--val-fields", type=int, default=200)
    ap.add_argument("--seed", type=int, default=1000)
    ap.add_argument("--epochs", type=int, default=12)
    ap.add_argument("--out", default=DEFAULT_MODEL)
    ap.add_argument("--report", default=None)
    args = ap.parse_args(argv)
    from . import build
    build.build()
    t0 = time.time()
    feat, rank = collect(args.fields, args.seed)
    vfeat, vrank = collect(args.val_fields, args.seed + args.fields)
    t1 = time.time()
    P, log = train(feat, rank, epochs=args.epochs)
    torch.cuda.synchronize()
    t2 = time.time()
    rep = {
        "fields": args.fields, "samples": int(feat.shape[0]), "val_samples": int(vfeat.shape[0]),
        "collect_s": t1 - t0, "train_s": t2 - t1, "epoch_loss": log,
        "train_exact_rank_acc": accuracy(P, feat, rank), "val_exact_rank_acc": accuracy(P, vfeat, vrank),
        "tail_estimate_val_acc": float((vfeat[:, 31] == vrank).float().mean().item()),
        "rank_hist": np.bincount(rank.cpu().numpy().astype(int), minlength=17).tolist(),
    }
    save_model(args.out, P.cpu().numpy())
    print(json.dumps(rep))
    if args.report:
        with open(args.report, "w") as fh:
            json.dump(rep, fh, indent=1)
    return 0


if __name__ == "__main__":
    sys.exit(main())
