#!/usr/bin/env python3
"""Throughput bench of the GB300 block-local DLS compressor.

Workload (one step = one dls_compress call over the whole field): the
multiscale 3-D float32 field of 256^3 points x 64 timesteps (4 GiB) made of
64 seeded sinusoidal modes (|k| <= 8, amplitudes ~ |k|^(-5/3), random phases)
plus N(0, 1e-3^2) noise, blocks 16^3 x 16 (16384 blocks), absolute pointwise
bound 1e-3 x value range, rank cap 16.

Metric: compress GB/s per GPU (input bytes / time per step), inputs resident
in HBM (4 GiB > 129 MB L2, so no flush between steps).  `e2e` times the same
work through the host-buffer C entry point (pinned host in, host stream out).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

N > 1 runs under torchrun: every rank compresses its own field (independent
problems, no data-path collective, weak scaling); rank 0 prints one JSON line.
`--impl reference` times the CPU oracle on a bounded sample of the workload.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "compress GB/s/GPU at fixed pointwise abs bound"
DIMS = (256, 256, 256, 64)          # nx, ny, nz, nt
BLOCK = (16, 16, 16, 16)
REL_BOUND = 1e-3
RANK_CAP = 16
SEED = 2
# (precision, rank mode) of each form
FORMS = {"plain": (0, 0), "fp32": (3, 0), "learned": (3, 1), "tail": (3, 2)}
FORM_TEXT = {
    "plain": "plain FP64 (Gram, Jacobi, projection, bisection, correction in FP64)",
    "fp32": "FP32 products, FP32 Jacobi + orthonormalisation (error-free FP32 transforms), bisection on E(r) for "
            "all r, FP64-semantics decisions",
    "learned": "FP32 products, FP32 Jacobi + orthonormalisation (error-free FP32 transforms), MLP-predicted rank "
               "checked exactly (bisection fallback), FP64-semantics decisions",
    "tail": "FP32 products, FP32 Jacobi + orthonormalisation (error-free FP32 transforms), eigenvalue-tail rank "
            "estimate checked exactly (bisection fallback), FP64-semantics decisions",
}


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def _rank_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class Clocks:
    """Samples nvidia-smi clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        import tempfile
        self.path = os.path.join(tempfile.gettempdir(), f"dls_bench_clocks_{os.getpid()}_{index}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as fh:
            for line in fh:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax = float(parts[2])
                except ValueError:
                    continue
                for nm, val in zip(names, parts[5:9]):
                    if val.lower() == "active":
                        reasons.add(nm)
        sm.sort()
        med = sm[len(sm) // 2] if sm else None
        return {"sm_mhz": med, "sm_max_mhz": smax, "reasons": sorted(reasons), "samples": len(sm)}


def make_field(device, seed=SEED):
    from paper_2601_20113_gb300 import synth
    return synth.modes3d(*DIMS, seed=seed, count=64, device=device)


def oracle_sample_bench(field_cpu_np, eb, budget_s=20.0):
    """Times the CPU oracle (as it stands) on a bounded sample of the workload:
    sub-fields of whole 16^3 x 16 blocks cut from the same field, same absolute
    bound.  Returns (GB/s, cores, description)."""
    import numpy as np

    import oracle

    cores = os.cpu_count() or 1
    # one block-row slab: x 256 (16 blocks), y 16*ny_b, z 16, t 16
    ny_b = 1
    t0 = time.time()
    done_bytes = 0
    nblocks = 0
    elapsed = 0.0
    while True:
        sub = np.ascontiguousarray(field_cpu_np[:, 0:16, 0:16, 0:16 * ny_b, :])
        dims = (sub.shape[4], sub.shape[3], sub.shape[2], sub.shape[1])
        cfg = oracle.Config(dims, BLOCK, oracle.F32, eb=eb, rank_cap=RANK_CAP)
        ts = time.time()
        st, s, _ = oracle.compress(cfg, sub, nthreads=cores)
        dt = time.time() - ts
        assert st == 0
        elapsed = dt
        done_bytes = sub.nbytes
        nblocks = oracle.num_blocks(cfg)
        if dt * 2 > budget_s or ny_b >= 16:
            break
        ny_b = min(16, ny_b * 2)
    del t0
    desc = f"{nblocks} blocks of 16^3x16 (x 0..255, y 0..{16 * ny_b - 1}, z 0..15, t 0..15), same abs bound"
    return done_bytes / elapsed / 1e9, cores, desc, elapsed


def _sample_for_oracle(budget_s=None):
    """The oracle's bounded sample of the workload: whole 16^3 x 16 blocks
    (x 0..255, y 0..63, z 0..15, t 0..15) of the same field, with the same
    absolute bound.  Uses the GPU to evaluate the full field when one is
    present (so the bytes and the bound match the GPU arm), else evaluates the
    window on the host and takes the bound from the window's range."""
    import torch

    from paper_2601_20113_gb300 import synth
    if torch.cuda.is_available():
        f = make_field("cuda")
        eb = REL_BOUND * float(f.max() - f.min())
        sub = f[:, 0:16, 0:16, 0:64, :].contiguous().cpu().numpy()
        del f
        torch.cuda.empty_cache()
    else:
        w = ((0, 0, 0, 0), (256, 64, 16, 16))
        sub = synth.modes3d(*DIMS, seed=SEED, count=64, window=w).numpy()
        eb = REL_BOUND * float(sub.max() - sub.min())
    return sub, eb


def run_reference(args):
    """CPU oracle arm: each step compresses the bounded sample on the host cores."""
    rank, world, _ = _rank_env()
    if rank != 0:
        return 0
    import oracle
    sample, eb = _sample_for_oracle()
    cores = os.cpu_count() or 1
    dims = (sample.shape[4], sample.shape[3], sample.shape[2], sample.shape[1])
    cfg = oracle.Config(dims, BLOCK, oracle.F32, eb=eb, rank_cap=RANK_CAP)
    for _ in range(args.warmup):
        oracle.compress(cfg, sample, nthreads=cores)
    ts = time.time()
    for _ in range(args.steps):
        st, s, _ = oracle.compress(cfg, sample, nthreads=cores)
        assert st == 0
    el = time.time() - ts
    val = sample.nbytes * args.steps / el / 1e9
    desc = (f"{oracle.num_blocks(cfg)} blocks of 16^3x16 per step (x 0..255, y 0..63, z 0..15, t 0..15), "
            f"same abs bound")
    line = {
        "impl": "reference", "metric": METRIC, "value": val, "unit": "GB/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": _config(),
        "cpu_baseline": {"value": val, "unit": "GB/s", "cores": cores, "kind": "oracle", "sample": desc},
        "e2e": {"value": val, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


KERNEL_SOURCES = {
    "plain": ["k_plain.cu", "dls_internal.cuh"],
    "mixed": ["k_tile.cu", "mixed_common.cuh", "dls_device.cuh", "dls_internal.cuh"],
}
PROFILE = {"plain": "profiles/k_plain_fp64_modes3d.md", "mixed": "profiles/k_enc_modes3d.md"}
# stage of a mixed-form plan -> (kernel, what its algorithmic bytes are)
PHASE_KERNEL = {"gram": ("k_gram", "input, read once"), "eig": ("k_eig", None), "rr": ("k_rrgram", None),
                "enc": ("k_enc", "input, read once (records: deferred packer)"), "tile": ("k_tile", None),
                "pack": ("k_pack_tile", "stream written")}


def _sources_sha(kind):
    import hashlib
    h = hashlib.sha256()
    for fn in KERNEL_SOURCES[kind]:
        with open(os.path.join(ROOT, "paper_2601_20113_gb300", "csrc", fn), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def _profile_traffic(kind, blocks):
    """DRAM bytes per launch from the committed ncu summary of the kernel, scaled
    from the captured case to `blocks` blocks; None when the summary is missing
    or was taken on other sources."""
    try:
        txt = open(os.path.join(ROOT, PROFILE[kind])).read()
    except OSError:
        return None
    vals = {}
    for line in txt.splitlines():
        if ":" in line and line.strip().startswith(("source_sha256", "dram_bytes_per_block")):
            k, v = line.strip().split(":", 1)
            vals[k.strip()] = v.strip().strip("`")
    if vals.get("source_sha256") != _sources_sha(kind) or "dram_bytes_per_block" not in vals:
        return None
    return float(vals["dram_bytes_per_block"]) * blocks


def _roofline(form, in_bytes, out_bytes, kernel_ms, hbm, peak_kind, dims, phases=None):
    """Dominant kernel, timed by CUDA events inside the captured graph.  The
    plain form has one per-block kernel (k_plain): algorithmic bytes = the field
    read once + the records written.  The mixed forms run as stages (k_gram,
    k_eig, the Rayleigh-Ritz kernels, k_enc, k_tile, scan + k_pack_tile); the
    dominant one is the stage with the largest share of the step, and its
    algorithmic bytes are those of PHASE_KERNEL (k_gram and k_enc: the field
    read once; k_pack_tile: the stream written)."""
    blocks = 1
    for d, b in zip(dims, BLOCK):
        blocks *= -(-d // b)
    if form == "plain":
        alg = in_bytes + out_bytes
        ach = alg / (kernel_ms * 1e-3) / 1e9
        return {"bound": "hbm", "kernel": "k_plain", "achieved": ach, "peak": hbm, "unit": "GB/s",
                "frac": ach / hbm, "traffic": _profile_traffic("plain", blocks), "algorithmic_bytes": alg,
                "kernel_ms": kernel_ms,
                "note": f"peak = {peak_kind} HBM copy bandwidth; algorithmic bytes = input + records"}
    top = max(phases, key=phases.get)
    kern, what = PHASE_KERNEL[top]
    alg = out_bytes if top == "pack" else in_bytes
    ms = phases[top]
    ach = alg / (ms * 1e-3) / 1e9
    return {"bound": "hbm", "kernel": kern, "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
            "traffic": _profile_traffic("mixed", blocks) if kern == "k_enc" else None,
            "algorithmic_bytes": alg, "kernel_ms": ms,
            "note": f"peak = {peak_kind} HBM copy bandwidth; algorithmic bytes = {what or 'n/a'}; "
                    f"share of the step {ms / sum(phases.values()):.2f}"}


def _config(form="learned"):
    nb = 1
    for d, b in zip(DIMS, BLOCK):
        nb *= -(-d // b)
    gib = DIMS[0] * DIMS[1] * DIMS[2] * DIMS[3] * 4 / 2 ** 30
    return {"workload": f"modes3d {DIMS[0]}x{DIMS[1]}x{DIMS[2]} x {DIMS[3]} float32 ({gib:g} GiB), 64 modes "
                        f"|k|<=8, k^-5/3, N(0,1e-3^2) noise, blocks 16^3x16 ({nb}), abs bound {REL_BOUND:g} x range, "
                        "rank cap 16",
            "form": FORM_TEXT[form],
            "l2": "inputs 4 GiB > 129 MB L2 (no flush)"}


PRECISIONS = {"bf16": 5, "tf32": 4, "bf16x3": 2, "tf32x3": 1, "fp32": 3}


def run_precision_sweep(args):
    """Every precision mode of the Gram (BF16, TF32, BF16x3, 3xTF32, FP32) at
    bounds 1e-2 .. 1e-5 x range on the at-scale field, against the FP64 oracle
    (compressed and decompressed on the host cores): ratio, max pointwise error
    over the bound, NRMSE, the reconstruction difference from the oracle's, and
    GB/s of each mode's captured plan (search rank mode, so that the modes
    differ in the Gram alone)."""
    import numpy as np
    import torch

    import oracle
    from paper_2601_20113_gb300 import build, dls

    build.build()
    oracle.build()
    dev = torch.device("cuda", 0)
    field = make_field(dev)
    fh = field.cpu().numpy()
    x = fh.astype(np.float64)
    xnorm = float(np.linalg.norm(x))
    rng = float(field.max() - field.min())
    in_bytes = field.numel() * 4
    rows = []
    for rel in (1e-2, 1e-3, 1e-4, 1e-5):
        eb = rel * rng
        cfg = oracle.Config(DIMS, BLOCK, oracle.F32, eb=eb, rank_cap=RANK_CAP)
        ts = time.time()
        st, ref, _ = oracle.compress(cfg, fh)
        assert st == 0
        st, xo = oracle.decompress(ref)
        assert st == 0
        o_s = time.time() - ts
        xo = xo.astype(np.float64)
        o_nrmse = 100 * float(np.linalg.norm(xo - x)) / xnorm
        for name, prec in PRECISIONS.items():
            p = dls.make_params(tuple(field.shape), torch.float32, BLOCK, eb, dls.EB_ABS, RANK_CAP, precision=prec,
                                rank_mode=dls.RANK_SEARCH)
            out = torch.empty(dls.compress_bound(p), dtype=torch.uint8, device=dev)
            ws = torch.empty(dls.workspace_size(p), dtype=torch.uint8, device=dev)
            plan = dls.CompressPlan(p, field, out, ws)
            nb = plan.execute()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(3):
                nb = plan.execute()
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / 3
            ntc = dls.phase_cycles(p, ws)["n_tensor_core_gram"]
            plan.close()
            rec = dls.decompress(out[:nb]).cpu().numpy().astype(np.float64)
            rows.append({"precision": name, "rel_bound": rel, "ratio": in_bytes / nb,
                         "ratio_vs_oracle": (in_bytes / nb) / (in_bytes / ref.size) - 1.0,
                         "max_err_over_eb": float(np.abs(rec - x).max()) / eb,
                         "nrmse_pct": 100 * float(np.linalg.norm(rec - x)) / xnorm, "oracle_nrmse_pct": o_nrmse,
                         "recon_diff_vs_oracle": float(np.linalg.norm(rec - xo)) / xnorm,
                         "gbs": in_bytes / (ms * 1e-3) / 1e9, "tensor_core_gram_blocks": ntc,
                         "oracle_ratio": in_bytes / ref.size, "oracle_s": o_s})
            del out, ws, rec
            torch.cuda.empty_cache()
    print(json.dumps({"precision_sweep": rows, "config": _config("fp32"),
                      "note": "Gram precision modes; projection, quantizer, rank test and corrections are FP32 with "
                              "FP64-semantics decisions in every mode; oracle = plain FP64 CPU implementation"}))
    return 0


def _plan_run(p, field, steps, stream=None):
    """Times a captured plan of params p on field: (ms per step, nbytes, stages,
    counters, stream bytes on the host)."""
    import torch

    from paper_2601_20113_gb300 import dls
    out = torch.empty(dls.compress_bound(p), dtype=torch.uint8, device=field.device)
    ws = torch.empty(dls.workspace_size(p), dtype=torch.uint8, device=field.device)
    plan = dls.CompressPlan(p, field, out, ws, stream)
    tuning = plan.tuning()
    for _ in range(3):
        nb = plan.execute(stream)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    phs = []
    for _ in range(steps):
        nb = plan.execute(stream)
        phs.append(plan.phase_timing())
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    counters = dls.phase_cycles(p, ws)
    counters["tuning"] = tuning
    plan.close()
    stages = {k: sum(d[k] for d in phs) / len(phs) for k in phs[0]}
    comp = out[:nb].clone()
    del out, ws
    torch.cuda.empty_cache()
    return ms, nb, stages, counters, comp


def _pin_near_gpu(dev):
    """Binds this process to the CPUs of the GPU's NUMA node (from sysfs) for
    the pinned allocations; returns (node, the previous CPU set) or (None,
    None) where the node is not known."""
    import torch
    try:
        idx = torch.device(dev).index or 0
        pr = torch.cuda.get_device_properties(idx)
        bus = f"{pr.pci_domain_id:04x}:{pr.pci_bus_id:02x}:{pr.pci_device_id:02x}.0"
        node = int(open(f"/sys/bus/pci/devices/{bus}/numa_node").read().strip())
        if node < 0:
            return None, None
        cpus = set()
        for part in open(f"/sys/devices/system/node/node{node}/cpulist").read().strip().split(","):
            a, _, b = part.partition("-")
            cpus.update(range(int(a), int(b or a) + 1))
        keep = os.sched_getaffinity(0)
        if not cpus & keep:
            return node, None
        os.sched_setaffinity(0, cpus & keep)
        return node, keep
    except (OSError, ValueError, AttributeError):
        return None, None


def run_global_basis(dev):
    """The global-basis mode (one FP64 basis per variable from 4 m^3 random
    patches of the first snapshot, magnitude-ordered coefficients by
    bisection): modes3d 128^3 x 16 float32 (128 MiB), patches of 4^3, NRMSE
    target 1%; compression and decompression timed with CUDA events around the
    calls (each synchronizes once), three runs after one warm-up."""
    import torch

    from paper_2601_20113_gb300 import dls, synth
    dims, m, eps_t = (128, 128, 128, 16), 4, 1.0
    f = synth.modes3d(*dims, seed=2, count=64, device=dev)[0].contiguous()
    origins = synth.patch_origins(dims[:3], (m, m, m), 4 * m ** 3, seed=3)
    comp = dls.gb_compress(f, m, eps_t, origins)
    rec = dls.gb_decompress(comp)
    e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
    torch.cuda.synchronize()
    e0.record()
    for _ in range(3):
        comp = dls.gb_compress(f, m, eps_t, origins)
    e1.record()
    for _ in range(3):
        rec = dls.gb_decompress(comp)
    e2.record()
    torch.cuda.synchronize()
    nb = f.numel() * 4
    cms, dms = e0.elapsed_time(e1) / 3, e1.elapsed_time(e2) / 3
    nrmse = 100.0 * ((rec - f.double()).norm() / f.double().norm()).item()
    return {"workload": "modes3d 128x128x128 x 16 float32 (128 MiB), patches 4^3 (M = 64), S = 256, "
                        "NRMSE target 1%", "value": nb / (cms * 1e-3) / 1e9, "unit": "GB/s", "ms": cms,
            "decompress_gbs": nb / (dms * 1e-3) / 1e9, "ratio": nb / comp.numel(), "nrmse_percent": nrmse,
            "dtype": "f64"}


def run_config(args):
    """The other at-scale configurations, one JSON line each:
    4 -- five float32 variables (u, v, w, p, T: vortex + mode mixtures) on
         250 x 190 x 130 x 50 with edge blocks on every axis (mixed block
         shapes up to 16^3 x 16), bounds 1e-3 / 1e-3 / 1e-3 / 1e-4 / 1e-4 x each
         variable's range, one captured plan; the oracle's ratio on sampled
         block ranges of every variable beside the GPU's on the same blocks;
    5 -- the learned-rank evaluation field: 512^3 x 32 float32 (16 GiB), abs
         bound 1e-3 x range, learned rank with the search fallback, beside the
         tail and search rank modes."""
    import numpy as np
    import torch

    import oracle
    from oracle import replay
    from paper_2601_20113_gb300 import build, dls, synth, train_rank

    build.build()
    dev = torch.device("cuda", 0)
    dls.set_rank_model(train_rank.load_model())
    line = {"metric": METRIC, "unit": "GB/s", "n_gpus": 1, "steps": args.steps, "data": "synthetic"}
    if args.config == 4:
        dims = (250, 190, 130, 50)
        field = synth.multivar(*dims, device=dev)
        rels = [1e-3, 1e-3, 1e-3, 1e-4, 1e-4]
        in_bytes = field.numel() * 4
        modes = {}
        comp = None
        for name, rm in (("learned", dls.RANK_LEARNED), ("tail", dls.RANK_TAIL), ("search", dls.RANK_SEARCH)):
            p = dls.make_params(tuple(field.shape), torch.float32, BLOCK, rels, dls.EB_REL_RANGE, RANK_CAP,
                                precision=dls.PREC_FP32, rank_mode=rm)
            ms, nb, stages, c, cs = _plan_run(p, field, args.steps)
            modes[name] = {"value": in_bytes / (ms * 1e-3) / 1e9, "ms_per_step": ms, "ratio": in_bytes / nb,
                           "n_accepted": c["n_accepted"], "n_searched": c["n_searched"], "phases_ms": stages,
                           "tuning": c["tuning"]}
            if name == "learned":
                comp = cs
        rec = dls.decompress(comp)
        rep = dls.verify(field, rec, comp)
        del rec
        # the oracle on sampled block ranges of every variable
        cfg_all = oracle.Config(dims, BLOCK, oracle.F32, eb=rels, eb_type=oracle.EB_REL_RANGE, rank_cap=RANK_CAP,
                                nvars=5)
        nbv = oracle.num_blocks(cfg_all) // 5
        fh = field.cpu().numpy()
        s_g, h_g = replay.parse_stream(comp.cpu().numpy())
        samp = []
        for v in range(5):
            for start in (0, nbv // 2, nbv - 64):
                b0 = v * nbv + start
                cfg = oracle.Config(dims, BLOCK, oracle.F32, eb=rels, eb_type=oracle.EB_REL_RANGE,
                                    rank_cap=RANK_CAP, nvars=5, block_begin=b0, block_end=b0 + 64)
                st, so, _ = oracle.compress(cfg, fh)
                assert st == 0
                s_o, h_o = replay.parse_stream(so)
                samp.append((int(h_o["offsets"][-1]), int(h_g["offsets"][b0 + 64] - h_g["offsets"][b0])))
        o_bytes = sum(a for a, _ in samp)
        g_bytes = sum(b for _, b in samp)
        line.update({
            "value": modes["learned"]["value"], "ms_per_step": modes["learned"]["ms_per_step"],
            "config": {"workload": "multivar 5 x 250x190x130 x 50 float32 (5.75 GiB), blocks up to 16^3x16 "
                                   f"({oracle.num_blocks(cfg_all)}, mixed shapes), rel bounds {rels}, rank cap 16, "
                                   "FP32 form, one captured plan"},
            "ratio": in_bytes / comp.numel(), "max_err_over_bound": [rep["var_max_abs_err"][v] / rep["var_eb"][v]
                                                                    for v in range(5)],
            "n_over_bound": rep["n_over_bound"], "forms": modes,
            "oracle_sample": {"blocks": 5 * 3 * 64, "oracle_record_bytes": o_bytes, "gpu_record_bytes": g_bytes,
                              "ratio_gpu_over_oracle_bytes": g_bytes / o_bytes,
                              "what": "64-block ranges at the start, middle and end of each variable"}})
    else:
        dims = (512, 512, 512, 32)
        field = synth.modes3d(*dims, seed=5, count=64, device=dev)
        eb = 1e-3 * float(field.max() - field.min())
        in_bytes = field.numel() * 4
        modes = {}
        comp = None
        for name, rm in (("learned", dls.RANK_LEARNED), ("tail", dls.RANK_TAIL), ("search", dls.RANK_SEARCH)):
            p = dls.make_params(tuple(field.shape), torch.float32, BLOCK, eb, dls.EB_ABS, RANK_CAP,
                                precision=dls.PREC_FP32, rank_mode=rm)
            ms, nb, stages, c, cs = _plan_run(p, field, args.steps)
            modes[name] = {"value": in_bytes / (ms * 1e-3) / 1e9, "ms_per_step": ms, "ratio": in_bytes / nb,
                           "n_accepted": c["n_accepted"], "n_searched": c["n_searched"], "phases_ms": stages,
                           "tuning": c["tuning"]}
            if name == "learned":
                comp = cs
            else:
                del cs
        rec = dls.decompress(comp)
        err = float((rec - field).abs().max())
        del rec
        line.update({
            "value": modes["learned"]["value"], "ms_per_step": modes["learned"]["ms_per_step"],
            "config": {"workload": "modes3d 512^3 x 32 float32 (16 GiB), 64 modes |k|<=8, k^-5/3, N(0,1e-3^2) "
                                   "noise, blocks 16^3x16 (65536), abs bound 1e-3 x range, rank cap 16, FP32 form, "
                                   "learned rank with the search fallback"},
            "ratio": in_bytes / comp.numel(), "max_err_over_eb": err / eb, "forms": modes})
    print(json.dumps(line))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--dims", default=None, help="nx,ny,nz,nt override (profiling on a small case)")
    ap.add_argument("--form", default="learned", choices=sorted(FORMS))
    ap.add_argument("--no-plain", action="store_true", help="skip timing the plain FP64 form beside")
    ap.add_argument("--no-forms", action="store_true", help="skip timing the search and tail rank modes beside")
    ap.add_argument("--rel", type=float, default=1e-3,
                    help="absolute bound as a fraction of the value range (1e-2, 1e-3, 1e-4 in the at-scale config)")
    ap.add_argument("--sweep-precision", action="store_true",
                    help="every Gram precision mode at bounds 1e-2..1e-5 against the FP64 oracle (one JSON line)")
    ap.add_argument("--config", type=int, default=2, choices=(2, 4, 5),
                    help="4: five-variable uneven field; 5: 512^3 x 32 learned-rank evaluation (one JSON line each)")
    args = ap.parse_args()
    global DIMS, REL_BOUND
    if args.dims:
        DIMS = tuple(int(v) for v in args.dims.split(","))
    REL_BOUND = args.rel
    if args.impl == "reference":
        return run_reference(args)
    if args.sweep_precision:
        return run_precision_sweep(args)
    if args.config != 2:
        return run_config(args)

    import numpy as np
    import torch

    from paper_2601_20113_gb300 import build, dls

    rank, world, local = _rank_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    if rank == 0 or world == 1:
        build.build()
    if dist is not None:
        dist.barrier()
    field = make_field(dev, seed=SEED + 1000 * rank)
    rng = float(field.max() - field.min())
    eb = REL_BOUND * rng
    from paper_2601_20113_gb300 import train_rank
    have_model = os.path.exists(train_rank.DEFAULT_MODEL)
    if args.form == "learned" and not have_model:
        raise SystemExit("learned form needs paper_2601_20113_gb300/rank_model.bin (train_rank.py)")
    if have_model:
        dls.set_rank_model(train_rank.load_model())
    form = FORMS[args.form]
    p = dls.make_params(tuple(field.shape), torch.float32, BLOCK, eb, dls.EB_ABS, RANK_CAP,
                        precision=form[0], rank_mode=form[1])
    cap = dls.compress_bound(p)
    out = torch.empty(cap, dtype=torch.uint8, device=dev)
    ws = torch.empty(dls.workspace_size(p), dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()
    in_bytes = field.numel() * field.element_size()

    # the captured plan: occupancy form tuned per shape class, whole compression in one CUDA graph
    plan = dls.CompressPlan(p, field, out, ws, stream)
    for _ in range(args.warmup):
        nb = plan.execute(stream)
    torch.cuda.synchronize()
    clocks = Clocks(local)
    clocks.start()
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    kms = []
    phs = []
    e0.record(stream)
    for _ in range(args.steps):
        nb = plan.execute(stream)
        kms.append(plan.timing()[0])
        if args.form != "plain":
            phs.append(plan.phase_timing())
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    clk = clocks.stop()
    kernel_ms = sum(kms) / len(kms)
    phases = {k: sum(d[k] for d in phs) / len(phs) for k in phs[0]} if phs else None
    counters = dls.phase_cycles(p, ws) if args.form != "plain" else None
    graph_kernels = plan.timing()[1]
    variant, tune_ms = plan.info()
    tuning = plan.tuning()
    plan.close()
    if dist is not None:
        t = torch.tensor([ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
        dist.barrier()

    ratio = in_bytes / nb
    rec = dls.decompress(out[:nb])
    rep = dls.verify(field, rec, out[:nb])
    # decompression throughput
    d0 = torch.cuda.Event(enable_timing=True)
    d1 = torch.cuda.Event(enable_timing=True)
    d0.record(stream)
    for _ in range(args.steps):
        assert dls.decompress_into(out[:nb], rec) == 0
    d1.record(stream)
    torch.cuda.synchronize()
    dms = d0.elapsed_time(d1) / args.steps

    # end-to-end through the host-buffer entry point; the pinned buffers are
    # allocated from the CPUs of the GPU's NUMA node, so that on a machine with
    # several nodes their pages sit next to the GPU's host link
    node, keep = _pin_near_gpu(dev)
    try:
        h_in = torch.empty(field.shape, dtype=field.dtype, pin_memory=True)
        h_in.copy_(field)
        h_out = torch.empty(cap, dtype=torch.uint8, pin_memory=True)
    finally:
        if keep is not None:
            os.sched_setaffinity(0, keep)
    staging = torch.empty(dls.host_staging_size(p), dtype=torch.uint8, device=dev)
    st, enb = dls.compress_host_into(p, h_in, h_out, staging)
    assert st == 0
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    esteps = max(1, min(args.steps, 3))
    for _ in range(esteps):
        st, enb = dls.compress_host_into(p, h_in, h_out, staging)
        assert st == 0
    e2e_s = (time.perf_counter() - t0) / esteps
    del staging, h_in, h_out

    hbm, peak_kind = _peaks()
    line = {
        "metric": METRIC, "value": in_bytes * world / (ms * 1e-3) / 1e9, "unit": "GB/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64" if args.form == "plain" else "f32+f64",
        "data": "synthetic", "config": _config(args.form),
        "ratio": ratio, "max_abs_err": rep["max_abs_err"], "eb": eb, "n_over_bound": rep["n_over_bound"],
        "mean_rank": rep["mean_rank"], "decompress_gbs": in_bytes / (dms * 1e-3) / 1e9,
        "roofline": _roofline(args.form, in_bytes, nb, kernel_ms, hbm, peak_kind, DIMS, phases),
        "phases_ms": phases,
        "rank_selection": ({"accepted": counters["n_accepted"], "searched": counters["n_searched"],
                            "exact_fp64_fallbacks": counters["n_exact_fallback"]} if counters else None),
        "e2e": {"value": in_bytes * world / e2e_s / 1e9, "unit": "GB/s", "h2d_bytes_per_step": in_bytes,
                "d2h_bytes_per_step": enb, "host_numa_node": node},
        "gpu_launches": graph_kernels * args.steps,
        "plan": {"variant": variant, "tune_ms": list(tune_ms), "tuning": tuning, "kernel_ms": kernel_ms,
                 "graph_kernel_nodes": graph_kernels},
        "clocks": clk,
    }
    if args.form != "plain" and not args.no_plain:
        pp = dls.make_params(tuple(field.shape), torch.float32, BLOCK, eb, dls.EB_ABS, RANK_CAP)
        wsp = torch.empty(dls.workspace_size(pp), dtype=torch.uint8, device=dev)
        st, pnb = dls.compress_into(pp, field, out, wsp)
        assert st == 0
        p0 = torch.cuda.Event(enable_timing=True)
        p1 = torch.cuda.Event(enable_timing=True)
        p0.record(stream)
        st, pnb = dls.compress_into(pp, field, out, wsp)
        p1.record(stream)
        torch.cuda.synchronize()
        pms = p0.elapsed_time(p1)
        line["plain_fp64"] = {"value": in_bytes / (pms * 1e-3) / 1e9, "unit": "GB/s", "ratio": in_bytes / pnb,
                              "ms_per_step": pms, "speedup_of_headline": pms / ms}
        del wsp
    if args.form != "plain" and not args.no_forms:
        # the same field through the other rank modes of the FP32 form, each
        # with its own captured plan: what the network buys over the search
        # and over the eigenvalue-tail heuristic it is fed
        # (and, last, the learned form with the Rice-coded correction sections:
        # what the lossless stage costs and gains)
        line["forms"] = {}
        names = ("fp32", "tail", "learned") if have_model else ("fp32", "tail")
        for fname in names + (names[-1] + "_rice",):
            base, codec = (fname[:-5], 1) if fname.endswith("_rice") else (fname, 0)
            fp = dls.make_params(tuple(field.shape), torch.float32, BLOCK, eb, dls.EB_ABS, RANK_CAP,
                                 precision=FORMS[base][0], rank_mode=FORMS[base][1], corr_codec=codec)
            fws = torch.empty(dls.workspace_size(fp), dtype=torch.uint8, device=dev)
            fplan = dls.CompressPlan(fp, field, out, fws, stream)
            for _ in range(2):
                fplan.execute(stream)
            torch.cuda.synchronize()
            q0 = torch.cuda.Event(enable_timing=True)
            q1 = torch.cuda.Event(enable_timing=True)
            q0.record(stream)
            for _ in range(args.steps):
                fnb = fplan.execute(stream)
            q1.record(stream)
            torch.cuda.synchronize()
            fms = q0.elapsed_time(q1) / args.steps
            fc = dls.phase_cycles(fp, fws)
            line["forms"][fname] = {"ms_per_step": fms, "value": in_bytes / (fms * 1e-3) / 1e9, "unit": "GB/s",
                                    "ratio": in_bytes / fnb, "n_accepted": fc["n_accepted"],
                                    "n_searched": fc["n_searched"], "phases_ms": fplan.phase_timing()}
            fplan.close()
            del fws
    if not args.no_forms:
        line["global_basis"] = run_global_basis(dev)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        fcpu = field[:, :16, :16].cpu().numpy()
        v, cores, desc, el = oracle_sample_bench(fcpu, eb)
        line["cpu_baseline"] = {"value": v, "unit": "GB/s", "cores": cores, "kind": "oracle", "sample": desc}
    if rank == 0:
        print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
