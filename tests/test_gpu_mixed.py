"""Mixed-precision form (FP32 products, FP64-accurate eigenbasis, FP64-semantics
decisions) against the CPU oracle, through the C ABI.

Stage tests feed identical inputs to the GPU's FP32-filtered decisions and to
the oracle's FP64 definitions and require identical results, with inputs placed
on the rounding boundaries where a filter could go wrong.  End-to-end tests
require the pointwise bound at every point and the compression ratio within 1%
of the oracle's, and replay every record through the oracle from its own
stored modes (oracle/replay.py): codes, rank, corrections, escapes and record
bytes must match exactly.
"""
import numpy as np
import pytest
import torch

import oracle
from oracle import replay
from paper_2601_20113_gb300 import dls, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2601_20113_gb300 import build
    build.build()
    oracle.build()


def _adversarial_coeffs(delta, n, seed):
    rng = np.random.default_rng(seed)
    k = rng.integers(-20000, 20000, size=n).astype(np.float64)
    base = (k + 0.5) * delta                              # exact half-way points
    c = base.astype(np.float32)
    # nudge by a few ulps around the half-way points
    nud = rng.integers(-3, 4, size=n).astype(np.int32)
    for s in range(1, 4):
        m = nud == s
        c[m] = np.nextafter(c[m], np.float32(np.inf))
        m = nud == -s
        c[m] = np.nextafter(c[m], np.float32(-np.inf))
    ints = (rng.integers(-1000, 1000, size=n) * delta).astype(np.float32)
    rnd = (rng.standard_normal(n) * 300 * delta).astype(np.float32)
    big = ((2.0 ** 24 + rng.integers(-4, 4, size=n)) * delta).astype(np.float32)
    return np.concatenate([c, ints, rnd, big, -big])


@pytest.mark.parametrize("delta", [1e-3, 7.3e-4, 0.25, 3.1e-7])
def test_stage_quantizer_bit_exact(delta):
    c = _adversarial_coeffs(delta, 20000, seed=int(delta * 1e7) % 1000)
    q, ovf = dls.stage_quantize(torch.from_numpy(c).cuda(), delta)
    qo, _ = oracle.quantize(c.astype(np.float64), delta, oracle.F32)
    y = c.astype(np.float64) / delta
    ovf_o = ~(np.abs(y) < 2.0 ** 24)
    qg = q.cpu().numpy()
    og = ovf.cpu().numpy().astype(bool)
    np.testing.assert_array_equal(og, ovf_o)
    np.testing.assert_array_equal(qg[~ovf_o], qo[~ovf_o])


@pytest.mark.parametrize("eb", [1e-3, 3.7e-2, 2.5e-5])
def test_stage_correction_bit_exact(eb):
    rng = np.random.default_rng(int(eb * 1e6) % 997)
    n = 30000
    x = (rng.standard_normal(n) * 2.0).astype(np.float32)
    # residuals on and around the decision points |R| = eb, 3eb, 5eb and far
    kk = rng.integers(-3, 4, size=n)
    r = (kk * 2 * eb + np.where(rng.random(n) < 0.5, eb, -eb)).astype(np.float64)
    xh = (x.astype(np.float64) - r).astype(np.float32)
    for s in range(1, 3):
        m = rng.random(n) < 0.2
        xh[m] = np.nextafter(xh[m], np.float32(np.inf) if s == 1 else np.float32(-np.inf))
    xh[: n // 10] = (x[: n // 10].astype(np.float64) - rng.uniform(-3 * eb, 3 * eb, n // 10)).astype(np.float32)
    xh[n // 10: n // 10 + 100] = x[n // 10: n // 10 + 100] + np.float32(1e9 * eb)     # beyond 2^20 steps
    k = dls.stage_correct(torch.from_numpy(x).cuda(), torch.from_numpy(xh).cuda(), eb).cpu().numpy()
    ko, esc = oracle.correct(x.astype(np.float64)[:, None], xh.astype(np.float64)[:, None], 0, n,
                             oracle.F32, eb, 2 * eb)
    esc = esc.astype(bool)
    np.testing.assert_array_equal(k == np.iinfo(np.int32).min, esc)
    np.testing.assert_array_equal(k[~esc], ko[~esc])


def _mixed_vs_oracle(f, dims, block, eb, eb_type=oracle.EB_ABS, rank_cap=16, nvars=1, rank_mode=dls.RANK_SEARCH):
    cfg = oracle.Config(dims, block, oracle.F32, eb=eb, eb_type=eb_type, rank_cap=rank_cap, nvars=nvars)
    st, ref, trs = oracle.compress(cfg, f, traces=True)
    assert st == 0
    fd = torch.from_numpy(np.ascontiguousarray(f)).cuda()
    comp = dls.compress(fd, block=block, eb=eb, eb_type=eb_type, rank_cap=rank_cap, precision=dls.PREC_FP32,
                        rank_mode=rank_mode)
    rec = dls.decompress(comp)
    return ref, comp, rec, fd, trs


@pytest.mark.parametrize("rel", [1e-2, 1e-3, 1e-4, 1e-5])
def test_mixed_bound_and_ratio(rel):
    dims = (40, 36, 20, 36)
    f = synth.modes3d(*dims, seed=2, count=32).numpy()
    eb = rel * float(f.max() - f.min())
    ref, comp, rec, fd, trs = _mixed_vs_oracle(f, dims, (16, 16, 16, 16), eb)
    err = (rec.double() - fd.double()).abs().max().item()
    assert err <= eb
    ratio_gpu = f.nbytes / comp.numel()
    ratio_ref = f.nbytes / ref.size
    assert abs(ratio_gpu / ratio_ref - 1) <= 0.01, (ratio_gpu, ratio_ref)
    # every record replayed through the oracle from its own stored modes
    # (codes, rank property, corrections, escapes and record bytes exact)
    cfg = oracle.Config(dims, (16, 16, 16, 16), oracle.F32, eb=eb, rank_cap=16)
    res, errs = replay.replay_stream(cfg, f, comp.cpu().numpy())
    assert errs == [] and all(r["errors"] == [] for r in res), [r["errors"] for r in res if r["errors"]][:3]


def _same_payload(a, b):
    """Streams equal except header byte 67 (the rank mode used)."""
    a = a.cpu().numpy().copy()
    b = b.cpu().numpy().copy()
    a[67] = b[67] = 0
    return a.size == b.size and np.array_equal(a, b)


def test_predicted_rank_equals_search_stream():
    """A predicted rank is accepted only when it is the smallest passing rank
    next to the prediction, so the prediction changes no stored byte."""
    dims = (64, 64, 32, 32)
    f = synth.modes3d(*dims, seed=5, count=48)
    fd = f.cuda()
    for rel in (1e-2, 1e-3, 1e-4):
        eb = rel * float(f.max() - f.min())
        a = dls.compress(fd, block=(16, 16, 16, 16), eb=eb, rank_cap=16, precision=dls.PREC_FP32,
                         rank_mode=dls.RANK_SEARCH)
        b = dls.compress(fd, block=(16, 16, 16, 16), eb=eb, rank_cap=16, precision=dls.PREC_FP32,
                         rank_mode=dls.RANK_TAIL)
        assert _same_payload(a, b)


def test_mixed_multivariable_uneven_blocks():
    """Five variables with edge blocks on every axis (T = 2 and short spatial
    edges), per-variable relative bounds."""
    f = synth.multivar(50, 38, 26, 18).numpy()
    ebs = [1e-3, 1e-3, 1e-3, 1e-4, 1e-4]
    cfg = oracle.Config((50, 38, 26, 18), (16, 16, 16, 16), oracle.F32, eb=ebs, eb_type=oracle.EB_REL_RANGE,
                        rank_cap=16, nvars=5)
    st, ref, _ = oracle.compress(cfg, f)
    fd = torch.from_numpy(f).cuda()
    comp = dls.compress(fd, block=(16, 16, 16, 16), eb=ebs, eb_type=dls.EB_REL_RANGE, rank_cap=16,
                        precision=dls.PREC_FP32, rank_mode=dls.RANK_TAIL)
    rec = dls.decompress(comp)
    x = f.astype(np.float64)
    y = rec.cpu().numpy().astype(np.float64)
    for v in range(5):
        assert np.abs(y[v] - x[v]).max() <= ebs[v] * (x[v].max() - x[v].min())
    assert abs((f.nbytes / comp.numel()) / (f.nbytes / ref.size) - 1) <= 0.01
    res, errs = replay.replay_stream(cfg, f, comp.cpu().numpy())
    assert errs == [] and all(r["errors"] == [] for r in res), [r["errors"] for r in res if r["errors"]][:3]


def test_mixed_nrmse_mode():
    dims = (32, 32, 16, 32)
    f = synth.modes3d(*dims, seed=7, count=16).numpy()
    fd = torch.from_numpy(f).cuda()
    for eps in (0.5, 2.0):
        comp = dls.compress(fd, block=(16, 16, 8, 16), eb=eps, eb_type=dls.EB_NRMSE, precision=dls.PREC_FP32,
                            rank_mode=dls.RANK_TAIL)
        rec = dls.decompress(comp)
        x = f.astype(np.float64)
        assert 100 * np.linalg.norm(rec.cpu().numpy() - x) / np.linalg.norm(x) <= eps


def test_mixed_mode_on_f64_field_takes_fp64_form():
    f = synth.vortex2d(64, 64, 32, seed=1).numpy()
    eb = 1e-3 * float(f.max() - f.min())
    cfg = oracle.Config((64, 64, 1, 32), (8, 8, 1, 32), oracle.F64, eb=eb, rank_cap=16)
    st, ref, _ = oracle.compress(cfg, f)
    comp = dls.compress(torch.from_numpy(f).cuda(), block=(8, 8, 1, 32), eb=eb, rank_cap=16,
                        precision=dls.PREC_FP32)
    got = comp.cpu().numpy()
    assert got.size == ref.size and np.array_equal(got[128:], ref[128:])   # header differs in the precision byte


# Tensor-core Gram modes: (precision, relative error of each product's operands,
# allowed ratio deviation from the FP64 oracle).  The split modes keep the
# ratio within 1% of the oracle's; the one-term modes (10- and 8-bit
# mantissas) are allowed a few percent: their bases come from a coarser Gram.
TC_MODES = [(dls.PREC_TF32X3, 2.0 ** -21, 0.01), (dls.PREC_BF16X3, 2.0 ** -16, 0.01),
            (dls.PREC_TF32, 2.0 ** -11, 0.05), (dls.PREC_BF16, 2.0 ** -8, 0.10)]


@pytest.mark.parametrize("mode,u_prod,tol", TC_MODES)
@pytest.mark.parametrize("rel", [1e-2, 1e-3, 1e-4])
def test_tensor_core_gram_modes(rel, mode, u_prod, tol):
    """Gram on the tensor cores (tcgen05; kind::tf32 for the TF32 modes,
    kind::f16 for the BF16 ones): every block's Gram runs there (counter), the
    bound holds at every point, every record replays exactly through the
    oracle (its modes within the Gram perturbation bound of the mode) and the
    ratio stays within the mode's tolerance of the oracle's."""
    dims = (64, 48, 32, 40)                     # edge blocks in z (0) and t (8 steps)
    f = synth.modes3d(*dims, seed=21, count=32).numpy()
    eb = rel * float(f.max() - f.min())
    cfg = oracle.Config(dims, (16, 16, 16, 16), oracle.F32, eb=eb, rank_cap=16)
    st, ref, _ = oracle.compress(cfg, f)
    fd = torch.from_numpy(f).cuda()
    p = dls.make_params(tuple(f.shape), torch.float32, (16, 16, 16, 16), eb, dls.EB_ABS, 16,
                        precision=mode, rank_mode=dls.RANK_TAIL)
    out = torch.empty(dls.compress_bound(p), dtype=torch.uint8, device="cuda")
    ws = torch.empty(dls.workspace_size(p), dtype=torch.uint8, device="cuda")
    st, nb = dls.compress_into(p, fd, out, ws)
    assert st == 0
    ph = dls.phase_cycles(p, ws)
    assert ph["n_tensor_core_gram"] == oracle.num_blocks(cfg)
    rec = dls.decompress(out[:nb])
    assert (rec.double() - fd.double()).abs().max().item() <= eb
    assert abs((f.nbytes / nb) / (f.nbytes / ref.size) - 1) <= tol, (f.nbytes / nb, f.nbytes / ref.size)
    res, errs = replay.replay_stream(cfg, f, out[:nb].cpu().numpy(), u_prod=u_prod)
    assert errs == [] and all(r["errors"] == [] for r in res), [r["errors"] for r in res if r["errors"]][:3]


def test_mixed_both_block_sides():
    """Edge blocks of 2 x 4 x 1 points over 16 steps take the spatial Gram side
    (M = 8 < T = 16) while the full 4 x 4 x 1 blocks tie and take time; both
    kinds run in one call."""
    dims = (10, 8, 3, 32)
    f = synth.modes3d(*dims, seed=11, count=8).numpy()
    eb = 1e-3 * float(f.max() - f.min())
    ref, comp, rec, fd, _ = _mixed_vs_oracle(f, dims, (4, 4, 1, 16), eb)
    assert (rec.double() - fd.double()).abs().max().item() <= eb
    assert abs((f.nbytes / comp.numel()) / (f.nbytes / ref.size) - 1) <= 0.01
    cfg = oracle.Config(dims, (4, 4, 1, 16), oracle.F32, eb=eb, rank_cap=16)
    res, errs = replay.replay_stream(cfg, f, comp.cpu().numpy())
    assert errs == [] and all(r["errors"] == [] for r in res), [r["errors"] for r in res if r["errors"]][:3]


@pytest.mark.parametrize("dims,block", [((48, 20, 20, 16), (12, 8, 8, 16)),     # TMA, several z-planes per chunk
                                        ((37, 21, 9, 20), (16, 16, 8, 16)),     # TMA on the pitched copy, ragged edges
                                        ((37, 21, 9, 20), (10, 8, 8, 16)),      # cp.async, 4 bytes (odd x extent)
                                        ((38, 21, 9, 20), (10, 8, 8, 16)),      # cp.async, pairs of floats
                                        ((64, 64, 16, 40), (16, 16, 16, 16))])  # T edge of 8 steps
def test_mixed_chunk_shapes(dims, block):
    f = synth.modes3d(*dims, seed=13, count=24).numpy()
    eb = 1e-3 * float(f.max() - f.min())
    ref, comp, rec, fd, _ = _mixed_vs_oracle(f, dims, block, eb, rank_mode=dls.RANK_TAIL)
    assert (rec.double() - fd.double()).abs().max().item() <= eb
    assert abs((f.nbytes / comp.numel()) / (f.nbytes / ref.size) - 1) <= 0.01
    cfg = oracle.Config(dims, block, oracle.F32, eb=eb, rank_cap=16)
    res, errs = replay.replay_stream(cfg, f, comp.cpu().numpy())
    assert errs == [] and all(r["errors"] == [] for r in res), [r["errors"] for r in res if r["errors"]][:3]


def _record_escapes(comp):
    """Escape count of every record (record header word 2)."""
    s = comp.cpu().numpy()
    b0, b1, offp, payp = (int(s[o:o + 8].view(np.uint64)[0]) for o in (72, 80, 104, 112))
    offs = s[offp:offp + 8 * (b1 - b0 + 1)].view(np.uint64)
    return [int(s[payp + int(o) + 8:payp + int(o) + 12].view(np.uint32)[0]) for o in offs[:-1]]


@pytest.mark.parametrize("rank_mode", [dls.RANK_SEARCH, dls.RANK_TAIL])
def test_mixed_escapes_on_full_blocks(rank_mode):
    """A correction beyond 2^20 steps is stored as an escape (raw value).  Full
    16^3 x 16 blocks write their corrections through the nonzero-correction
    bitmap; a block with escapes is encoded again with every element written,
    and its stream must decode within the bound, identically on both decoders."""
    dims = (32, 32, 16, 16)
    f = synth.modes3d(*dims, seed=7, count=16)
    # two spikes in block 0 at different time steps: a rank-1 basis keeps the
    # larger, and the other one's residual (5e3 / 2e-3 steps) must escape
    # (at rank 1 every element is corrected, and a few corrected values land
    # beyond eb by rounding: those escape too, in every block, as in the oracle)
    f[0, 3, 2, 5, 7] = 1.0e4
    f[0, 9, 4, 11, 13] = 5.0e3
    eb = 1e-3
    fd = f.cuda()
    comp = dls.compress(fd, block=(16, 16, 16, 16), eb=eb, rank_cap=1, precision=dls.PREC_FP32,
                        rank_mode=rank_mode)
    esc = _record_escapes(comp)
    assert esc[0] >= 1, esc
    rec = dls.decompress(comp)
    assert (rec.double() - fd.double()).abs().max().item() <= eb
    # an escape stores the raw value: the spike comes back exactly
    assert rec[0, 9, 4, 11, 13].item() == 5.0e3
    st, rref = oracle.decompress(comp.cpu().numpy())
    assert st == oracle.OK
    assert np.array_equal(rref.astype(np.float32), rec.cpu().numpy())


def test_mixed_stream_is_deterministic():
    """More blocks than resident CTAs: each CTA takes several blocks in an order
    that changes from run to run; every stored byte depends on the block alone."""
    f = synth.modes3d(128, 128, 128, 32, seed=9, count=48, device="cuda")
    eb = 1e-3 * float(f.max() - f.min())
    runs = [dls.compress(f, block=(16, 16, 16, 16), eb=eb, rank_cap=16, precision=dls.PREC_FP32,
                         rank_mode=dls.RANK_TAIL).cpu().numpy() for _ in range(3)]
    assert all(r.size == runs[0].size and np.array_equal(r, runs[0]) for r in runs[1:])


def test_mixed_escapes_in_deferred_records():
    """A full block whose record the deferred packer writes can carry escapes:
    the encode pass lists them as it finds them, in no particular order, and
    the packer writes them in element order with their raw values."""
    dims = (32, 32, 16, 16)
    f = torch.zeros((1, dims[3], dims[2], dims[1], dims[0]), dtype=torch.float32)
    # four spikes in block 0 at different time steps: a rank-1 basis keeps
    # the largest, the other three need more than 2^20 steps of 2 eb and
    # escape; the field is zero elsewhere, so no correction widens the record
    # beyond what the deferred packer takes
    spikes = [((2, 3, 5, 7), 1.0e4), ((5, 11, 2, 9), 3.0e3), ((9, 4, 13, 1), 2.6e3), ((12, 8, 8, 14), 2.2e3)]
    for (t, z, y, x), v in spikes:
        f[0, t, z, y, x] = v
    eb = 1e-3
    fd = f.cuda()
    comp = dls.compress(fd, block=(16, 16, 16, 16), eb=eb, rank_cap=1, precision=dls.PREC_FP32,
                        rank_mode=dls.RANK_SEARCH)
    esc = _record_escapes(comp)
    assert esc[0] == 3 and sum(esc[1:]) == 0, esc
    rec = dls.decompress(comp)
    assert (rec.double() - fd.double()).abs().max().item() <= eb
    for (t, z, y, x), v in spikes[1:]:
        assert rec[0, t, z, y, x].item() == v
    st, rref = oracle.decompress(comp.cpu().numpy())
    assert st == oracle.OK
    assert np.array_equal(rref.astype(np.float32), rec.cpu().numpy())
    # the escape-carrying deferred record, byte for byte against the oracle's packer
    cfg = oracle.Config(dims, (16, 16, 16, 16), oracle.F32, eb=eb, rank_cap=1)
    res, errs = replay.replay_stream(cfg, f.numpy(), comp.cpu().numpy())
    assert errs == [] and all(r["errors"] == [] for r in res), [r["errors"] for r in res if r["errors"]][:3]
    assert res[0]["nesc"] == 3


@pytest.mark.parametrize("nvars,eb_type", [(1, dls.EB_ABS), (2, dls.EB_ABS), (2, dls.EB_REL_RANGE)])
def test_host_entry_matches_device_entry(nvars, eb_type):
    """dls_compress_host on pinned host buffers gives the device entry's stream
    byte for byte.  With an absolute bound the copy of each (variable, time
    block) slab overlaps the compression of the slabs before it; a bound
    relative to the range needs the whole field first."""
    dims = (64, 64, 32, 48)                         # three time blocks of 16
    f = torch.cat([synth.modes3d(*dims, seed=11 + v, count=24) for v in range(nvars)], 0).contiguous()
    eb = 1e-3 * float(f.max() - f.min()) if eb_type == dls.EB_ABS else 1e-3
    ref = dls.compress(f.cuda(), block=(16, 16, 16, 16), eb=eb, eb_type=eb_type, rank_cap=16,
                       precision=dls.PREC_FP32, rank_mode=dls.RANK_SEARCH).cpu().numpy()
    p = dls.make_params(tuple(f.shape), torch.float32, (16, 16, 16, 16), eb, eb_type, 16,
                        precision=dls.PREC_FP32, rank_mode=dls.RANK_SEARCH)
    h_in = f.pin_memory()
    h_out = torch.empty(dls.compress_bound(p), dtype=torch.uint8).pin_memory()
    staging = torch.empty(dls.host_staging_size(p), dtype=torch.uint8, device="cuda")
    for _ in range(2):
        st, nb = dls.compress_host_into(p, h_in, h_out, staging)
        assert st == 0
        assert nb == ref.size and np.array_equal(h_out[:nb].numpy(), ref)


@pytest.mark.parametrize("dims", [(50, 38, 26, 48), (37, 21, 20, 32)])
def test_pitched_copy_matches_direct_reads(dims):
    """A field whose x extent is not a multiple of 4 floats: the device entry
    stages its chunks by TMA from a pitched copy of the field, the host entry's
    slab-by-slab launches read the field itself by cp.async; the two streams
    are byte-identical, and the oracle decodes the same field."""
    f = torch.cat([synth.modes3d(*dims, seed=61 + v, count=24) for v in range(2)], 0).contiguous()
    eb = 1e-3 * float(f.max() - f.min())
    p = dls.make_params(tuple(f.shape), torch.float32, (16, 16, 16, 16), eb, dls.EB_ABS, 16,
                        precision=dls.PREC_FP32, rank_mode=dls.RANK_TAIL)
    ref = dls.compress(f.cuda(), block=(16, 16, 16, 16), eb=eb, rank_cap=16, precision=dls.PREC_FP32,
                       rank_mode=dls.RANK_TAIL).cpu().numpy()
    h_in = f.pin_memory()
    h_out = torch.empty(dls.compress_bound(p), dtype=torch.uint8).pin_memory()
    staging = torch.empty(dls.host_staging_size(p), dtype=torch.uint8, device="cuda")
    st, nb = dls.compress_host_into(p, h_in, h_out, staging)
    assert st == 0 and nb == ref.size and np.array_equal(h_out[:nb].numpy(), ref)
    cfg = oracle.Config(dims, (16, 16, 16, 16), oracle.F32, eb=eb, rank_cap=16, nvars=2)
    res, errs = replay.replay_stream(cfg, f.numpy(), ref)
    assert errs == [] and all(r["errors"] == [] for r in res), [r["errors"] for r in res if r["errors"]][:3]
