"""Parity of the headline form (FP32 products, learned rank, captured plan)
with the oracle, where the full-size code paths run.

The FP32 form's stored modes come from a binary32 Gram matrix, so they differ
from the FP64 oracle's in the last bits, and with them every later value.  The
replay (oracle/replay.py) therefore takes each record's own stored modes and
recomputes everything else with the oracle: codes (the FP32 form's coefficient
definition, compared code for code, and each code a rounding of the FP64
projection within the binary32 evaluation bound), the rank property of
Algorithm 1's bisection, the decoded reconstruction, every correction and
escape, and the record bytes (the oracle's packer on the same inputs).  The
modes themselves are checked against the oracle's FP64 eigenproblem.  Around
that: the bound at every point and the ratio within 1% of the oracle's own
compression of the same field.
"""
import numpy as np
import pytest
import torch

import oracle
from oracle import replay
from paper_2601_20113_gb300 import dls, synth, train_rank

pytestmark = pytest.mark.gpu

BLOCK = (16, 16, 16, 16)


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2601_20113_gb300 import build
    build.build()
    oracle.build()
    dls.set_rank_model(train_rank.load_model())


def _replay_all(cfg, f, stream, coeff="f32"):
    res, errs = replay.replay_stream(cfg, f, stream, coeff=coeff)
    assert errs == [], errs
    bad = [(r["block"], r["errors"]) for r in res if r["errors"]]
    assert not bad, bad[:5]
    return res


@pytest.mark.parametrize("rel", [1e-3, 1e-4])
def test_headline_plan_replays_through_the_oracle(rel):
    """128 x 128 x 160 x 32 float32: 1280 full 16^3 x 16 blocks, more than
    the resident CTAs of the per-block kernel (so CTAs take several blocks and
    the records of most go through the deferred packer), through a captured
    plan in the FP32 form with the learned rank."""
    dims = (128, 128, 160, 32)
    fd = synth.modes3d(*dims, seed=31, count=64, device="cuda")
    f = fd.cpu().numpy()
    eb = rel * float(f.max() - f.min())
    p = dls.make_params(tuple(fd.shape), torch.float32, BLOCK, eb, dls.EB_ABS, 16, precision=dls.PREC_FP32,
                        rank_mode=dls.RANK_LEARNED)
    out = torch.empty(dls.compress_bound(p), dtype=torch.uint8, device="cuda")
    ws = torch.empty(dls.workspace_size(p), dtype=torch.uint8, device="cuda")
    plan = dls.CompressPlan(p, fd, out, ws)
    nb = plan.execute()
    plan.close()
    comp = out[:nb].clone()
    # every point within the bound, on the GPU decoder
    rec = dls.decompress(comp)
    assert (rec.double() - fd.double()).abs().max().item() <= eb
    # ratio within 1% of the oracle's on the same field
    cfg = oracle.Config(dims, BLOCK, oracle.F32, eb=eb, rank_cap=16)
    st, ref, _ = oracle.compress(cfg, f)
    assert st == oracle.OK
    assert abs(ref.size / nb - 1) <= 0.01, (nb, ref.size)
    # every record, replayed
    s = comp.cpu().numpy()
    res = _replay_all(cfg, f, s)
    assert oracle.num_blocks(cfg) == len(res) == 1280
    assert sum(r["raw"] for r in res) == 0
    assert sum(r["dense"] for r in res) + sum(r["sparse"] for r in res) > 0
    # the oracle's decoder reads the GPU stream into the GPU decoder's field
    st, rref = oracle.decompress(s)
    assert st == oracle.OK and np.array_equal(rref.astype(np.float32), rec.cpu().numpy())


@pytest.mark.parametrize("path", [dls.CORR_PATH_SPARSE, dls.CORR_PATH_DENSE])
@pytest.mark.parametrize("eb", [1e-3, 3.7e-2, 2.5e-5])
def test_stage_correction_paths_bit_exact(eb, path):
    """The per-block kernel's own correction code (candidate filter, FP32 test,
    FP64 definition where the test cannot decide) on residuals placed on and
    around the decision points, against the oracle's FP64 definition."""
    rng = np.random.default_rng(int(eb * 1e6) % 991 + path)
    n = 40000
    x = (rng.standard_normal(n) * 2.0).astype(np.float32)
    kk = rng.integers(-3, 4, size=n)
    r = (kk * 2 * eb + np.where(rng.random(n) < 0.5, eb, -eb)).astype(np.float64)
    xh = (x.astype(np.float64) - r).astype(np.float32)
    for s in range(1, 3):
        m = rng.random(n) < 0.2
        xh[m] = np.nextafter(xh[m], np.float32(np.inf) if s == 1 else np.float32(-np.inf))
    q = n // 10
    xh[:q] = (x[:q].astype(np.float64) - rng.uniform(-3 * eb, 3 * eb, q)).astype(np.float32)
    # residuals just below and above the candidate threshold eb (1 - 1e-6)
    t = (x[q:2 * q].astype(np.float64) - eb * (1.0 + rng.uniform(-3e-6, 3e-6, q))).astype(np.float32)
    xh[q:2 * q] = t
    xh[2 * q:2 * q + 100] = x[2 * q:2 * q + 100] + np.float32(1e9 * eb)        # beyond 2^20 steps
    k = dls.stage_correct_path(torch.from_numpy(x).cuda(), torch.from_numpy(xh).cuda(), eb, path).cpu().numpy()
    ko, esc = oracle.correct(x.astype(np.float64)[:, None], xh.astype(np.float64)[:, None], 0, n,
                             oracle.F32, eb, 2 * eb)
    esc = esc.astype(bool)
    np.testing.assert_array_equal(k == np.iinfo(np.int32).min, esc)
    np.testing.assert_array_equal(k[~esc], ko[~esc])


def test_withheld_chunk_times_out_and_the_next_call_succeeds():
    """A chunk copy that never arrives (a host-set hook, no GPU fault): the
    bounded wait runs out, the call returns DLS_ERR_TIMEOUT, and the next call
    on the same workspace gives the reference stream."""
    dims = (64, 64, 32, 32)
    fd = synth.modes3d(*dims, seed=4, count=24, device="cuda")
    eb = 1e-3 * float(fd.max() - fd.min())
    p = dls.make_params(tuple(fd.shape), torch.float32, BLOCK, eb, dls.EB_ABS, 16, precision=dls.PREC_FP32,
                        rank_mode=dls.RANK_TAIL)
    out = torch.empty(dls.compress_bound(p), dtype=torch.uint8, device="cuda")
    ws = torch.empty(dls.workspace_size(p), dtype=torch.uint8, device="cuda")
    st, nb = dls.compress_into(p, fd, out, ws)
    assert st == dls.OK
    ref = out[:nb].cpu().numpy().copy()
    assert dls.set_fault_hook(dls.FAULT_WITHHOLD_CHUNK, 3) == dls.OK
    try:
        st, _ = dls.compress_into(p, fd, out, ws)
    finally:
        assert dls.set_fault_hook(dls.FAULT_NONE, 0) == dls.OK
    assert st == dls.ERR_TIMEOUT, dls.status_string(st)
    torch.cuda.synchronize()
    st, nb2 = dls.compress_into(p, fd, out, ws)
    assert st == dls.OK and nb2 == nb and np.array_equal(out[:nb2].cpu().numpy(), ref)
