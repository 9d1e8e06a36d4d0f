"""GPU training and inference kernels of the block-rank MLP against the CPU
oracle (oracle/mlp.py), and the learned rank mode end to end."""
import numpy as np
import pytest
import torch

from oracle import mlp
from paper_2601_20113_gb300 import dls, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2601_20113_gb300 import build
    build.build()


def _data(n, seed):
    rng = np.random.default_rng(seed)
    feat = (rng.standard_normal((n, mlp.F)) * 2 + 1).astype(np.float32)
    target = np.clip(np.rint(feat[:, 1] + 3 + 0.5 * feat[:, 2]), 0, 16).astype(np.float32)
    p = mlp.init_params(seed, feat.mean(0), feat.std(0) + 0.1)
    return feat, target, p


def test_forward_matches_oracle():
    feat, target, p = _data(300, 1)
    y = dls.mlp_forward(torch.from_numpy(p).cuda(), torch.from_numpy(feat).cuda()).cpu().numpy()
    yo, _ = mlp.forward(p, feat)
    np.testing.assert_allclose(y, yo, rtol=1e-4, atol=1e-4 * np.abs(yo).max())


@pytest.mark.parametrize("n", [128, 37, 1])
def test_gradient_matches_oracle(n):
    feat, target, p = _data(n, 2 + n)
    loss, g = dls.mlp_grad(torch.from_numpy(p).cuda(), torch.from_numpy(feat).cuda(), torch.from_numpy(target).cuda())
    lo, go = mlp.grad(p, feat, target)
    g = g.cpu().numpy()
    np.testing.assert_allclose(loss, lo, rtol=1e-5)
    np.testing.assert_allclose(g, go, rtol=1e-3, atol=2e-5 * np.abs(go).max())


def test_adam_steps_match_oracle():
    feat, target, p = _data(256, 9)
    order = np.arange(256, dtype=np.int32)
    P = torch.from_numpy(p.copy()).cuda()
    A = torch.zeros(2 * mlp.NPARAM, dtype=torch.float32, device="cuda")
    losses = dls.mlp_train(P, A, torch.from_numpy(feat).cuda(), torch.from_numpy(target).cuda(),
                           torch.from_numpy(order).cuda(), steps=4, batch=64, lr=1e-3)
    po = p.astype(np.float64)
    m = np.zeros(mlp.NPARAM)
    v = np.zeros(mlp.NPARAM)
    for s in range(4):
        idx = order[s * 64:(s + 1) * 64]
        lo, g = mlp.grad(po.astype(np.float32), feat[idx], target[idx])
        assert abs(losses[s].item() - lo) <= 1e-4 * max(1.0, lo)
        po, m, v = mlp.adam_step(po, m, v, g, s + 1, 1e-3)
    np.testing.assert_allclose(P.cpu().numpy(), po, rtol=1e-4, atol=1e-5)


def test_training_reduces_loss():
    feat, target, p = _data(4096, 4)
    order = np.random.default_rng(0).permutation(4096).astype(np.int32)
    P = torch.from_numpy(p).cuda()
    A = torch.zeros(2 * mlp.NPARAM, dtype=torch.float32, device="cuda")
    F, T, O = torch.from_numpy(feat).cuda(), torch.from_numpy(target).cuda(), torch.from_numpy(order).cuda()
    l = dls.mlp_train(P, A, F, T, O, steps=600, batch=128, lr=3e-3).cpu().numpy()
    assert l[-50:].mean() < 0.2 * l[:10].mean()


def test_learned_mode_changes_no_stored_byte():
    """With any loaded model (here an untrained one) the learned mode stores
    exactly what the bisection stores: a wrong prediction only costs time."""
    dims = (64, 64, 32, 32)
    f = synth.modes3d(*dims, seed=5, count=48).cuda()
    feat, rank = dls.block_features(f, (16, 16, 16, 16), 1e-3 * float(f.max() - f.min()))
    fe = feat.cpu().numpy()
    p = mlp.init_params(7, fe.mean(0), fe.std(0) + 1e-3)
    dls.set_rank_model(p)
    eb = 1e-3 * float(f.max() - f.min())
    a = dls.compress(f, block=(16, 16, 16, 16), eb=eb, rank_cap=16, precision=dls.PREC_FP32,
                     rank_mode=dls.RANK_SEARCH).cpu().numpy().copy()
    b = dls.compress(f, block=(16, 16, 16, 16), eb=eb, rank_cap=16, precision=dls.PREC_FP32,
                     rank_mode=dls.RANK_LEARNED).cpu().numpy().copy()
    a[67] = b[67] = 0
    assert a.size == b.size and np.array_equal(a, b)
    r = rank.cpu().numpy()
    assert r.min() >= -1 and r.max() <= 16


def _run_mode(f, eb, mode):
    p = dls.make_params(tuple(f.shape), torch.float32, (16, 16, 16, 16), eb, dls.EB_ABS, 16,
                        precision=dls.PREC_FP32, rank_mode=mode)
    out = torch.empty(dls.compress_bound(p), dtype=torch.uint8, device="cuda")
    ws = torch.empty(dls.workspace_size(p), dtype=torch.uint8, device="cuda")
    st, nb = dls.compress_into(p, f, out, ws)
    assert st == 0
    ph = dls.phase_cycles(p, ws)
    s = out[:nb].cpu().numpy().copy()
    s[67] = 0                                    # header byte: rank mode used
    return s, ph


def test_trained_model_skips_the_search():
    """What the trained network gains over the method without it.  On a field
    of the training kind but a seed outside the training set, the trained model
    predicts the rank the bisection of Algorithm 1 would choose for nearly every
    block, so those blocks take one encode pass instead of the search; an
    untrained network of the same shape gets far fewer; the stored bytes equal
    the bisection's in both cases, and the device cycles drop."""
    from paper_2601_20113_gb300 import train_rank
    f = synth.modes3d(64, 64, 64, 32, seed=48_211, count=40, noise=10 ** -2.7, device="cuda")
    eb = 10 ** -3.3 * float(f.max() - f.min())
    ref, ph_search = _run_mode(f, eb, dls.RANK_SEARCH)
    nb = ph_search["n_searched"]
    assert nb == 128 and ph_search["n_accepted"] == 0

    dls.set_rank_model(train_rank.load_model())
    got, ph_learned = _run_mode(f, eb, dls.RANK_LEARNED)
    assert np.array_equal(got, ref)
    acc_trained = ph_learned["n_accepted"] / nb
    assert acc_trained >= 0.9, acc_trained

    feat, _ = dls.block_features(f, (16, 16, 16, 16), eb)
    fe = feat.cpu().numpy()
    dls.set_rank_model(mlp.init_params(11, fe.mean(0), fe.std(0) + 1e-3))
    got_u, ph_untrained = _run_mode(f, eb, dls.RANK_LEARNED)
    assert np.array_equal(got_u, ref)
    assert ph_untrained["n_accepted"] / nb < acc_trained - 0.3

    work = ("gram", "jacobi", "refine", "rayleigh_ritz", "predict", "encode", "decide", "search", "pack")
    cyc = {k: sum(ph[x] for x in work) for k, ph in (("search", ph_search), ("learned", ph_learned))}
    print(f"accepted trained {acc_trained:.3f} untrained {ph_untrained['n_accepted'] / nb:.3f}; "
          f"cycles learned / search = {cyc['learned'] / cyc['search']:.3f}")
    assert cyc["learned"] < 0.9 * cyc["search"]
