"""The oracle's record parser and stream replay (CPU only).

The replay is what the GPU parity tests of the FP32 form use: it recomputes
every part of a record from the block's data and the record's own stored modes.
Here it is pinned on streams the oracle itself wrote, and on records with one
planted mistake each, which it must report.
"""
import numpy as np
import pytest

import oracle
from oracle import replay
from paper_2601_20113_gb300 import synth


@pytest.fixture(scope="module")
def case():
    dims = (48, 32, 32, 32)                   # 3 x 2 x 2 x 2 = 24 blocks of 16^3 x 16
    f = synth.modes3d(*dims, seed=3, count=32).numpy()
    eb = 1e-3 * float(f.max() - f.min())
    cfg = oracle.Config(dims, (16, 16, 16, 16), oracle.F32, eb=eb, rank_cap=16)
    st, s, trs = oracle.compress(cfg, f, traces=True)
    assert st == oracle.OK
    return cfg, f, s, trs


def test_parse_inverts_pack():
    """parse_record(pack_record(r, Vst, q, k, esc, A)) gives back every input,
    for a dense, a sparse, an escape-carrying and a spatial-side record."""
    rng = np.random.default_rng(4)
    for side, n, L, M, dense, nesc in [(0, 8, 64, 64, True, 0), (0, 8, 64, 64, False, 0), (0, 4, 32, 32, False, 3),
                                       (1, 6, 10, 6, True, 2)]:
        N = L * n
        r = 3
        Vst = rng.standard_normal((n, r)).astype(np.float32).astype(np.float64)
        q = rng.integers(-500, 500, size=(L, r)).astype(np.int32)
        k = np.zeros(N, np.int32)
        nz = rng.choice(N, size=N // 2 if dense else N // 20, replace=False)
        k[nz] = rng.integers(-3, 4, size=nz.size)
        esc = np.zeros(N, np.uint8)
        esc[rng.choice(N, size=nesc, replace=False)] = 1
        k[esc.astype(bool)] = 0
        A = rng.standard_normal((L, n)).astype(np.float32).astype(np.float64)
        rec = oracle.pack_record(r, side, n, L, M, oracle.F32, Vst, q, k, esc, A)
        p = oracle.parse_record(rec, side, n, L, M, oracle.F32)
        assert p is not None and p["r"] == r
        assert bool(p["flags"] & 4) == (bool(dense) and np.count_nonzero(k) > 0 and
                                        (rec[1] & 4) != 0)
        np.testing.assert_array_equal(p["Vst"], Vst)
        np.testing.assert_array_equal(p["q"], q)
        np.testing.assert_array_equal(p["k"], k)
        np.testing.assert_array_equal(p["esc"], esc.astype(bool))
        e = np.flatnonzero(esc)
        xe = A.T.reshape(-1) if side == 0 else A.reshape(-1)
        np.testing.assert_array_equal(p["escval"][e], xe[e])
        # a truncated or resized record does not parse
        assert oracle.parse_record(rec[:-16], side, n, L, M, oracle.F32) is None
        bad = bytearray(rec)
        bad[3] ^= 1                                   # index width
        assert oracle.parse_record(bytes(bad), side, n, L, M, oracle.F32) is None


def test_replay_accepts_the_oracles_own_stream(case):
    cfg, f, s, trs = case
    res, errs = replay.replay_stream(cfg, f, s, coeff="f64")
    assert errs == []
    assert all(r["errors"] == [] for r in res), [r["errors"] for r in res if r["errors"]]
    assert [r["r"] for r in res] == [t.r for t in trs]
    assert max(r["orth"] for r in res) <= 4e-7
    assert max(r["lam_err"] for r in res) <= 1.0


def _replay_one(cfg, f, s, i, rec):
    sb, h = replay.parse_stream(s)
    b = h["block_begin"] + i
    return replay.replay_block(cfg, f, b, rec, float(h["eb"][0]), float(h["delta"][0]), float(h["step"][0]),
                               coeff="f64")


def _repacked(cfg, b, p, A):
    g = oracle.block_geom(cfg, b)
    return oracle.pack_record(p["r"], g.side, g.n, g.L, g.M, cfg.dtype, p["Vst"], p["q"], p["k"],
                              p["esc"].astype(np.uint8), A)


def test_replay_reports_planted_mistakes(case):
    cfg, f, s, trs = case
    sb, h = replay.parse_stream(s)
    i = next(j for j, t in enumerate(trs) if t.r >= 2 and t.n_corr > 0)
    rec = bytes(replay.record_of(sb, h, i))
    g = oracle.block_geom(cfg, i)
    A = oracle.gather(cfg, f, i)
    base = oracle.parse_record(rec, g.side, g.n, g.L, g.M, cfg.dtype)
    assert _replay_one(cfg, f, s, i, rec)["errors"] == []

    def errors_after(mut):
        p = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in base.items()}
        mut(p)
        return _replay_one(cfg, f, s, i, _repacked(cfg, i, p, A))["errors"]

    def code(p):                                     # one code off by one
        p["q"][5, 0] += 1
    def corr(p):                                     # one correction changed
        e = int(np.flatnonzero(p["k"])[0])
        p["k"][e] += 1
    def rank_up(p):                                  # one (zero) mode more than needed
        p["Vst"] = np.column_stack([p["Vst"], np.zeros(g.n)])
        p["q"] = np.column_stack([p["q"], np.zeros(g.L, np.int32)])
        p["r"] += 1
    def sign(p):                                     # a stored mode with its sign flipped
        p["Vst"][:, 0] = -p["Vst"][:, 0]
    assert any("codes differ" in e for e in errors_after(code))
    assert any("corrections differ" in e for e in errors_after(corr))
    assert any("pass(r - 1)" in e for e in errors_after(rank_up))
    assert errors_after(sign) != []
    # a byte of padding changed: the repacked record differs
    pad = bytearray(rec)
    pad[-1] ^= 0xFF
    assert _replay_one(cfg, f, s, i, bytes(pad))["errors"] != []


def _rn32(x):
    """Exact rational x rounded to the nearest binary32 (ties to even), for
    normal-range values: one rounding, as an fma does."""
    from fractions import Fraction
    x = Fraction(x)
    if x == 0:
        return 0.0
    a = abs(x)
    e = a.numerator.bit_length() - a.denominator.bit_length()
    if Fraction(2) ** e > a:
        e -= 1
    ulp = Fraction(2) ** (e - 23)
    m = a / ulp
    fl = m.numerator // m.denominator
    rem = m - fl
    if rem > Fraction(1, 2) or (rem == Fraction(1, 2) and fl % 2 == 1):
        fl += 1
    v = float(fl * ulp)
    return v if x > 0 else -v


def test_fp32_coefficients_match_binary32_evaluation():
    """project_f32 is the shifted projection in binary32 in its fixed order:
    checked against an exact-rational evaluation of that definition, every
    subtraction, fma and addition rounded once to binary32."""
    from fractions import Fraction as F
    rng = np.random.default_rng(8)
    for n in (16, 7):
        A = (rng.standard_normal((20, n)) * 3 + 100).astype(np.float32).astype(np.float64)
        V = rng.standard_normal((n, 3)).astype(np.float32).astype(np.float64)
        got = oracle.project_f32(A, V)
        for k in range(3):
            vs = float(np.float32(sum(float(v) for v in V[:, k])))     # double sum, one rounding
            for l in range(20):
                a0 = A[l, 0]
                s = [0.0] * 4
                for j in range(n):
                    d = _rn32(F(A[l, j]) - F(a0))
                    s[j & 3] = _rn32(F(d) * F(V[j, k]) + F(s[j & 3]))
                tot = _rn32(F(_rn32(F(s[0]) + F(s[1]))) + F(_rn32(F(s[2]) + F(s[3]))))
                ref = _rn32(F(a0) * F(vs) + F(tot))
                assert got[l, k] == ref, (n, k, l, got[l, k], ref)
        # and it is the FP64 projection up to binary32 evaluation error
        C64 = oracle.project(A, V)
        assert np.abs(got - C64).max() <= 1e-4 * np.abs(A).max() * np.abs(V).sum(0).max()


def test_replay_reads_rice_coded_records():
    """With the Rice-coded correction section asked for, the oracle's own
    stream (Rice where smaller) parses and replays; the parser recovers the
    corrections the plain stream carries, record for record."""
    dims = (48, 48, 32, 32)
    f = synth.modes3d(*dims, seed=2, count=64).numpy()
    eb = 1e-3 * float(f.max() - f.min())
    cfg = oracle.Config(dims, (16, 16, 16, 16), oracle.F32, eb=eb, rank_cap=16)
    cfg_r = oracle.Config(dims, (16, 16, 16, 16), oracle.F32, eb=eb, rank_cap=16, corr_codec=1)
    st, s, trs = oracle.compress(cfg, f, traces=True)
    assert st == oracle.OK
    st, sr, _ = oracle.compress(cfg_r, f)
    assert st == oracle.OK and sr.size < s.size
    res, errs = replay.replay_stream(cfg_r, f, sr, coeff="f64")
    assert errs == [] and all(r["errors"] == [] for r in res)
    a, ha = replay.parse_stream(s)
    b, hb = replay.parse_stream(sr)
    nrice = 0
    for i in range(len(trs)):
        g = oracle.block_geom(cfg, i)
        pa = oracle.parse_record(replay.record_of(a, ha, i), g.side, g.n, g.L, g.M, cfg.dtype)
        pb = oracle.parse_record(replay.record_of(b, hb, i), g.side, g.n, g.L, g.M, cfg.dtype)
        nrice += bool(pb["flags"] & 8)
        np.testing.assert_array_equal(pa["k"], pb["k"])
        np.testing.assert_array_equal(pa["q"], pb["q"])
    assert nrice > 0
    # a Rice record with a flipped bit in its coded words does not parse
    i = next(j for j in range(len(trs)) if replay.record_of(b, hb, j)[1] & 8)
    g = oracle.block_geom(cfg, i)
    rec = bytearray(bytes(replay.record_of(b, hb, i)))
    bad = 0
    for pos in range(200, len(rec) - 64, 97):
        r2 = bytearray(rec)
        r2[pos] ^= 0x10
        p2 = oracle.parse_record(bytes(r2), g.side, g.n, g.L, g.M, cfg.dtype)
        pa = oracle.parse_record(bytes(rec), g.side, g.n, g.L, g.M, cfg.dtype)
        if p2 is None or not np.array_equal(p2["k"], pa["k"]) or not np.array_equal(p2["q"], pa["q"]):
            bad += 1
    assert bad > 0
