"""Pins of the Rice-coded correction section in the oracle (a proposed record
section, not yet used by records): a hand-derived bit pattern, round trips,
the exact size against a run-length count done here with numpy, the
parameter choice against brute force, the size against the entropy of
Bernoulli positions, malformed input rejected, and the size against the
current correction section on the oracle's own corrections."""
import numpy as np
import pytest

import oracle
from paper_2601_20113_gb300 import synth


@pytest.fixture(scope="module", autouse=True)
def _build():
    oracle.build()


def _zz(k):
    k = k.astype(np.int64)
    return ((k << 1) ^ (k >> 63)).astype(np.uint64)


def _bits_by_runs(k, chunk, kr, wv):
    """Size from the definition: per chunk, a code per nonzero (zeros before it,
    then the value) and a closing code for the trailing zeros."""
    total = 0
    for c0 in range(0, k.size, chunk):
        seg = k[c0:c0 + chunk]
        nz = np.flatnonzero(seg)
        runs = np.diff(np.concatenate(([-1], nz))) - 1
        closing = seg.size - 1 - (nz[-1] if nz.size else -1)
        total += int(np.sum((runs >> kr) + 1 + kr + wv)) + (closing >> kr) + 1 + kr
    return total


def test_hand_derived_bit_pattern():
    """chunk 8, kr 1, wv 2, k = [0 0 0 2 0 0 0 0]: run 3 -> '1','0', low bit 1;
    zigzag(2) - 1 = 3 -> bits 1,1; closing run 4 -> '1','1','0', low bit 0:
    bits 1,0,1,1,1,1,1,0,0 LSB first = 125."""
    k = np.array([0, 0, 0, 2, 0, 0, 0, 0], np.int32)
    words, off, bits = oracle.rice_encode(k, 8, 1, 2)
    assert bits == 9 and int(words[0]) == 125 and off.tolist() == [0]


@pytest.mark.parametrize("N,chunk", [(1, 32), (31, 32), (1024, 32), (65541, 1024), (5000, 1000)])
@pytest.mark.parametrize("p", [0.0, 0.01, 0.1, 0.5, 1.0])
def test_round_trip(N, chunk, p):
    rng = np.random.default_rng(int(N * 7 + p * 100))
    k = np.where(rng.random(N) < p, rng.integers(-300, 301, N), 0).astype(np.int32)
    kr, wv = oracle.rice_choose(k, chunk)
    words, off, bits = oracle.rice_encode(k, chunk, kr, wv)
    assert bits == _bits_by_runs(k, chunk, kr, wv) == oracle.rice_bits(k, chunk, kr, wv)
    back = oracle.rice_decode(words, off, N, chunk, kr, wv)
    assert back is not None and np.array_equal(back, k)
    # every chunk decodes alone from its offset: a chunk's code ends where the next begins
    assert off[0] == 0 and np.all(np.diff(off.astype(np.int64)) > 0)


def test_choice_is_the_minimum():
    rng = np.random.default_rng(5)
    for p in (0.003, 0.05, 0.3, 0.8):
        k = np.where(rng.random(20000) < p, rng.integers(-9, 10, 20000), 0).astype(np.int32)
        kr, wv = oracle.rice_choose(k, 1024)
        nz = k[k != 0]
        assert wv == (int((_zz(nz) - 1).max()).bit_length() if nz.size else 0)
        sizes = [oracle.rice_bits(k, 1024, r, wv) for r in range(21)]
        assert sizes[kr] == min(sizes) and kr == int(np.argmin(sizes))


@pytest.mark.parametrize("p", [0.02, 0.05, 0.1, 0.2, 0.3])
def test_size_near_the_entropy(p):
    """Bernoulli(p) positions with values +-1: Rice codes of geometric runs stay
    within 12% of the entropy H(p) + p bits per point (plus one closing code
    per chunk)."""
    N, chunk = 1 << 20, 1024
    rng = np.random.default_rng(int(p * 1000))
    k = np.where(rng.random(N) < p, np.where(rng.random(N) < 0.5, 1, -1), 0).astype(np.int32)
    kr, wv = oracle.rice_choose(k, chunk)
    H = -(p * np.log2(p) + (1 - p) * np.log2(1 - p)) + p
    per_point = oracle.rice_bits(k, chunk, kr, wv) / N
    assert per_point <= 1.12 * H + (1 + kr + 8) / chunk, (per_point, H)


def test_malformed_sections_are_rejected():
    rng = np.random.default_rng(6)
    k = np.where(rng.random(4096) < 0.1, rng.integers(-5, 6, 4096), 0).astype(np.int32)
    kr, wv = oracle.rice_choose(k, 512)
    words, off, bits = oracle.rice_encode(k, 512, kr, wv)
    assert oracle.rice_decode(words[: len(words) // 2], off, 4096, 512, kr, wv) is None   # truncated
    bad = words.copy()
    bad[:] = 0xFFFFFFFF                                                                  # endless unary runs
    assert oracle.rice_decode(bad, off, 4096, 512, kr, wv) is None


def test_smaller_than_the_current_section_on_real_corrections():
    """On the oracle's corrections of modes3d 64^3 x 32 blocks at 1e-3 x range,
    wherever at least 2% of the points carry a correction, the Rice section
    (with its chunk offsets and parameters) takes less than 55% of the current
    one (dense wk bits per point or an index list, whichever is smaller).
    Sparser blocks keep the index list, which is then the smaller one."""
    dims = (64, 64, 64, 32)
    f = synth.modes3d(*dims, seed=2, count=64).numpy()
    eb = 1e-3 * float(f.max() - f.min())
    cfg = oracle.Config(dims, (16, 16, 16, 16), oracle.F32, eb=eb, rank_cap=16)
    cur = rice = used = 0
    for b in range(0, oracle.num_blocks(cfg), 8):
        res = oracle.block_compress(cfg, f, b)
        k = res["k"].astype(np.int32)
        tr = res["trace"]
        N = k.size
        if tr.wk == 0 or tr.n_corr < 0.02 * N:
            continue
        used += 1
        cur += min(N * tr.wk, tr.n_corr * (tr.ib + tr.wk))
        kr, wv = oracle.rice_choose(k, 1024)
        rice += oracle.rice_bits(k, 1024, kr, wv) + 32 * (-(-N // 1024)) + 10   # offsets + parameters
    assert used >= 4 and rice < 0.55 * cur, (used, rice, cur)


@pytest.mark.parametrize("rel,eb_type", [(1e-3, oracle.EB_ABS), (1e-4, oracle.EB_ABS), (1e-3, oracle.EB_REL_RANGE)])
def test_rice_records_decode_to_the_same_field(rel, eb_type):
    """Records with the Rice section (corr_codec = 1) carry the same
    corrections as the default records: the decompressed fields are
    bit-identical, the bound holds, and the stream is smaller."""
    dims = (48, 48, 32, 32)
    f = synth.modes3d(*dims, seed=2, count=64).numpy()
    eb = rel * float(f.max() - f.min()) if eb_type == oracle.EB_ABS else rel
    base = oracle.Config(dims, (16, 16, 16, 16), oracle.F32, eb=eb, eb_type=eb_type, rank_cap=16)
    rice = oracle.Config(dims, (16, 16, 16, 16), oracle.F32, eb=eb, eb_type=eb_type, rank_cap=16, corr_codec=1)
    st0, s0, _ = oracle.compress(base, f)
    st1, s1, _ = oracle.compress(rice, f)
    assert st0 == 0 and st1 == 0
    st0, r0 = oracle.decompress(s0)
    st1, r1 = oracle.decompress(s1)
    assert st0 == 0 and st1 == 0
    assert np.array_equal(r0.view(np.uint32), r1.view(np.uint32))
    bound = eb if eb_type == oracle.EB_ABS else rel * float(f.max() - f.min())
    assert np.abs(r1.astype(np.float64) - f.astype(np.float64)).max() <= bound
    assert s1.size < s0.size, (s1.size, s0.size)


def test_rice_record_corruption_is_detected():
    dims = (32, 32, 16, 16)
    f = synth.modes3d(*dims, seed=3, count=64).numpy()
    cfg = oracle.Config(dims, (16, 16, 16, 16), oracle.F32, eb=1e-4 * float(f.max() - f.min()), rank_cap=16,
                        corr_codec=1)
    st, s, _ = oracle.compress(cfg, f)
    assert st == 0
    hdr = s[:128].view(np.uint64)
    payp, offp = int(hdr[14]), int(hdr[13])
    off0 = int(s[offp:offp + 8].view(np.uint64)[0])
    rec = payp + off0
    assert s[rec + 1] & 8                                   # the first record took the Rice section
    bad = s.copy()
    # the Rice word count sits at the start of the correction section; make it disagree with the record size
    r = int(s[rec])
    n, es, L = 16, 4, 16 * 16 * 16
    wq = s[rec + 16:rec + 16 + r]
    al = lambda x, a: (x + a - 1) // a * a
    off_c = 16 + al(r, 8) + al(n * r * es, 8) + al(sum((L * int(w) + 31) // 32 for w in wq) * 4, 8)
    bad[rec + off_c:rec + off_c + 4] = np.frombuffer(np.uint32(10 ** 6).tobytes(), np.uint8)
    st, _ = oracle.decompress(bad)
    assert st != 0
