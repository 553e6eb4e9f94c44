"""GPU path vs the oracle, bit-exact, through the C ABI (via the binding).

Sizes: short strings (brute-force territory), windows spanning many 4096-key
tiles with ragged tails, and the full workload sizes (2^20 hashed tasks,
2^24 adversarial windows)."""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

FIELDS = ("sa", "lcp", "cand_len", "cand_id", "cand_start", "sel_start", "sel_len", "sel_trace",
          "trace_len", "trace_start")


@pytest.fixture(scope="module")
def apo():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2406_18111_gb300 import Apo
    a = Apo(0)
    yield a
    a.close()


def dev(a, dt):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a).view(dt)).cuda()


def tokens_dev(S, tb):
    S = np.asarray(S)
    if tb == 4:
        return dev(S.astype(np.uint32), np.int32)
    return dev(S.astype(np.uint64), np.int64)


def compare(apo, S, min_len, tb=4, sa_method="direct"):
    from paper_2406_18111_gb300 import as_u32
    S = np.asarray(S)
    r = apo.find_repeats(tokens_dev(S, tb), min_len)
    o = oracle.find_repeats(S.astype(np.uint64), min_len, sa_method=sa_method)
    for f in FIELDS:
        got = as_u32(getattr(r, f))
        want = getattr(o, f)
        if got.shape != want.shape or not np.array_equal(got, want):
            bad = np.nonzero(got[:min(len(got), len(want))] != want[:min(len(got), len(want))])[0]
            raise AssertionError(f"{f}: shapes {got.shape} vs {want.shape}, first diffs at {bad[:5]}")
    assert np.array_equal(r.cand_accepted.cpu().numpy(), o.accepted)
    return r, o


# ---------------------------------------------------------------- hashing
@pytest.mark.parametrize("n", [1, 1000, 1 << 14, 1 << 20])
def test_hash_config2(apo, n):
    from paper_2406_18111_gb300 import as_u64
    ts = W.config2_tasks(n)
    tok = apo.hash_tasks(dev(ts.task_id, np.int32), dev(ts.arg_off, np.int32), dev(ts.region, np.int32),
                         dev(ts.field_mask, np.int64), dev(ts.priv, np.uint8))
    assert np.array_equal(as_u64(tok), oracle.hash_tasks(ts))


def test_hash_jacobi(apo):
    from paper_2406_18111_gb300 import as_u64
    ts = W.jacobi_tasks(6)
    tok = apo.hash_tasks(dev(ts.task_id, np.int32), dev(ts.arg_off, np.int32), dev(ts.region, np.int32),
                         dev(ts.field_mask, np.int64), dev(ts.priv, np.uint8))
    assert np.array_equal(as_u64(tok), oracle.hash_tasks(ts))


# ---------------------------------------------------------------- repeats, small
def test_worked_examples(apo, golden):
    for name in ("aabcbcbaa.json", "ababab.json"):
        g = golden(name)
        S = [ord(c) for c in g["string"]]
        for ml in g["results"]:
            r, o = compare(apo, S, int(ml))
            assert o.sa.tolist() == g["sa"]


def test_short_strings(apo):
    k = 0
    for n in range(2, 13):
        for sigma in (1, 2, 3):
            for rep in range(3):
                S = W.uniform_int(9000 + k, n, 0, sigma - 1)
                k += 1
                compare(apo, S, 1 + rep, tb=4 if rep % 2 == 0 else 8)


@pytest.mark.parametrize("n", [0, 1, 2, 3])
def test_degenerate_sizes(apo, n):
    compare(apo, np.arange(n) % 2, 1)


def test_constant_run_and_huge_tokens(apo):
    compare(apo, np.zeros(5000, dtype=np.uint32), 1)
    compare(apo, np.full(4097, 0xFFFFFFFF, dtype=np.uint32), 3, tb=4)
    big = W.splitmix64(3, 6000) | np.uint64(1 << 63)
    big[::7] = np.uint64(0xFFFFFFFFFFFFFFFF)
    compare(apo, np.concatenate([big, big[:3000]]), 2, tb=8)


# ---------------------------------------------------------------- repeats, workloads
@pytest.mark.parametrize("min_len", [1, 5, 25])
def test_config1(apo, min_len):
    compare(apo, W.config1_window(), min_len)


@pytest.mark.parametrize("n", [1 << 14, (1 << 16) + 123])
def test_config2_tokens_scaled(apo, n):
    tok = oracle.hash_tasks(W.config2_tasks(n))
    compare(apo, tok, 5, tb=8)


def test_config2_full(apo):
    """The window of 2^20 hashed tasks end to end, as the bench runs it: the
    repeats, then their traces matched against the window with the window's
    suffix and LCP arrays (long self-slices: the exact halo pass)."""
    from paper_2406_18111_gb300 import as_u32
    tok = oracle.hash_tasks(W.config2_tasks(1 << 20))
    r, o = compare(apo, tok, 5, tb=8)
    assert r.rounds >= 1
    t = tokens_dev(tok, 8)
    rs = apo.find_repeats(t, 5, stages=False, sa_lcp=True)
    apo.profile_reset()
    e, i = apo.match_candidates(t, None, t, pat_start=rs.trace_start, pat_len=rs.trace_len, src_sa=rs.sa,
                                src_lcp=rs.lcp)
    prof = apo.profile_read()
    assert "ac.ac_halo" in prof and "ac.ac_states" not in prof and "ac.ac_fix" not in prof
    st, tl = o.trace_start.astype(np.int64), o.trace_len.astype(np.int64)
    off = np.zeros(len(tl) + 1, np.uint64)
    off[1:] = np.cumsum(tl)
    pt = np.concatenate([tok[a:a + b] for a, b in zip(st, tl)])
    oe, oi = oracle.match(pt, off, tok)
    assert len(oe) > 0
    assert np.array_equal(as_u32(e), oe) and np.array_equal(as_u32(i), oi)


def test_config3_windows(apo):
    toks, off, periods = W.config3_windows(24)
    order = np.argsort(np.diff(off.astype(np.int64)))
    pick = list(order[:4]) + list(order[-3:])
    pick += [w for w in range(24) if periods[w] > off[w + 1] - off[w]][:2]  # only noise repeats
    for w in sorted(set(int(x) for x in pick)):
        S = toks[int(off[w]):int(off[w + 1])]
        compare(apo, S, 5)


def test_config4_scaled(apo):
    a, b = W.config4_windows(3 * (1 << 12) + 5)
    compare(apo, a, 5, sa_method="doubling")
    compare(apo, b, 5)
    compare(apo, a, 1, sa_method="doubling")


def test_config4_full(apo):
    """2^24 tokens, both windows, every field element by element: the random
    window against the direct oracle, the adversarial window (a constant run
    of 5.59M tokens, then period-2 and period-3 runs; 23 doubling rounds)
    against the oracle's Manber-Myers suffix array and LCE comparisons."""
    a, b = W.config4_windows()
    compare(apo, b, 5)
    r, o = compare(apo, a, 5, sa_method="doubling")
    assert r.rounds >= 18  # h0 = 21 tokens per first key (3-bit codes): log2(5592405 / 21) > 18


def test_batched_config3_full(apo):
    """All 512 windows of config 3 (23.3M tokens) in one batched call, every
    window's fields against the oracle (run on a pool of host threads)."""
    import concurrent.futures as cf
    import os
    toks, off, periods = W.config3_windows()
    wins = [toks[int(off[w]):int(off[w + 1])] for w in range(len(off) - 1)]
    res = apo.find_repeats_batched(tokens_dev(toks, 4), off, 5)
    with cf.ThreadPoolExecutor(max_workers=os.cpu_count() or 4) as ex:
        want = list(ex.map(lambda S: oracle.find_repeats(np.asarray(S, np.uint64), 5), wins))
    _check_batch_against(res, wins, lambda w, S: want[w])


# ---------------------------------------------------------------- matching
def test_match_ushers(apo, golden):
    from paper_2406_18111_gb300 import as_u32
    g = golden("ushers.json")
    toks, off = [], [0]
    for p in g["patterns"]:
        toks += [ord(c) for c in p]
        off.append(len(toks))
    for tb in (4, 8):
        e, i = apo.match_candidates(tokens_dev(toks, tb), np.array(off, np.uint64),
                                    tokens_dev([ord(c) for c in g["text"]], tb))
        assert list(zip(as_u32(e).tolist(), as_u32(i).tolist())) == [tuple(x) for x in g["matches"]]


@pytest.mark.parametrize("tb", [4, 8])
def test_match_random(apo, tb):
    from paper_2406_18111_gb300 import as_u32
    for trial in range(5):
        n = 5000 + 37 * trial
        text = W.uniform_int(300 + trial, n, 0, 2)
        P = 60
        lens = W.uniform_int(400 + trial, P, 1, 9)
        pats = [W.uniform_int(500 + 13 * trial + p, int(lens[p]), 0, 2) for p in range(P)]
        pats.append(pats[3])
        off = np.zeros(len(pats) + 1, np.uint64)
        off[1:] = np.cumsum([len(p) for p in pats])
        pt = np.concatenate(pats)
        e, i = apo.match_candidates(tokens_dev(pt, tb), off, tokens_dev(text, tb))
        oe, oi = oracle.match(pt, off, text)
        assert np.array_equal(as_u32(e), oe) and np.array_equal(as_u32(i), oi)


@pytest.mark.parametrize("n,P", [(1 << 20, 400), (1 << 22, 2000)])
def test_match_config5_scaled(apo, n, P):
    from paper_2406_18111_gb300 import as_u32
    stream = W.match_stream(n, seed=7)
    pt, off = W.match_patterns(stream, P, 5, 2000, seed=7)
    apo.profile_reset()
    e, i = apo.match_candidates(tokens_dev(pt, 4), off, tokens_dev(stream, 4))
    prof = apo.profile_read()
    assert "ac.ac_states" in prof and "ac.ac_halo" not in prof  # chunks and repairs
    oe, oi = oracle.match(pt, off, stream)
    assert len(oe) > 0
    assert np.array_equal(as_u32(e), oe) and np.array_equal(as_u32(i), oi)


# ---------------------------------------------------------------- errors
def test_invalid_arguments(apo):
    import torch
    from paper_2406_18111_gb300 import ApoError
    t = tokens_dev(np.arange(10), 4)
    with pytest.raises(ApoError):
        apo.find_repeats(t, 0)
    with pytest.raises((ApoError, TypeError)):
        apo.find_repeats(t.to(torch.int16), 1)
    with pytest.raises(ApoError):
        apo.match_candidates(t, np.array([0, 2, 2], np.uint64), t)
    # source mode: the source arrays must cover the slices
    r = apo.find_repeats(t, 1, stages=False, sa_lcp=True)
    ps = dev(np.array([0, 5], np.uint32), np.int32)
    pl = dev(np.array([3, 5], np.uint32), np.int32)
    with pytest.raises(ApoError):
        apo.match_candidates(t[:6], None, t, pat_start=ps, pat_len=pl, src_sa=r.sa[:6], src_lcp=r.lcp[:6])
    # sort-shape modes: 0, 1 and 2 + k for the six shapes, nothing else
    for bad in (-1, 8):
        with pytest.raises(ApoError):
            apo.sort_tuning(bad)


def test_match_source_mode_edges(apo):
    """Source mode at the edges: one-token patterns, a pattern that is the
    whole source, patterns ending at the source's end, a constant source."""
    from paper_2406_18111_gb300 import as_u32
    for S in (np.array([3, 1, 4, 1, 5, 9, 2, 6, 5, 3, 5], np.uint32), np.full(40, 7, np.uint32),
              (np.arange(50) % 3).astype(np.uint32)):
        n = len(S)
        t = tokens_dev(S, 4)
        r = apo.find_repeats(t, 1, stages=False, sa_lcp=True)
        starts = np.array([0, n - 1, 0, n - 3, 1, 2, 2], np.uint32)
        lens = np.array([1, 1, n, 3, 2, n - 2, 1], np.uint32)
        e1, i1 = apo.match_candidates(t, None, t, pat_start=dev(starts, np.int32), pat_len=dev(lens, np.int32),
                                      src_sa=r.sa, src_lcp=r.lcp)
        off = np.zeros(len(lens) + 1, np.uint64)
        off[1:] = np.cumsum(lens)
        pt = np.concatenate([S[a:a + l] for a, l in zip(starts, lens)]).astype(np.uint64)
        oe, oi = oracle.match(pt, off, S.astype(np.uint64))
        assert np.array_equal(as_u32(e1), oe) and np.array_equal(as_u32(i1), oi)


def test_match_traces_slice_form(apo):
    """The traces apo_find_repeats returns, matched as device slices of the
    window against the window itself (the bench's pipeline)."""
    from paper_2406_18111_gb300 import as_u32
    tok = oracle.hash_tasks(W.config2_tasks(1 << 14))
    t = tokens_dev(tok, 8)
    r = apo.find_repeats(t, 5, stages=False)
    e, i = apo.match_candidates(t, None, t, pat_start=r.trace_start, pat_len=r.trace_len)
    o = oracle.find_repeats(tok, 5)
    st, tl = o.trace_start.astype(np.int64), o.trace_len.astype(np.int64)
    off = np.zeros(len(tl) + 1, np.uint64)
    off[1:] = np.cumsum(tl)
    pt = np.concatenate([tok[s:s + l] for s, l in zip(st, tl)])
    oe, oi = oracle.match(pt, off, tok)
    assert len(oe) > 0
    assert np.array_equal(as_u32(e), oe) and np.array_equal(as_u32(i), oi)


@pytest.mark.parametrize("n,period,tb", [(1000, 7, 4), (3 * 4096 + 77, 300, 8), (50000, 1500, 4)])
def test_match_halo_pass(apo, n, period, tb):
    """Long slices of the stream matched against the stream itself (the
    exact pass that starts each segment one longest-pattern length early):
    ragged segments, segments nearer the start than that length, a pattern
    ending at the stream's end, long failure chains in a noisy periodic
    stream.  The same
    matches as the oracle and as the chunked pass (the patterns as CSR)."""
    from paper_2406_18111_gb300 import as_u32
    S = W.periodic_window(n, period, 0.02, 50, seed=n)
    rng = np.random.default_rng(period)
    k = max(8, n // 100)
    lens = rng.integers(65, min(512, n) + 1, k)
    starts = rng.integers(0, n - lens + 1)
    lens[0], starts[0] = min(512, n), n - min(512, n)  # a pattern ending at the stream's end
    assert 4 * lens.sum() >= n
    t = tokens_dev(S, tb)
    apo.profile_reset()
    e1, i1 = apo.match_candidates(t, None, t, pat_start=dev(starts.astype(np.uint32), np.int32),
                                  pat_len=dev(lens.astype(np.uint32), np.int32))
    prof = apo.profile_read()
    assert "ac.ac_halo" in prof and "ac.ac_states" not in prof
    off = np.zeros(k + 1, np.uint64)
    off[1:] = np.cumsum(lens)
    pt = np.concatenate([S[a:a + b] for a, b in zip(starts, lens)])
    apo.profile_reset()
    e2, i2 = apo.match_candidates(tokens_dev(pt, tb), off, t)
    assert "ac.ac_states" in apo.profile_read()
    oe, oi = oracle.match(pt.astype(np.uint64), off, S.astype(np.uint64))
    assert len(oe) > 0
    assert np.array_equal(as_u32(e1), oe) and np.array_equal(as_u32(i1), oi)
    assert np.array_equal(as_u32(e2), oe) and np.array_equal(as_u32(i2), oi)


@pytest.mark.parametrize("n,tb", [(1 << 14, 8), ((1 << 16) + 77, 8), (20000, 4)])
def test_match_source_mode(apo, n, tb):
    """Slices matched with the source's suffix and LCP arrays given (the
    automaton read off the source's suffix array): the same matches as the
    oracle, and as the call that builds a suffix array of the patterns; also
    arbitrary overlapping, nested and duplicate slices."""
    from paper_2406_18111_gb300 import as_u32
    import torch
    if tb == 8:
        tok = oracle.hash_tasks(W.config2_tasks(n, seed=9))
    else:
        tok, _, _ = W.config3_windows(1, seed0=41)
        tok = tok[:n].astype(np.uint64)
    t = tokens_dev(tok, tb)
    r = apo.find_repeats(t, 5, stages=False, sa_lcp=True)
    starts = [as_u32(r.trace_start).astype(np.int64)]
    lens = [as_u32(r.trace_len).astype(np.int64)]
    rng = np.random.default_rng(n)
    k = 300
    a = rng.integers(0, len(tok) - 1, k)
    l = np.minimum(rng.integers(1, 400, k), len(tok) - a)
    starts.append(a)
    lens.append(l)
    starts.append(starts[0][:20])  # duplicates
    lens.append(lens[0][:20])
    ps = np.concatenate(starts)
    pl = np.concatenate(lens)
    dps = dev(ps.astype(np.uint32), np.int32)
    dpl = dev(pl.astype(np.uint32), np.int32)
    e1, i1 = apo.match_candidates(t, None, t, pat_start=dps, pat_len=dpl, src_sa=r.sa, src_lcp=r.lcp)
    e2, i2 = apo.match_candidates(t, None, t, pat_start=dps, pat_len=dpl)
    assert np.array_equal(as_u32(e1), as_u32(e2)) and np.array_equal(as_u32(i1), as_u32(i2))
    off = np.zeros(len(pl) + 1, np.uint64)
    off[1:] = np.cumsum(pl)
    pt = np.concatenate([tok[x:x + y] for x, y in zip(ps, pl)])
    oe, oi = oracle.match(pt, off, tok)
    assert len(oe) > 0
    assert np.array_equal(as_u32(e1), oe) and np.array_equal(as_u32(i1), oi)
    del torch


# ---------------------------------------------------------------- batched form
def _window_slice(res, w, name, off_name):
    from paper_2406_18111_gb300 import as_u32
    off = getattr(res, off_name)
    a = getattr(res, name)
    x = a[int(off[w]):int(off[w + 1])]
    return x.cpu().numpy() if name == "cand_accepted" else as_u32(x)


def _check_batch_against(res, wins, per_window):
    from paper_2406_18111_gb300 import as_u32
    for w, S in enumerate(wins):
        o = per_window(w, S)
        a, b = int(res.win_off[w]), int(res.win_off[w + 1])
        assert np.array_equal(as_u32(res.sa[a:b]), o.sa), ("sa", w)
        assert np.array_equal(as_u32(res.lcp[a:b]), o.lcp), ("lcp", w)
        for f in ("cand_len", "cand_start", "cand_accepted"):
            want = o.accepted if f == "cand_accepted" else getattr(o, f)
            assert np.array_equal(_window_slice(res, w, f, "cand_off"), want), (f, w)
        for f in ("sel_start", "sel_len", "sel_trace"):
            assert np.array_equal(_window_slice(res, w, f, "sel_off"), getattr(o, f)), (f, w)
        for f in ("trace_len", "trace_start"):
            assert np.array_equal(_window_slice(res, w, f, "trace_off"), getattr(o, f)), (f, w)


def _concat(wins):
    off = np.zeros(len(wins) + 1, np.uint64)
    off[1:] = np.cumsum([len(x) for x in wins])
    return np.concatenate(wins).astype(np.uint32) if len(wins) else np.zeros(0, np.uint32), off


def test_batched_config3_vs_oracle(apo):
    toks, off, periods = W.config3_windows(24)
    wins = [toks[int(off[w]):int(off[w + 1])] for w in range(24)]
    wins += [np.zeros(0, np.uint32), np.array([7], np.uint32), np.array([3, 3, 3, 3, 3, 3], np.uint32)]
    cat, o = _concat(wins)
    res = apo.find_repeats_batched(tokens_dev(cat, 4), o, 5)
    _check_batch_against(res, wins, lambda w, S: oracle.find_repeats(np.asarray(S, np.uint64), 5))


def test_batched_equals_plain_and_u64(apo):
    """Each window's bytes are the same alone (plain call) and in the batch."""
    from paper_2406_18111_gb300 import as_u32
    wins = [oracle.hash_tasks(W.config2_tasks(3000 + 977 * k, seed=20 + k)) for k in range(5)]
    cat = np.concatenate(wins)
    off = np.zeros(len(wins) + 1, np.uint64)
    off[1:] = np.cumsum([len(x) for x in wins])
    res = apo.find_repeats_batched(tokens_dev(cat, 8), off, 5)

    class Plain:
        pass

    def plain(w, S):
        r = apo.find_repeats(tokens_dev(S, 8), 5)
        p = Plain()
        for f in FIELDS:
            setattr(p, f, as_u32(getattr(r, f)))
        p.accepted = p.cand_accepted = r.cand_accepted.cpu().numpy()
        return p
    _check_batch_against(res, wins, plain)
    _check_batch_against(res, wins, lambda w, S: oracle.find_repeats(S, 5))


def _tile_cases():
    """Windows whose doubling groups straddle the round kernel's tile span
    (1024 list entries): periodic strings whose level groups hold about
    n / p suffixes, with and without noise."""
    cases = []
    k = 0
    for p in (1, 2, 3, 5):
        for g in (1023, 1024, 1025, 1026, 2047, 2049, 4100):
            n = p * g + (k % 3)
            S = (np.arange(n) % p).astype(np.uint32)
            if k % 2:
                pos = W.uniform_int(700 + k, max(1, n // 200), 0, n - 1)
                S[pos] = W.uniform_int(800 + k, len(pos), 0, 7).astype(np.uint32)
            cases.append(S)
            k += 1
    return cases


def test_doubling_tile_boundaries(apo):
    """Group sizes around the tile span, one window per call and all of them
    in one batched call, SA and LCP against the oracle."""
    from paper_2406_18111_gb300 import as_u32
    cases = _tile_cases()
    for S in cases[::3]:
        compare(apo, S, 5, sa_method="doubling")
    wins = cases + [np.zeros(0, np.uint32), np.zeros(3000, np.uint32)]
    cat, off = _concat(wins)
    res = apo.find_repeats_batched(tokens_dev(cat, 4), off, 5)
    for w, S in enumerate(wins):
        a, b = int(res.win_off[w]), int(res.win_off[w + 1])
        sa = oracle.suffix_array(np.asarray(S, np.uint64), "doubling")
        assert np.array_equal(as_u32(res.sa[a:b]), sa), ("sa", w)
        assert np.array_equal(as_u32(res.lcp[a:b]), oracle.lcp(np.asarray(S, np.uint64), sa)), ("lcp", w)


# ---------------------------------------------------------------- sort shapes
def test_sort_shapes_give_identical_results(apo):
    """Every radix-sort shape the tuner may pick gives the same bytes: the
    same windows with tuning off (default shape) and on (timed shapes), and
    against the oracle; the tuner reports what it chose."""
    from paper_2406_18111_gb300 import Apo, as_u32
    S = oracle.hash_tasks(W.config2_tasks((1 << 16) + 321, seed=31))
    want = oracle.find_repeats(S, 5)
    for mode in (1, 0):
        a = Apo(0)
        a.sort_tuning(mode)
        r = a.find_repeats(tokens_dev(S, 8), 5)
        for f in FIELDS:
            assert np.array_equal(as_u32(getattr(r, f)), getattr(want, f)), (mode, f)
        if mode == 0:
            tab = a.sort_tuning_read()
            assert tab and all(t["threads"] in (256, 512) and t["digit_bits"] in (8, 9) for t in tab)
            assert all(t["best_ms"] <= t["default_ms"] + 1e-9 for t in tab)
        a.close()


# ---------------------------------------------------------------- served form
def test_served_results_equal_alone(apo):
    """Requests submitted together are batched by the server; every result
    equals what the same window gives alone (plain call) and the oracle."""
    from paper_2406_18111_gb300 import Server, as_u32
    srv = Server(0, min_len=5, token_bytes=4, max_batch_tokens=300000, max_batch_windows=8, lanes=2)
    wins = []
    for r in range(14):
        L = [5000, 60000, 1, 0, 12345, 100000, 4096][r % 7] + r
        wins.append(W.periodic_window(L, 3 + (r * 977) % 4000, 0.05, 1000, seed=900 + r))
    ids = [srv.submit(S) for S in wins]
    res = [srv.wait(i) for i in ids]
    srv.close()
    assert max(x.batch_windows for x in res) > 1  # some requests shared a batch
    for S, got in zip(wins, res):
        alone = apo.find_repeats(tokens_dev(S, 4), 5, stages=False)
        o = oracle.find_repeats(S.astype(np.uint64), 5)
        for f in ("sel_start", "sel_len", "sel_trace", "trace_len", "trace_start"):
            assert np.array_equal(getattr(got, f), as_u32(getattr(alone, f))), f
            assert np.array_equal(getattr(got, f), getattr(o, f)), f


def test_served_config5_mix(apo):
    """Config 5's request mix (window lengths log-uniform 4,096..2^20, the
    first 0.1 s of its Poisson arrivals: about 200 requests) submitted in
    bursts while earlier batches run: every result equals the plain call on
    its window, and every tenth one also the oracle (on a thread pool)."""
    import time
    from concurrent.futures import ThreadPoolExecutor
    from paper_2406_18111_gb300 import Server, as_u32
    t_arr, L, P = W.served_requests(0.1, 2000.0, seed=77)
    wins = [W.served_window(k, int(L[k]), int(P[k]), seed=77) for k in range(len(L))]
    assert len(wins) >= 150
    srv = Server(0, min_len=5, token_bytes=4, max_batch_tokens=1 << 24, max_batch_windows=64, lanes=2)
    ids = []
    for k, S in enumerate(wins):
        ids.append(srv.submit(S))
        if k % 25 == 24:
            time.sleep(0.002)  # let lanes start batches while more requests arrive
    res = [srv.wait(i) for i in ids]
    srv.close()
    assert max(x.batch_windows for x in res) > 1
    fields = ("sel_start", "sel_len", "sel_trace", "trace_len", "trace_start")
    for S, got in zip(wins, res):
        alone = apo.find_repeats(tokens_dev(S, 4), 5, stages=False)
        for f in fields:
            assert np.array_equal(getattr(got, f), as_u32(getattr(alone, f))), f
    sample = list(range(0, len(wins), 10))
    with ThreadPoolExecutor(max_workers=16) as ex:
        ors = list(ex.map(lambda k: oracle.find_repeats(wins[k].astype(np.uint64), 5), sample))
    for k, o in zip(sample, ors):
        for f in fields:
            assert np.array_equal(getattr(res[k], f), getattr(o, f)), (k, f)


def test_served_admission_by_footprint(apo):
    """A pool that holds one request's footprint at a time: the second and
    third requests wait for the one before to return its slice, never more
    than the budget is held, results equal the plain call and the oracle,
    and a request larger than the whole pool is refused."""
    from paper_2406_18111_gb300 import ApoError, Server, as_u32
    n = 1 << 18
    fp = Server.footprint(n, 4, 5)
    srv = Server(0, min_len=5, token_bytes=4, max_batch_tokens=1 << 24, max_batch_windows=8, lanes=2,
                 hbm_budget=int(fp * 1.6))
    wins = [W.periodic_window(n, 97 + 13 * k, 0.05, 1000, seed=500 + k) for k in range(3)]
    ids = [srv.submit(S) for S in wins]
    res = [srv.wait(i) for i in ids]
    assert all(r.batch_windows == 1 for r in res)
    order = sorted(res, key=lambda r: r.t_start)
    for x, y in zip(order, order[1:]):
        assert y.t_start >= x.t_done  # admitted only once the slice before it came back
    mem = srv.memory()
    assert mem["held"] == 0 and fp <= mem["held_max"] <= mem["budget"]
    for S, got in zip(wins, res):
        alone = apo.find_repeats(tokens_dev(S, 4), 5, stages=False)
        o = oracle.find_repeats(S.astype(np.uint64), 5)
        for f in ("sel_start", "sel_len", "sel_trace", "trace_len", "trace_start"):
            assert np.array_equal(getattr(got, f), as_u32(getattr(alone, f))), f
            assert np.array_equal(getattr(got, f), getattr(o, f)), f
    big = srv.submit(np.zeros(2 * n, np.uint32))
    with pytest.raises(ApoError, match="APO_ECAPACITY"):
        srv.wait(big)
    srv.close()


def test_match_config5_full(apo):
    """Full-size matching workload: 2^26-token stream, 10,000 patterns."""
    from paper_2406_18111_gb300 import as_u32
    stream = W.match_stream(1 << 26, seed=5)
    pt, off = W.match_patterns(stream, 10000, 5, 2000, seed=5)
    e, i = apo.match_candidates(tokens_dev(pt, 4), off, tokens_dev(stream, 4))
    oe, oi = oracle.match(pt, off, stream)
    assert len(oe) > 0
    assert np.array_equal(as_u32(e), oe) and np.array_equal(as_u32(i), oi)


# ---------------------------------------------------------------- online finder (Sec. 4.4)
@pytest.mark.parametrize("unit,buffer,tb", [(250, 5000, 8), (100, 1000, 4)])
def test_finder_ruler_sampling_equals_oracle(apo, unit, buffer, tb):
    """Tokens pushed in uneven chunks: the analyses are the ruler-function
    slices, each with the oracle's traces (stream coordinates), in order."""
    from paper_2406_18111_gb300 import Finder, Server
    if tb == 8:
        S = oracle.hash_tasks(W.config2_tasks(12000, seed=17))
    else:
        S = (np.arange(9000) % 37).astype(np.uint32)
        S[W.uniform_int(18, 300, 0, 8999)] = 500
    srv = Server(0, min_len=5, token_bytes=tb, max_batch_tokens=1 << 20, max_batch_windows=64, lanes=2)
    f = Finder(srv, buffer_tokens=buffer, unit=unit)
    rng = np.random.default_rng(unit)
    pos = 0
    got = []
    while pos < len(S):
        k = int(rng.integers(1, 3 * unit))
        f.push(S[pos:pos + k])
        pos += k
        r = f.poll()
        if r is not None:
            got.append(r)
    got += f.drain()
    want = oracle.online_traces(S, unit, buffer, 5)
    assert len(got) == len(want) == len(S) // unit
    for g, (i, start, length, tl, ts) in zip(got, want):
        assert (g.index, g.slice_start, g.slice_len) == (i, start, length)
        assert np.array_equal(g.trace_len, tl) and np.array_equal(g.trace_start, ts), i
    st = f.stats()
    assert st["analyses"] == len(want)
    assert st["analysed_tokens"] == sum(w[2] for w in want)
    f.close()
    srv.close()


# ---------------------------------------------------------------- trace replay
def _replay_both(apo, S, starts, lens, ingest, tb=4, max_len=0, cap=0, half_life=0, bonus=(1, 1), window=0):
    S = np.asarray(S)
    starts = np.asarray(starts, dtype=np.uint32)
    lens = np.asarray(lens, dtype=np.uint32)
    ingest = np.asarray(ingest, dtype=np.uint32)
    o = oracle.replay(S.astype(np.uint64), starts, lens, ingest, max_len, cap, half_life, bonus)
    end, ln, tr, traced, curve, counts = apo.replay(
        tokens_dev(S, tb), dev(starts, np.int32), dev(lens, np.int32), dev(ingest, np.int32),
        max_trace_len=max_len, count_cap=cap, half_life=half_life, bonus=bonus, window=window, curve=True)
    got = (end.cpu().numpy().view(np.uint32), ln.cpu().numpy().view(np.uint32), tr.cpu().numpy().view(np.uint32))
    assert np.array_equal(got[0], o.end), "replay ends"
    assert np.array_equal(got[1], o.length), "replay lengths"
    assert np.array_equal(got[2], o.trace), "replay traces"
    n = S.shape[0]
    assert np.array_equal(traced.cpu().numpy(), o.traced)
    pre = np.concatenate([[0], np.cumsum(o.traced.astype(np.int64))])
    w = window if window else n
    want_curve = pre[1:] - pre[np.maximum(0, np.arange(1, n + 1) - w)]
    assert np.array_equal(curve.cpu().numpy().astype(np.int64), want_curve)
    assert counts[0] == len(o.end) and counts[1] == int(o.traced.sum())
    return o, counts


_TOKS = {ch: i + 1 for i, ch in enumerate("abcdexy")}


def _txt(t):
    return np.array([_TOKS[ch] for ch in t], dtype=np.uint32)


def test_replay_hand_cases(apo):
    # the oracle's hand-worked cases (tests/test_oracle_pins.py), GPU = oracle
    bc_abc = _txt("xbc" * 4 + "abc" * 3)
    cases = [
        (_txt("abc" * 5), [0], [3], [0], {}),
        (_txt("abc" * 5), [0], [3], [4], {}),
        (_txt("abcabc"), [0, 0], [2, 3], [0, 0], {}),
        (_txt("abcabc"), [1, 0], [2, 3], [0, 0], {}),
        (_txt("abcxabd"), [4, 0], [3, 3], [0, 2], {}),
        (_txt("abcxaxd"), [4, 0], [3, 3], [0, 2], {}),
        (bc_abc, [1, 12], [2, 3], [0, 0], {}),
        (bc_abc, [1, 12], [2, 3], [0, 0], {"cap": 2}),
        (bc_abc, [1, 12], [2, 3], [0, 0], {"half_life": 1}),
        (_txt("xycd" * 2 + "abcd" * 2), [2, 8], [2, 4], [0, 0], {"cap": 2, "bonus": (2, 1)}),
        (_txt("abcde" * 2), [0], [5], [0], {"max_len": 2}),
        (_txt("abcabc"), [3, 0], [3, 3], [0, 0], {}),
    ]
    for S, st, ln, ig, kw in cases:
        for tb in (4, 8):
            _replay_both(apo, S, st, ln, ig, tb=tb, **kw)


def test_replay_random_small(apo):
    rng = np.random.default_rng(11)
    for case in range(250):
        n = int(rng.integers(1, 80))
        per = int(rng.integers(1, 7))
        S = rng.integers(0, 3, size=per)[np.arange(n) % per]
        S = np.where(rng.random(n) < 0.1, rng.integers(0, 3, size=n), S).astype(np.uint32)
        P = int(rng.integers(0, 7))
        lens = rng.integers(1, min(n, 8) + 1, size=P)
        starts = np.array([rng.integers(0, n - l + 1) for l in lens], dtype=np.int64)
        ingest = rng.integers(0, n + 3, size=P)
        _replay_both(apo, S, starts, lens, ingest, max_len=int(rng.choice([0, 0, 2, 3])),
                     cap=int(rng.choice([0, 1, 2, 4])), half_life=int(rng.choice([0, 1, 3])),
                     bonus=[(1, 1), (2, 1), (17, 16), (1, 2)][int(rng.integers(0, 4))],
                     window=int(rng.choice([0, 1, 7])))


def _online_inputs(S, unit=250, buffer=5000, min_len=5):
    st, ln, ig = [], [], []
    for i, _, _, tl, ts in oracle.online_traces(S, unit, buffer, min_len):
        st += ts.tolist()
        ln += tl.tolist()
        ig += [(i + 1) * unit] * len(tl)  # ingested one analysis period after its point
    return np.array(st, np.uint32), np.array(ln, np.uint32), np.array(ig, np.uint32)


@pytest.mark.parametrize("n,kw", [
    (1 << 16, {}),
    (1 << 16, {"max_len": 16, "cap": 8, "half_life": 1000, "bonus": (17, 16), "window": 5000}),
    ((1 << 17) + 321, {"cap": 2, "half_life": 50, "bonus": (2, 1), "window": 1000}),
])
def test_replay_online_finder_traces(apo, n, kw):
    S = W.replay_stream(n, seed=6)
    st, ln, ig = _online_inputs(S)
    _, counts = _replay_both(apo, S, st, ln, ig, **kw)
    assert counts[0] > 100  # the stream does replay


@pytest.mark.parametrize("tb", [4, 8])
def test_replay_random_slices(apo, tb):
    n = (1 << 17) + 77
    S = W.replay_stream(n, seed=7)
    st, ln, ig = W.replay_random_traces(n, 4000, seed=8)
    _replay_both(apo, S, st, ln, ig, tb=tb, cap=4, half_life=200, bonus=(9, 8))


def test_replay_full_size(apo):
    # the replay workload's size: 2^20 tasks with every trace the online
    # finder (ruler sampling, unit 250, buffer 5000) reports over them
    S = W.replay_stream(1 << 20, seed=6)
    st, ln, ig = _online_inputs(S)
    _replay_both(apo, S, st, ln, ig, cap=8, half_life=1000, bonus=(17, 16), window=5000)


def test_replay_edges(apo):
    from paper_2406_18111_gb300 import ApoError
    S = _txt("abcabcabc")
    # no traces; traces that never enter; one-token pieces; all traces equal
    _replay_both(apo, S, [], [], [])
    _replay_both(apo, S, [0, 3], [3, 2], [9, 100])
    _replay_both(apo, S, [0], [9], [0], max_len=1)
    _replay_both(apo, S, [0, 3, 6, 3], [3, 3, 3, 3], [5, 2, 0, 7], cap=1)
    _replay_both(apo, S[:1], [0], [1], [0])
    # the whole stream as one trace: it can never repeat inside it
    _replay_both(apo, S, [0], [9], [0])
    # a constant stream with nested traces
    C = np.zeros(500, np.uint32)
    _replay_both(apo, C, [0, 0, 0, 7], [1, 5, 50, 13], [0, 10, 3, 100], cap=3, half_life=2, bonus=(3, 2))
    # errors: empty trace, trace past the end, bad bonus, bad token width
    import torch
    t = tokens_dev(S, 4)
    one = dev(np.array([0], np.uint32), np.int32)
    for st, ln, kw in [([0], [0], {}), ([7], [3], {}), ([0], [3], {"bonus": (0, 1)}), ([0], [3], {"bonus": (1, 70000)})]:
        with pytest.raises(ApoError):
            apo.replay(t, dev(np.array(st, np.uint32), np.int32), dev(np.array(ln, np.uint32), np.int32), one, **kw)
    with pytest.raises(TypeError):
        apo.replay(t.view(torch.int16), one, one, one)
    # too small a replay array: APO_ECAPACITY
    with pytest.raises(ApoError):
        apo.replay(t, one, dev(np.array([3], np.uint32), np.int32), one, rep_cap=1)


# ---------------------------------------------------------------- Sec. 3 optimum
def _optimum_both(apo, wins, m, tb=4):
    toks = np.concatenate([np.asarray(w, dtype=np.uint64) for w in wins]) if wins else np.zeros(0, np.uint64)
    off = np.zeros(len(wins) + 1, dtype=np.uint64)
    off[1:] = np.cumsum([len(w) for w in wins])
    t = tokens_dev(toks if len(toks) else np.zeros(1, np.uint64), tb)[:len(toks)]
    best, ws_, wl, wc = apo.optimum_batched(t, off, m)
    best, ws_, wl, wc = (x.cpu().numpy() for x in (best, ws_, wl, wc))
    for k, w in enumerate(wins):
        want, wit = oracle.optimum(np.asarray(w, dtype=np.uint64), m)
        assert tuple(best[k].tolist()) == want, (list(w), m)
        a = int(off[k])
        got = list(zip(ws_[a:a + wc[k]].tolist(), wl[a:a + wc[k]].tolist()))
        assert got == wit, (list(w), m)  # the first optimal set in the same order


def test_optimum_hand_and_random(apo):
    T = {c: i + 1 for i, c in enumerate("abcdxy")}
    hand = ["abab", "abcab", "abababab", "abcd", "abcabcxabc", "aabaab", "aaaa", "xyabxyab", "", "a"]
    _optimum_both(apo, [[T[c] for c in h] for h in hand], 2)
    rng = np.random.default_rng(21)
    for m, nmax, count in ((1, 11, 150), (2, 16, 250), (3, 20, 200), (5, 24, 100)):
        wins = []
        for _ in range(count):
            n = int(rng.integers(0, nmax + 1))
            if rng.random() < 0.5:
                w = rng.integers(0, int(rng.integers(1, 5)), size=n)
            else:
                per = int(rng.integers(1, 6))
                w = rng.integers(0, 4, size=per)[np.arange(n) % per]
                w = np.where(rng.random(n) < 0.1, rng.integers(0, 4, size=n), w)
            wins.append(w.astype(np.uint64))
        _optimum_both(apo, wins, m, 4)
        _optimum_both(apo, wins[:40], m, 8)


def test_optimum_limits(apo):
    from paper_2406_18111_gb300 import ApoError
    t = tokens_dev(np.zeros(25, np.uint32), 4)
    with pytest.raises(ApoError):  # a window past 24 tokens
        apo.optimum_batched(t, [0, 25], 2)
    with pytest.raises(ApoError):  # 2^24 interval sets exceeded (20 tokens, min_len 1)
        apo.optimum_batched(t[:20], [0, 20], 1)
    with pytest.raises(ApoError):
        apo.optimum_batched(t[:4], [0, 4], 0)


# ---------------------------------------------------------------- graph mode
@pytest.mark.parametrize("kind", ["u32", "u64"])
def test_graph_mode_single_window(apo, kind):
    """One window replayed as a CUDA graph (apo_find_repeats in graph mode)
    gives the same bytes as the plain call: on repeats of the same window,
    after its contents change (the replay's checks fail and it is
    recorded again), and back; u64 windows take the token dictionary."""
    import torch
    from paper_2406_18111_gb300 import Apo, as_u32
    n = 1 << 15
    if kind == "u32":
        a = W.periodic_window(n, 113, 0.03, 1000, seed=41)
        dt, tdt = np.int32, torch.int32
    else:
        ts = W.config2_tasks(n, seed=42)
        a = oracle.hash_tasks(ts)
        dt, tdt = np.int64, torch.int64
    b = a.copy()
    rng = np.random.default_rng(5)
    pos = rng.integers(0, n, size=n // 40)
    b[pos] = a[rng.integers(0, n, size=len(pos))]
    names = ("sa", "lcp", "cand_len", "cand_id", "cand_start", "sel_start", "sel_len", "sel_trace",
             "trace_len", "trace_start")

    def snap(r):
        d = {k: as_u32(getattr(r, k)).copy() for k in names}
        d["acc"] = r.cand_accepted.cpu().numpy().copy()
        d["rounds"] = r.rounds
        return d

    want = {name: snap(apo.find_repeats(dev(t, dt), 5)) for name, t in (("a", a), ("b", b))}
    o = oracle.find_repeats(a.astype(np.uint64), 5)
    assert np.array_equal(want["a"]["sel_start"], o.sel_start)
    g = Apo(0)
    try:
        g.graph_mode(True)
        buf = torch.empty(n, dtype=tdt, device="cuda")
        for name in ("a", "a", "a", "b", "b", "a"):
            buf.copy_(torch.from_numpy((a if name == "a" else b).view(dt)))
            got = snap(g.find_repeats(buf, 5, reuse=True))
            for k, v in want[name].items():
                assert np.array_equal(np.asarray(got[k]), np.asarray(v)), (name, k)
        st = g.graph_stats()
        assert st["replays"] >= 3 and st["captures"] >= 2 and st["discarded"] >= 1, st
        g.graph_mode(False)
    finally:
        g.close()


def test_graph_mode_results_equal_eager(apo):
    """Batched calls replayed as CUDA graphs give the same bytes as the plain
    path: on a repeated batch (the replay is valid), on a batch of the same
    shape whose contents changed (the replay's checks fail and the call runs
    as usual), and back on the first batch."""
    import torch
    from paper_2406_18111_gb300 import Apo, as_u32
    toks, off, _ = W.config3_windows(48, 1024, 16384, seed0=31)
    other = toks.copy()
    rng = np.random.default_rng(3)
    pos = rng.integers(0, len(other), size=len(other) // 50)
    other[pos] = rng.integers(0, 1000, size=len(pos)).astype(np.uint32)
    names = ("sa", "lcp", "cand_len", "cand_id", "cand_start", "sel_start", "sel_len", "sel_trace",
             "trace_len", "trace_start")

    def snap(r):
        d = {k: as_u32(getattr(r, k)).copy() for k in names}
        d["acc"] = r.cand_accepted.cpu().numpy().copy()
        d["rounds"] = r.rounds
        for k in ("cand_off", "sel_off", "trace_off"):
            d[k] = np.asarray(getattr(r, k)).copy()
        return d

    want = {}
    for name, t in (("a", toks), ("b", other)):
        want[name] = snap(apo.find_repeats_batched(dev(t, np.int32), off, 5))
    g = Apo(0)
    try:
        g.graph_mode(True)
        buf = torch.empty(len(toks), dtype=torch.int32, device="cuda")
        for name in ("a", "a", "a", "b", "b", "a"):
            buf.copy_(torch.from_numpy((toks if name == "a" else other).view(np.int32)))
            got = snap(g.find_repeats_batched(buf, off, 5, reuse=True))
            for k, v in want[name].items():
                assert np.array_equal(np.asarray(got[k]), np.asarray(v)), (name, k)
        st = g.graph_stats()
        # a: captured, replayed twice; b: the replay discarded, recaptured,
        # replayed; a again: discarded (the graph is b's), recaptured
        assert st["replays"] >= 3 and st["captures"] >= 2 and st["discarded"] >= 1, st
        g.graph_mode(False)
    finally:
        g.close()
