"""Pins for the oracle: brute force on short strings, the paper's worked
examples, published test vectors, invariants and the agreement of independent
formulations.  CPU only."""
import itertools
import struct

import numpy as np
import pytest

import oracle
import workloads as W


# ---------------------------------------------------------------- brute force
def bf_sa(S):
    """Sort the materialised suffixes (Python list order: a proper prefix is smaller)."""
    S = list(S)
    return sorted(range(len(S)), key=lambda i: S[i:])


def bf_lcp_pair(S, a, b):
    k = 0
    while a + k < len(S) and b + k < len(S) and S[a + k] == S[b + k]:
        k += 1
    return k


def bf_nonoverlapping_repeats(S):
    """All (length, start) with a second, non-overlapping occurrence."""
    n = len(S)
    out = set()
    for l in range(1, n // 2 + 1):
        for s in range(n - l + 1):
            for t in range(n - l + 1):
                if abs(s - t) >= l and S[s:s + l] == S[t:t + l]:
                    out.add((l, s))
                    break
    return out


def fnv1a64_py(data: bytes) -> int:
    h = 0xCBF29CE484222325
    for b in data:
        h = ((h ^ b) * 0x100000001B3) & 0xFFFFFFFFFFFFFFFF
    return h


def check_window(S, min_len):
    """Every oracle output for S against its definition."""
    S = list(S)
    n = len(S)
    sa = oracle.suffix_array(np.array(S, dtype=np.uint64)) if n else np.zeros(0, np.uint32)
    assert list(sa) == bf_sa(S)
    lc = oracle.lcp(np.array(S, dtype=np.uint64), sa)
    for i in range(n - 1):
        assert lc[i] == bf_lcp_pair(S, int(sa[i]), int(sa[i + 1]))
    if n:
        assert lc[n - 1] == 0
    rl, rs = oracle.candidates_raw(sa, lc)
    assert len(rl) == 2 * max(0, n - 1)
    reps = bf_nonoverlapping_repeats(S)
    for l, s in zip(rl, rs):
        if l > 0:
            assert (int(l), int(s)) in reps, (S, l, s)
    r = oracle.find_repeats(np.array(S, dtype=np.uint64), min_len)
    # candidate list: the filtered raw candidates, once each, in Alg. 2's order
    want = sorted({(int(l), int(s)) for l, s in zip(rl, rs) if l >= min_len},
                  key=lambda c: (-c[0], S[c[1]:c[1] + c[0]], c[1]))
    got = list(zip(r.cand_len.tolist(), r.cand_start.tolist()))
    assert got == want
    # id = number of suffixes whose first l tokens are smaller than the sub-string
    for l, s, cid in zip(r.cand_len.tolist(), r.cand_start.tolist(), r.cand_id.tolist()):
        sub = S[s:s + l]
        assert cid == sum(1 for j in range(n) if S[j:j + l] < sub)
    # greedy: taken iff it meets no interval taken before it
    acc = r.accepted.tolist()
    for k, (l, s) in enumerate(got):
        blocked = any(acc[j] and s < got[j][1] + got[j][0] and got[j][1] < s + l for j in range(k))
        assert acc[k] == (not blocked)
    for v in (1, 2):
        assert oracle.greedy(n, r.cand_len, r.cand_start, v).tolist() == acc
    # R in first-acceptance order; selected intervals by start
    taken = [got[k] for k in range(len(got)) if acc[k]]
    R = []
    for l, s in taken:
        if S[s:s + l] not in R:
            R.append(S[s:s + l])
    assert [list(S[s:s + l]) for l, s in zip(r.trace_len.tolist(), r.trace_start.tolist())] == R
    for t, sub in enumerate(R):
        starts = [s for l, s in taken if S[s:s + l] == sub]
        assert r.trace_start[t] == min(starts)
    sel = sorted((s, l) for l, s in taken)
    assert list(zip(r.sel_start.tolist(), r.sel_len.tolist())) == sel
    for s, l, t in zip(r.sel_start.tolist(), r.sel_len.tolist(), r.sel_trace.tolist()):
        assert S[s:s + l] == R[t]
    return r


# ---------------------------------------------------------------- hashing
def test_fnv1a64_published_vectors():
    assert oracle.fnv1a64(b"") == 0xCBF29CE484222325
    assert oracle.fnv1a64(b"a") == 0xAF63DC4C8601EC8C
    assert oracle.fnv1a64(b"foobar") == 0x85944171F73967E8


def test_task_serialisation_by_hand():
    ts = W.TaskStream(task_id=np.array([0x01020304, 7], np.uint32),
                      arg_off=np.array([0, 2, 3], np.uint32),
                      region=np.array([0xA1B2C3D4, 5, 9], np.uint32),
                      field_mask=np.array([0x1122334455667788, 1, 2], np.uint64),
                      priv=np.array([3, 0, 1], np.uint8))
    want0 = (struct.pack("<II", 0x01020304, 2)
             + struct.pack("<IQB", 0xA1B2C3D4, 0x1122334455667788, 3)
             + struct.pack("<IQB", 5, 1, 0))
    want1 = struct.pack("<II", 7, 1) + struct.pack("<IQB", 9, 2, 1)
    assert oracle.serialize_task(ts, 0) == want0
    assert oracle.serialize_task(ts, 1) == want1
    h = oracle.hash_tasks(ts)
    assert int(h[0]) == fnv1a64_py(want0) and int(h[1]) == fnv1a64_py(want1)


def test_hash_argument_order_and_fields_matter():
    base = dict(task_id=np.array([1, 1, 1, 1, 1], np.uint32),
                arg_off=np.array([0, 2, 4, 6, 8, 10], np.uint32))
    # t0 base, t1 arguments swapped, t2 another field mask, t3 another privilege, t4 = t0
    region = np.array([1, 2, 2, 1, 1, 2, 1, 2, 1, 2], np.uint32)
    mask = np.array([1, 1, 1, 1, 3, 1, 1, 1, 1, 1], np.uint64)
    priv = np.array([0, 1, 1, 0, 0, 1, 1, 1, 0, 1], np.uint8)
    h = oracle.hash_tasks(W.TaskStream(region=region, field_mask=mask, priv=priv, **base))
    # same regions in swapped order, a different field mask, a different privilege
    assert len(set(h[:4].tolist())) == 4
    assert h[0] == h[4]


def test_jacobi_stream(golden):
    g = golden("jacobi.json")
    ts = W.jacobi_tasks(g["iterations"])
    tok = oracle.hash_tasks(ts)
    cls = g["token_classes"]
    for i in range(len(cls)):
        for j in range(len(cls)):
            assert (tok[i] == tok[j]) == (cls[i] == cls[j])
    r = oracle.find_repeats(tok, g["min_len"])
    assert list(zip(r.sel_start.tolist(), r.sel_len.tolist())) == [tuple(x) for x in g["selected"]]
    assert len(r.trace_len) == g["n_traces"]


# ---------------------------------------------------------------- worked examples
@pytest.mark.parametrize("name", ["aabcbcbaa.json", "ababab.json"])
def test_worked_examples(golden, name):
    g = golden(name)
    S = [ord(c) for c in g["string"]]
    for ml, res in g["results"].items():
        r = check_window(S, int(ml))
        assert r.sa.tolist() == g["sa"]
        assert r.lcp.tolist() == g["lcp"]
        assert list(zip(r.sel_start.tolist(), r.sel_len.tolist())) == [tuple(x) for x in res["selected"]]
        got = ["".join(chr(S[s + k]) for k in range(l)) for l, s in zip(r.trace_len.tolist(), r.trace_start.tolist())]
        assert got == res["traces"]


def test_aabcbcbaa_raw_candidates(golden):
    g = golden("aabcbcbaa.json")
    S = [ord(c) for c in g["string"]]
    sa = oracle.suffix_array(S)
    rl, rs = oracle.candidates_raw(sa, oracle.lcp(S, sa))
    want = [(c["l"], st) for c in g["raw_candidates_per_pair"] for st in c["starts"]]
    assert list(zip(rl.tolist(), rs.tolist())) == want


def test_longest_repeat_claim_does_not_hold(golden):
    g = golden("abababa.json")
    S = [ord(c) for c in g["string"]]
    r = check_window(S, 1)
    assert r.sa.tolist() == g["sa"] and r.lcp.tolist() == g["lcp"]
    assert int(r.cand_len.max()) == g["max_candidate_length"]
    assert max(l for l, _ in bf_nonoverlapping_repeats(S)) == g["longest_nonoverlapping_repeat"]


# ---------------------------------------------------------------- brute force sweeps
def test_all_binary_strings_up_to_10():
    for n in range(0, 11):
        for S in itertools.product(range(2), repeat=n):
            check_window(S, 1 + (n % 3))


def test_all_ternary_strings_up_to_7():
    for n in range(1, 8):
        for S in itertools.product(range(3), repeat=n):
            check_window(S, 1 + (sum(S) % 2))


def test_random_strings_up_to_12():
    rng = W.uniform_int(77, 4000, 0, 1 << 30)
    k = 0
    for trial in range(400):
        n = int(rng[k] % 12) + 1
        sigma = int(rng[k + 1] % 4) + 1
        k += 2
        S = W.uniform_int(1000 + trial, n, 0, sigma - 1).tolist()
        check_window(S, 1 + trial % 3)


def test_unary_and_huge_tokens():
    check_window([5] * 12, 1)
    big = [0xFFFFFFFFFFFFFFFF, 0, 0xFFFFFFFFFFFFFFFF, 0, 1 << 63]
    check_window(big, 1)


# ---------------------------------------------------------------- larger cross-checks
@pytest.mark.parametrize("kind", ["periodic", "random", "runs"])
def test_sa_methods_and_lcp_methods_agree(kind):
    if kind == "periodic":
        S = W.config1_window(4096, seed=11)
    elif kind == "random":
        S = W.uniform_int(12, 4096, 0, 3)
    else:
        a, _ = W.config4_windows(3 * 1024)
        S = a
    S = np.asarray(S, dtype=np.uint64)
    sa = oracle.suffix_array(S, "direct")
    assert np.array_equal(np.sort(sa), np.arange(S.shape[0], dtype=np.uint32))
    assert np.array_equal(sa, oracle.suffix_array(S, "doubling"))
    assert np.array_equal(oracle.lcp(S, sa, "kasai"), oracle.lcp(S, sa, "direct"))


def _lce_strings():
    """Strings up to 2^16 tokens whose long repeats stress the LCE path:
    constant, period-2 and period-3 runs (up to 2^14 alone, at 2^16 as the
    three thirds of config 4's adversarial window), periodic
    windows with noise, random strings over small and large alphabets."""
    out = []
    for n in (1, 2, 7, 64, 1000, 4099, 1 << 14):
        out.append(np.zeros(n, np.uint64))
        out.append((np.arange(n) % 2).astype(np.uint64))
        out.append((np.arange(n) % 3).astype(np.uint64))
    a, _ = W.config4_windows(1 << 16)
    out.append(a.astype(np.uint64))
    out.append(np.asarray(W.config1_window(4096, seed=17), np.uint64))
    out.append(np.asarray(W.periodic_window(1 << 16, 37, 0.02, 50, 19), np.uint64))
    out.append(W.uniform_int(23, 1 << 16, 0, 1).astype(np.uint64))
    out.append(W.uniform_int(24, 5000, 0, 1 << 40).astype(np.uint64))
    return out


def test_lce_queries_equal_direct_comparison():
    """The sparse-table LCE equals the common prefix counted token by token
    (sampled pairs, every window; the equal-suffix case a == b included)."""
    for k, S in enumerate(_lce_strings()):
        n = S.shape[0]
        sa = oracle.suffix_array(S, "doubling")
        lc = oracle.lcp(S, sa)
        q = min(400, n * n)
        a = W.uniform_int(300 + k, q, 0, n - 1).astype(np.uint32)
        b = W.uniform_int(400 + k, q, 0, n - 1).astype(np.uint32)
        b[::17] = a[::17]
        got = oracle.lce(sa, lc, a, b)
        for x, y, g in zip(a.tolist(), b.tolist(), got.tolist()):
            m = min(n - x, n - y)
            eq = S[x:x + m] == S[y:y + m]
            want = m if eq.all() else int(np.argmin(eq))
            assert g == want, (k, x, y, g, want)


def test_candidate_order_lce_equals_direct():
    """Alg. 2's sort and the candidate ids are the same with sub-strings
    compared token by token and through LCE queries."""
    for k, S in enumerate(_lce_strings()):
        sa = oracle.suffix_array(S, "doubling")
        lc = oracle.lcp(S, sa)
        for ml in ((1, 5) if S.shape[0] < (1 << 14) else (5,)):
            d = oracle.find_repeats(S, ml, sa=sa, lcp_arr=lc, cmp="direct")
            e = oracle.find_repeats(S, ml, sa=sa, lcp_arr=lc, cmp="lce")
            for f in ("cand_len", "cand_id", "cand_start", "accepted", "sel_start", "sel_len", "sel_trace",
                      "trace_len", "trace_start"):
                assert np.array_equal(getattr(d, f), getattr(e, f)), (k, ml, f)


def test_greedy_variants_agree_on_config1():
    S = W.config1_window()
    r = oracle.find_repeats(S, 5)
    for v in (1, 2):
        assert np.array_equal(oracle.greedy(S.shape[0], r.cand_len, r.cand_start, v), r.accepted)
    # taken intervals are disjoint, the first candidate is the longest and is taken
    ss, sl = r.sel_start.astype(np.int64), r.sel_len.astype(np.int64)
    assert np.all(ss[1:] >= ss[:-1] + sl[:-1])
    assert r.accepted[0] == 1 and r.cand_len[0] == r.cand_len.max()
    assert sl.sum() <= S.shape[0]


# ---------------------------------------------------------------- matching
def test_ushers(golden):
    g = golden("ushers.json")
    toks, off = [], [0]
    for p in g["patterns"]:
        toks += [ord(c) for c in p]
        off.append(len(toks))
    text = [ord(c) for c in g["text"]]
    for naive in (False, True):
        e, i = oracle.match(toks, off, text, naive)
        assert list(zip(e.tolist(), i.tolist())) == [tuple(x) for x in g["matches"]]


def test_match_bruteforce_random():
    for trial in range(30):
        n = 200
        text = W.uniform_int(500 + trial, n, 0, 2).tolist()
        P = 12
        lens = W.uniform_int(600 + trial, P, 1, 6).tolist()
        pats = [W.uniform_int(700 + 31 * trial + p, lens[p], 0, 2).tolist() for p in range(P)]
        pats.append(pats[0])  # duplicate pattern: reported under both ids
        toks = [t for p in pats for t in p]
        off = np.cumsum([0] + [len(p) for p in pats])
        want = sorted((e, -len(pat), p) for p, pat in enumerate(pats) for e in range(len(pat) - 1, n)
                      if text[e - len(pat) + 1:e + 1] == pat)
        want = [(e, p) for e, _, p in want]
        for naive in (False, True):
            e, i = oracle.match(toks, off, text, naive)
            assert list(zip(e.tolist(), i.tolist())) == want


# ---------------------------------------------------------------- Sec. 4.4 sampling
def test_ruler_function_values():
    # Sec. 4.4: applied to 1, 2, 3, 4, ... the ruler function gives 0, 1, 0, 2, ...
    assert [oracle.ruler(i) for i in range(1, 9)] == [0, 1, 0, 2, 0, 1, 0, 3]
    # its powers of two: 1, 2, 1, 4, ...
    assert [2 ** oracle.ruler(i) for i in range(1, 5)] == [1, 2, 1, 4]


def test_ruler_schedule_paper_examples():
    # Sec. 4.4: with a buffer of four, the first task, the first two, the
    # third, then all four
    assert oracle.ruler_schedule(4, 1, 4) == [(1, 0, 1), (2, 0, 2), (3, 2, 1), (4, 0, 4)]
    # Fig. (buffer of size 8): after task i, the slice labelled i ends at i
    # with 2^ruler(i) tasks
    sched = oracle.ruler_schedule(8, 1, 8)
    assert [l for _, _, l in sched] == [1, 2, 1, 4, 1, 2, 1, 8]
    assert all(s + l == i for i, s, l in sched)
    # the buffer caps a slice, and so do the tokens that have arrived
    assert oracle.ruler_schedule(32, 1, 8)[15] == (16, 8, 8)
    assert oracle.ruler_schedule(1000, 250, 5000)[3] == (4, 0, 1000)


def test_ruler_schedule_total_work():
    # tokens analysed grow as n log(buffer / unit): per analysis point the
    # mean slice is unit * (1 + log2(buffer/unit) / 2) at most (Sec. 4.4)
    import math
    unit, buffer = 250, 5000
    for n in (10 ** 4, 10 ** 5, 10 ** 6):
        sched = oracle.ruler_schedule(n, unit, buffer)
        total = sum(l for _, _, l in sched)
        assert total <= n * (1 + math.log2(buffer / unit) / 2 + 1)
        assert total >= n  # every token is analysed at least once


def test_online_traces_slices():
    S = [j % 7 for j in range(3000)]
    res = oracle.online_traces(S, 250, 1000, 5)
    assert [r[:3] for r in res] == oracle.ruler_schedule(3000, 250, 1000)
    for i, start, length, tl, ts in res:
        # every trace lies inside its slice
        assert np.all(ts >= start) and np.all(ts + tl <= start + length)


# ---------------------------------------------------------------- TraceReplayer
# Sec. 4.3: traces enter a trie, pointers follow the stream through it, a
# pointer at the end of a trace completes it, the completed trace with the
# best score (length x capped appearance count, decayed by the tasks since
# its previous appearance, raised for a trace already replayed) is replayed.
# Expected values below are worked by hand from that description.
_TOK = {ch: i + 1 for i, ch in enumerate("abcdexy")}


def _s(text):
    return np.array([_TOK[ch] for ch in text], dtype=np.uint64)


def _rep(r):
    return list(zip(r.end.tolist(), r.length.tolist(), r.trace.tolist()))


def test_replay_periodic_single_trace():
    r = oracle.replay(_s("abc" * 5), [0], [3], [0])
    assert _rep(r) == [(2, 3, 0), (5, 3, 0), (8, 3, 0), (11, 3, 0), (14, 3, 0)]
    assert r.traced.tolist() == [1] * 15


def test_replay_waits_for_ingestion():
    # the trace enters at task 4: no pointer can follow it before, and the
    # pointers started at tasks 4 and 5 meet no edge of the trie
    r = oracle.replay(_s("abc" * 5), [0], [3], [4])
    assert _rep(r) == [(8, 3, 0), (11, 3, 0), (14, 3, 0)]
    assert r.traced.tolist() == [0] * 6 + [1] * 9


def test_replay_prefix_trace_completes_first():
    # "ab" ends one task before "abc": it is replayed and takes the pointer
    # that was on its way to "abc"
    r = oracle.replay(_s("abcabc"), [0, 0], [2, 3], [0, 0])
    assert _rep(r) == [(1, 2, 0), (4, 2, 0)]
    assert r.traced.tolist() == [1, 1, 0, 1, 1, 0]


def test_replay_longer_of_two_completed_traces():
    # "bc" (piece 0) and "abc" (piece 1) complete together: 3 x 1 > 2 x 1
    r = oracle.replay(_s("abcabc"), [1, 0], [2, 3], [0, 0])
    assert _rep(r) == [(2, 3, 1), (5, 3, 1)]


def test_replay_growing_trie():
    # "abd" is in the trie from the start, "abc" enters at task 2; the
    # pointer started at task 0 stands at "ab" then and continues into "abc"
    r = oracle.replay(_s("abcxabd"), [4, 0], [3, 3], [0, 2])
    assert _rep(r) == [(2, 3, 1), (6, 3, 0)]
    # with "axd" instead, that pointer died at task 1 ("a" has no edge b)
    r = oracle.replay(_s("abcxaxd"), [4, 0], [3, 3], [0, 2])
    assert _rep(r) == [(6, 3, 0)]


_BC_ABC = _s("xbc" * 4 + "abc" * 3)


def test_replay_appearance_count_and_cap():
    # "bc" appears alone four times, then with "abc" at tasks 14, 17, 20
    # no cap: bc scores 2 x 5, 2 x 6, 2 x 7 against abc's 3, 6, 9
    r = oracle.replay(_BC_ABC, [1, 12], [2, 3], [0, 0])
    assert r.length.tolist() == [2] * 7
    assert r.end.tolist() == [2, 5, 8, 11, 14, 17, 20]
    # cap 2: bc scores 2 x 2 = 4 against abc's 3 x 1, then 3 x 2 = 6 twice
    r = oracle.replay(_BC_ABC, [1, 12], [2, 3], [0, 0], cap=2)
    assert r.length.tolist() == [2, 2, 2, 2, 2, 3, 3]
    assert r.traced.tolist() == [0, 1, 1] * 4 + [0, 1, 1] + [1] * 6


def test_replay_decay():
    # half-life 1 task: the score is shifted right by the tasks since the
    # previous appearance.  Task 14: abc 3 (first appearance) > bc 10 >> 3;
    # task 17: abc 6 >> 3 = 0 < bc 12 >> 3 = 1; task 20: 9 >> 3 = 14 >> 3,
    # the tie goes to the longer abc
    r = oracle.replay(_BC_ABC, [1, 12], [2, 3], [0, 0], half_life=1)
    assert r.length.tolist() == [2, 2, 2, 2, 3, 2, 3]
    assert r.end.tolist() == [2, 5, 8, 11, 14, 17, 20]
    # a half-life of 4 tasks shifts by 3 // 4 = 0: as without decay
    r = oracle.replay(_BC_ABC, [1, 12], [2, 3], [0, 0], half_life=4)
    assert r.length.tolist() == [2] * 7


def test_replay_bonus_for_replayed_trace():
    # "cd" replayed at tasks 3 and 7; at task 11 abcd (4 x 1) meets cd
    # (2 x min(3, 2) = 4): a tie the longer trace wins, unless the bonus
    # (2 against 1) lifts the already replayed cd to 8.  Task 15: abcd
    # 4 x 2 = 8 against cd 4 (x 2 with the bonus): a tie again
    S = _s("xycd" * 2 + "abcd" * 2)
    r = oracle.replay(S, [2, 8], [2, 4], [0, 0], cap=2)
    assert r.length.tolist() == [2, 2, 4, 4]
    r = oracle.replay(S, [2, 8], [2, 4], [0, 0], cap=2, bonus=(2, 1))
    assert r.length.tolist() == [2, 2, 2, 4]
    assert r.end.tolist() == [3, 7, 11, 15]


def test_replay_maximum_trace_length():
    # a 5-task trace with a maximum length of 2 enters as ab, cd, e
    r = oracle.replay(_s("abcde" * 2), [0], [5], [0], max_len=2)
    assert _rep(r) == [(1, 2, 0), (3, 2, 1), (4, 1, 2), (6, 2, 0), (8, 2, 1), (9, 1, 2)]
    # equal strings report the smallest piece number
    r = oracle.replay(_s("abcabc"), [3, 0], [3, 3], [0, 0])
    assert _rep(r) == [(2, 3, 0), (5, 3, 0)]


def _replay_by_occurrences(S, starts, lens, ingest, max_len, cap, half_life, bonus):
    """The same replay decisions formulated over occurrences instead of
    pointers: an occurrence [s, e] of trace t is followed by a pointer iff
    s >= need(t) = max over j < |t| of (B(t[:j]) - j + 1) and E(t) - |t| + 1,
    with B(u) the earliest ingestion of a piece starting with u and E(t) the
    earliest of t itself (the pointer stands at t[:j] while task s + j - 1 is
    processed, and completes t at task s + |t| - 1); replays end where the
    first such occurrence starting after the previous replay ends."""
    S = [int(x) for x in S]
    n = len(S)
    pieces = []
    for a, l, g in zip(starts, lens, ingest):
        off = 0
        while off < l:
            m = l - off if not max_len else min(max_len, l - off)
            pieces.append((tuple(S[a + off:a + off + m]), int(g)))
            off += m
    first = {}
    for pid, (u, _) in enumerate(pieces):
        first.setdefault(u, pid)

    def birth(u):
        return min(g for v, g in pieces if v[:len(u)] == u)

    def own(u):  # the trace itself ends a pointer only once it is in the trie
        return min(g for v, g in pieces if v == u)

    need = {u: max([birth(u[:j]) - j + 1 for j in range(1, len(u))] + [own(u) - len(u) + 1]) for u in first}
    occ = {}  # end -> [(start, string)]
    for u in first:
        L = len(u)
        for s in range(0, n - L + 1):
            if tuple(S[s:s + L]) == u and s >= need[u]:
                occ.setdefault(s + L - 1, []).append((s, u))
    state = {u: [0, -1, False] for u in first}  # count, last, replayed
    out, traced, c = [], [0] * n, 0
    for e in range(n):
        D = [(s, u) for s, u in occ.get(e, []) if s >= c]
        if not D:
            continue
        best = None
        for s, u in D:
            cnt, last, rep = state[u]
            sh = (e - last) // half_life if (last >= 0 and half_life) else 0
            cnt += 1
            state[u][0], state[u][1] = cnt, e
            x = len(u) * (min(cnt, cap) if cap else cnt) * (bonus[0] if rep else bonus[1])
            sc = 0 if sh >= 64 else x >> sh
            if best is None or (sc, len(u)) > best[0]:
                best = ((sc, len(u)), u)
        u = best[1]
        state[u][2] = True
        out.append((e, len(u), first[u]))
        for j in range(e - len(u) + 1, e + 1):
            traced[j] = 1
        c = e + 1
    return out, traced


def test_replay_agrees_with_occurrence_formulation():
    rng = np.random.default_rng(7)
    for case in range(400):
        n = int(rng.integers(1, 80))
        per = int(rng.integers(1, 7))
        S = rng.integers(0, 3, size=per)[np.arange(n) % per]
        flip = rng.random(n) < 0.1
        S = np.where(flip, rng.integers(0, 3, size=n), S).astype(np.uint64)
        P = int(rng.integers(0, 6))
        lens = rng.integers(1, min(n, 8) + 1, size=P)
        starts = np.array([rng.integers(0, n - l + 1) for l in lens], dtype=np.int64)
        ingest = rng.integers(0, n + 3, size=P)
        max_len = int(rng.choice([0, 0, 2, 3]))
        cap = int(rng.choice([0, 1, 2, 4]))
        half_life = int(rng.choice([0, 1, 3]))
        bonus = [(1, 1), (2, 1), (17, 16), (1, 2)][int(rng.integers(0, 4))]
        r = oracle.replay(S, starts, lens, ingest, max_len, cap, half_life, bonus)
        exp, traced = _replay_by_occurrences(S, starts, lens, ingest, max_len, cap, half_life, bonus)
        assert _rep(r) == exp, case
        assert r.traced.tolist() == traced, case


# ---------------------------------------------------------------- Sec. 3 optimum
# The optimisation problem of Sec. 3 with every trace repeated (as stated, one
# trace equal to S would cover everything).  Hand-derived optima:
#   abab        ab|ab                          coverage 4, 2 intervals, 1 trace
#   abcab       ab at 0 and 3                  4, 2, 1
#   abababab    ab x 4 beats abab x 2 on intervals  8, 4, 1
#   abcd        nothing repeats                0, 0, 0
#   abcabcxabc  x occurs once and is never covered; abc x 3   9, 3, 1
#   aabaab      aab x 2                        6, 2, 1
def test_optimum_hand_cases():
    cases = {"abab": (4, 2, 1), "abcab": (4, 2, 1), "abababab": (8, 4, 1), "abcd": (0, 0, 0),
             "abcabcxabc": (9, 3, 1), "aabaab": (6, 2, 1), "aaaa": (4, 2, 1)}
    for text, want in cases.items():
        (cov, cnt, dist), _ = oracle.optimum(_s(text), 2)
        assert (cov, cnt, dist) == want, text
    # min length 3: "abab" has no repeat of length 3 that fits twice
    assert oracle.optimum(_s("abab"), 3)[0] == (0, 0, 0)
    # xyabxyab: xy|ab|xy|ab (4 intervals, 2 traces) beats xyab x 2 (2
    # intervals, 1 trace): more intervals come before fewer traces
    assert oracle.optimum(_s("xyabxyab"), 2)[0] == (8, 4, 2)


def _check_witness(S, m, best, wit):
    S = [int(x) for x in S]
    last = -1
    groups = {}
    for a, l in wit:
        assert a > last and l >= m and a + l <= len(S)
        last = a + l - 1
        groups.setdefault(tuple(S[a:a + l]), []).append(a)
    assert all(len(v) >= 2 for v in groups.values())
    assert best == (sum(l for _, l in wit), len(wit), len(groups))


def _optimum_mask_first(S, m):
    """The same optimum enumerated another way: every set of covered
    positions, then every split of its maximal runs into pieces >= m."""
    S = [int(x) for x in S]
    n = len(S)
    best = (0, 0, 0)

    def splits(a, b):
        if a == b:
            yield []
            return
        for L in range(m, b - a + 1):
            for rest in splits(a + L, b):
                yield [(a, L)] + rest

    for mask in range(1 << n):
        runs, j = [], 0
        while j < n:
            if mask >> j & 1:
                k = j
                while k < n and mask >> k & 1:
                    k += 1
                runs.append((j, k))
                j = k
            else:
                j += 1
        if any(b - a < m for a, b in runs):
            continue
        parts = [list(splits(a, b)) for a, b in runs]
        for combo in itertools.product(*parts):
            ivs = [iv for part in combo for iv in part]
            g = {}
            for a, l in ivs:
                g[tuple(S[a:a + l])] = g.get(tuple(S[a:a + l]), 0) + 1
            if any(c < 2 for c in g.values()):
                continue
            key = (sum(l for _, l in ivs), len(ivs), -len(g))
            if key > (best[0], best[1], -best[2]):
                best = (key[0], key[1], -key[2])
    return best


def test_optimum_invariants_and_second_enumeration():
    rng = np.random.default_rng(5)
    for case in range(120):
        n = int(rng.integers(1, 11))
        m = int(rng.integers(1, 4)) if n <= 8 else int(rng.integers(2, 4))
        S = rng.integers(0, int(rng.integers(1, 4)), size=n).astype(np.uint64)
        best, wit = oracle.optimum(S, m)
        _check_witness(S, m, best, wit)
        assert best == _optimum_mask_first(S, m), (S.tolist(), m)
        # reversal and renaming of the alphabet keep the optimum
        assert oracle.optimum(S[::-1].copy(), m)[0] == best
        assert oracle.optimum((S * 7 + 3) % 11, m)[0] == best
        # a solution for a prefix is a solution for S
        if n > 1:
            assert oracle.optimum(S[:-1], m)[0][0] <= best[0]


def test_alg2_feasible_part_never_beats_the_optimum():
    rng = np.random.default_rng(6)
    for case in range(60):
        n = int(rng.integers(4, 15))
        per = int(rng.integers(2, 5))
        S = rng.integers(0, 3, size=per)[np.arange(n) % per]
        S = np.where(rng.random(n) < 0.15, rng.integers(0, 3, size=n), S).astype(np.uint64)
        r = oracle.find_repeats(S, 2)
        groups = {}
        for a, l in zip(r.sel_start.tolist(), r.sel_len.tolist()):
            groups.setdefault(tuple(S[a:a + l].tolist()), []).append(l)
        feasible = sum(sum(v) for v in groups.values() if len(v) >= 2)
        assert feasible <= oracle.optimum(S, 2)[0][0]
