"""Oracle for the trace finder -- TEST INFRASTRUCTURE ONLY.

A plain CPU restatement of the analysis in ``apo_oracle.cpp`` (C++, built with
g++ into ``liboracle.so`` next to this file) plus thin numpy wrappers.  Only the
test-suite, the smoke check and the CPU-baseline leg of the benchmark may use
it; the library's product path never does.  It shares no code with the CUDA
library.

Parity unpinned: none -- every routine is pinned by ``tests/test_oracle_pins.py``
(brute force on short strings, the paper's worked examples, published test
vectors, invariants, and agreement of independent formulations).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "apo_oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile liboracle.so with g++ (host code only; builds on x86 and Arm)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", _SRC, "-o", tmp])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        U64 = ctypes.c_uint64
        L.ora_fnv1a64.restype = U64
        L.ora_fnv1a64.argtypes = [P, U64]
        L.ora_serialize_task.restype = U64
        L.ora_serialize_task.argtypes = [U64, P, P, P, P, P, P, U64]
        L.ora_hash_tasks.restype = None
        L.ora_hash_tasks.argtypes = [U64, P, P, P, P, P, P]
        for f in ("ora_suffix_array", "ora_suffix_array_doubling"):
            getattr(L, f).restype = None
            getattr(L, f).argtypes = [P, U64, P]
        for f in ("ora_lcp_direct", "ora_lcp_kasai"):
            getattr(L, f).restype = None
            getattr(L, f).argtypes = [P, U64, P, P]
        L.ora_lce.restype = None
        L.ora_lce.argtypes = [P, P, U64, P, P, U64, P]
        L.ora_candidates_raw.restype = U64
        L.ora_candidates_raw.argtypes = [U64, P, P, P, P]
        L.ora_greedy.restype = None
        L.ora_greedy.argtypes = [U64, U64, P, P, P, ctypes.c_int]
        L.ora_find_repeats.restype = None
        L.ora_find_repeats.argtypes = [P, U64, P, P, ctypes.c_uint32, ctypes.c_int, ctypes.c_int] + [P] * 10
        L.ora_match.restype = U64
        L.ora_match.argtypes = [P, P, U64, P, U64, ctypes.c_int, P, P, U64]
        L.ora_optimum.restype = U64
        L.ora_optimum.argtypes = [P, U64, U64, P, P, P]
        L.ora_replay.restype = U64
        L.ora_replay.argtypes = [P, U64, U64, P, P, P] + [U64] * 5 + [P, P, P, U64, P]
        _lib = L
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _tok(S) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(S).astype(np.uint64))


def fnv1a64(data: bytes) -> int:
    b = np.frombuffer(bytes(data), dtype=np.uint8).copy() if len(data) else np.zeros(1, np.uint8)
    return int(lib().ora_fnv1a64(_p(b), len(data)))


def serialize_task(ts, t: int) -> bytes:
    arrs = [np.ascontiguousarray(x) for x in (ts.task_id, ts.arg_off, ts.region, ts.field_mask, ts.priv)]
    n = lib().ora_serialize_task(t, *[_p(a) for a in arrs], None, 0)
    out = np.zeros(max(1, n), dtype=np.uint8)
    lib().ora_serialize_task(t, *[_p(a) for a in arrs], _p(out), n)
    return out[:n].tobytes()


def hash_tasks(ts) -> np.ndarray:
    arrs = [np.ascontiguousarray(ts.task_id, dtype=np.uint32),
            np.ascontiguousarray(ts.arg_off, dtype=np.uint32),
            np.ascontiguousarray(ts.region, dtype=np.uint32),
            np.ascontiguousarray(ts.field_mask, dtype=np.uint64),
            np.ascontiguousarray(ts.priv, dtype=np.uint8)]
    n = ts.n_tasks
    out = np.zeros(n, dtype=np.uint64)
    lib().ora_hash_tasks(n, *[_p(a) for a in arrs], _p(out))
    return out


def suffix_array(S, method: str = "direct") -> np.ndarray:
    S = _tok(S)
    sa = np.zeros(S.shape[0], dtype=np.uint32)
    f = lib().ora_suffix_array if method == "direct" else lib().ora_suffix_array_doubling
    f(_p(S), S.shape[0], _p(sa))
    return sa


def lcp(S, sa, method: str = "kasai") -> np.ndarray:
    S = _tok(S)
    sa = np.ascontiguousarray(sa, dtype=np.uint32)
    out = np.zeros(S.shape[0], dtype=np.uint32)
    f = lib().ora_lcp_kasai if method == "kasai" else lib().ora_lcp_direct
    f(_p(S), S.shape[0], _p(sa), _p(out))
    return out


def lce(sa, lcp_arr, a, b) -> np.ndarray:
    """lcp of the suffixes at a[k] and b[k] by range minima over the LCP array."""
    sa = np.ascontiguousarray(sa, dtype=np.uint32)
    lcp_arr = np.ascontiguousarray(lcp_arr, dtype=np.uint32)
    a = np.ascontiguousarray(a, dtype=np.uint32)
    b = np.ascontiguousarray(b, dtype=np.uint32)
    out = np.zeros(max(1, a.shape[0]), np.uint64)
    lib().ora_lce(_p(sa), _p(lcp_arr), sa.shape[0], _p(a), _p(b), a.shape[0], _p(out))
    return out[:a.shape[0]]


def candidates_raw(sa, lcp_arr):
    sa = np.ascontiguousarray(sa, dtype=np.uint32)
    lcp_arr = np.ascontiguousarray(lcp_arr, dtype=np.uint32)
    n = sa.shape[0]
    L = np.zeros(max(1, 2 * n), dtype=np.uint32)
    Sx = np.zeros(max(1, 2 * n), dtype=np.uint32)
    m = lib().ora_candidates_raw(n, _p(sa), _p(lcp_arr), _p(L), _p(Sx))
    return L[:m], Sx[:m]


def greedy(n: int, l, s, variant: int = 0) -> np.ndarray:
    l = np.ascontiguousarray(l, dtype=np.uint32)
    s = np.ascontiguousarray(s, dtype=np.uint32)
    acc = np.zeros(max(1, l.shape[0]), dtype=np.uint8)
    lib().ora_greedy(n, l.shape[0], _p(l), _p(s), _p(acc), variant)
    return acc[:l.shape[0]]


@dataclass
class Repeats:
    sa: np.ndarray
    lcp: np.ndarray
    cand_len: np.ndarray
    cand_id: np.ndarray
    cand_start: np.ndarray
    accepted: np.ndarray
    sel_start: np.ndarray
    sel_len: np.ndarray
    sel_trace: np.ndarray
    trace_len: np.ndarray
    trace_start: np.ndarray


_CMP = {"direct": 0, "lce": 1, "auto": 2}


def find_repeats(S, min_len: int, greedy_variant: int = 0, sa_method: str = "direct",
                 sa=None, lcp_arr=None, cmp: str = "auto") -> Repeats:
    """Alg. 2 end to end on one window (SA, LCP, candidates, greedy, R).

    ``cmp`` selects how the candidate sort and the id search compare
    sub-strings: "direct" token by token, "lce" by LCE queries over the SA
    and LCP, "auto" token by token up to 2^16 tokens and by LCE above."""
    S = _tok(S)
    n = S.shape[0]
    if sa is None:
        sa = suffix_array(S, sa_method)
    if lcp_arr is None:
        lcp_arr = lcp(S, sa)
    sa = np.ascontiguousarray(sa, dtype=np.uint32)
    lcp_arr = np.ascontiguousarray(lcp_arr, dtype=np.uint32)
    cap = max(1, 2 * n)
    cl, ci, cs = (np.zeros(cap, np.uint32) for _ in range(3))
    acc = np.zeros(cap, np.uint8)
    ss, sl, st, tl, tst = (np.zeros(max(1, n), np.uint32) for _ in range(5))
    counts = np.zeros(3, np.uint64)
    lib().ora_find_repeats(_p(S), n, _p(sa), _p(lcp_arr), min_len, greedy_variant, _CMP[cmp],
                           _p(cl), _p(ci), _p(cs), _p(acc), _p(ss), _p(sl), _p(st), _p(tl), _p(tst),
                           _p(counts))
    m, k, t = (int(c) for c in counts)
    return Repeats(sa, lcp_arr, cl[:m], ci[:m], cs[:m], acc[:m], ss[:k], sl[:k], st[:k], tl[:t], tst[:t])


def match(pat_tokens, pat_off, stream, naive: bool = False):
    """All (end, pattern) occurrences by end, then pattern length descending, then id."""
    pt = _tok(pat_tokens)
    po = np.ascontiguousarray(pat_off, dtype=np.uint64)
    st = _tok(stream)
    P = po.shape[0] - 1
    cnt = lib().ora_match(_p(pt), _p(po), P, _p(st), st.shape[0], int(naive), None, None, 0)
    e = np.zeros(max(1, cnt), np.uint32)
    i = np.zeros(max(1, cnt), np.uint32)
    lib().ora_match(_p(pt), _p(po), P, _p(st), st.shape[0], int(naive), _p(e), _p(i), cnt)
    return e[:cnt], i[:cnt]


def ruler(i: int) -> int:
    """The ruler function of Sec. 4.4: how many times 2 divides i (i >= 1)."""
    r = 0
    while i % 2 == 0:
        i //= 2
        r += 1
    return r


def ruler_schedule(n_tokens: int, unit: int, buffer: int):
    """The analysis slices of Sec. 4.4's sampling over a stream of n_tokens:
    after every `unit` tokens (point i = 1, 2, ...), the most recent
    unit * 2^ruler(i) tokens, at most the buffer and what has arrived.
    Returns [(i, start, length)]."""
    out = []
    for i in range(1, n_tokens // unit + 1):
        end = i * unit
        length = min(unit * 2 ** ruler(i), buffer, end)
        out.append((i, end - length, length))
    return out


def online_traces(S, unit: int, buffer: int, min_len: int):
    """Alg. 1's TraceFinder with the ruler sampling: Alg. 2 on every slice
    of ruler_schedule, traces in stream coordinates.  Returns
    [(i, start, length, trace_len, trace_start)]."""
    S = np.asarray(S)
    out = []
    for i, start, length in ruler_schedule(len(S), unit, buffer):
        r = find_repeats(S[start:start + length].astype(np.uint64), min_len)
        out.append((i, start, length, r.trace_len.astype(np.uint32),
                    r.trace_start.astype(np.uint64) + np.uint64(start)))
    return out


@dataclass
class Replay:
    end: np.ndarray      # task index where each replayed trace ends
    length: np.ndarray   # its length
    trace: np.ndarray    # smallest piece number with its string
    traced: np.ndarray   # u8 per task: 1 = inside a replay


def replay(S, tr_start, tr_len, tr_ingest, max_len: int = 0, cap: int = 0, half_life: int = 0,
           bonus=(1, 1)) -> Replay:
    """Alg. 1's TraceReplayer (Sec. 4.3), task by task: candidate trace q is
    S[tr_start[q] : tr_start[q] + tr_len[q]] and enters the trie at task
    tr_ingest[q]; see ora_replay for the steps and the score."""
    S = _tok(S)
    n = S.shape[0]
    st = np.ascontiguousarray(tr_start, dtype=np.uint64)
    ln = np.ascontiguousarray(tr_len, dtype=np.uint64)
    ig = np.ascontiguousarray(tr_ingest, dtype=np.uint64)
    P = st.shape[0]
    assert ln.shape[0] == P and ig.shape[0] == P
    assert all(int(l) >= 1 and int(a) + int(l) <= n for a, l in zip(st, ln))
    cap_r = n + 1
    e = np.zeros(cap_r, np.uint32)
    l = np.zeros(cap_r, np.uint32)
    t = np.zeros(cap_r, np.uint32)
    traced = np.zeros(max(1, n), np.uint8)
    r = lib().ora_replay(_p(S), n, P, _p(st), _p(ln), _p(ig), max_len, cap, half_life, bonus[0], bonus[1],
                         _p(e), _p(l), _p(t), cap_r, _p(traced))
    return Replay(e[:r], l[:r], t[:r], traced[:n])


def optimum(S, min_len: int):
    """Sec. 3's optimisation problem with repeated traces, by exhaustive
    enumeration (small n only): ((coverage, intervals, |T|), [(start, len)])
    of one optimal interval set."""
    S = _tok(S)
    n = S.shape[0]
    best = np.zeros(3, np.uint64)
    ws = np.zeros(max(1, n), np.uint32)
    wl = np.zeros(max(1, n), np.uint32)
    k = lib().ora_optimum(_p(S), n, min_len, _p(best), _p(ws), _p(wl))
    return (int(best[0]), int(best[1]), int(best[2])), list(zip(ws[:k].tolist(), wl[:k].tolist()))


def ingestion_points(submit, ready, lag0: int, growth: int = 2):
    """Sec. 4.5's agreed ingestion across nodes, sequentially: analysis j,
    submitted at operation submit[j], is ingested when operation
    submit[j] + lag_j is reached on every node; ready[r][j] is the operation
    count at which node r has the result (it waits at the ingestion point if
    that is later); if any node waited, the lag of the next analysis grows by
    `growth` (lag_0 = lag0).  Returns (points, waited, lags)."""
    points, waited, lags = [], [], []
    lag = lag0
    for j, s in enumerate(submit):
        p = int(s) + lag
        w = any(int(r[j]) > p for r in ready)
        points.append(p)
        waited.append(w)
        lags.append(lag)
        if w:
            lag *= growth
    return points, waited, lags
