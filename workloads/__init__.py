"""Seeded synthetic inputs for the trace-finder workloads.

These generators produce the task streams and token windows that both the
oracle and the CUDA path consume.  They hold none of the method's arithmetic:
no hashing of descriptors, no suffix sorting, no repeat selection.  Every
random draw comes from splitmix64 (Steele, Lea & Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), evaluated counter-style so that
any element can be produced independently of the others.

The paper's applications (S3D, HTR, cuPyNumeric CFD/TorchSWE, FlexFlow,
Sec. 6) are not available; the shapes below stand in for their task streams:
loops whose bodies repeat, interleaved with irregular tasks (Sec. 4.2,
"Existing Techniques"), traces longer than a few thousand tasks, and task
descriptors made of a task id plus ordered region arguments (Sec. 2).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix64(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def splitmix64(seed: int, count: int, stream: int = 0) -> np.ndarray:
    """``count`` outputs of splitmix64 for (seed, stream), as uint64.

    Output k is mix(base + (k+1) * gamma), the k-th value a sequential
    splitmix64 generator started at ``base`` would return; ``base`` itself is
    one mix of the seed and the stream number so that streams do not overlap.
    """
    with np.errstate(over="ignore"):
        base = _mix64(np.array([(seed * 0x100000001B3 + stream * 0x9E3779B9 + 1) & 0xFFFFFFFFFFFFFFFF],
                               dtype=np.uint64))[0]
        k = np.arange(1, count + 1, dtype=np.uint64)
        return _mix64(base + k * _GAMMA)


def uniform_int(seed: int, count: int, lo: int, hi: int, stream: int = 0) -> np.ndarray:
    """``count`` integers uniform on [lo, hi] (inclusive), as int64."""
    r = splitmix64(seed, count, stream)
    return (r % np.uint64(hi - lo + 1)).astype(np.int64) + lo


def uniform01(seed: int, count: int, stream: int = 0) -> np.ndarray:
    """``count`` doubles uniform on [0, 1) from the top 53 bits."""
    r = splitmix64(seed, count, stream)
    return (r >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def distinct_positions(seed: int, n: int, k: int, stream: int = 0) -> np.ndarray:
    """``k`` distinct positions out of [0, n): a seeded random permutation cut at k."""
    if k <= 0:
        return np.zeros(0, dtype=np.int64)
    keys = splitmix64(seed, n, stream)
    return np.argsort(keys, kind="stable")[:k].astype(np.int64)


def log_uniform_int(u: np.ndarray, lo: int, hi: int) -> np.ndarray:
    """floor(exp(U[ln lo, ln hi])) for uniforms ``u`` in [0, 1), clamped to [lo, hi]."""
    v = np.floor(np.exp(math.log(lo) + u * (math.log(hi) - math.log(lo)))).astype(np.int64)
    return np.clip(v, lo, hi)


# --------------------------------------------------------------------------
# Token windows
# --------------------------------------------------------------------------

def periodic_window(n: int, period: int, noise_frac: float, alphabet: int, seed: int) -> np.ndarray:
    """A loop body of ``period`` tokens (0..period-1) repeated over n positions,
    with exactly floor(noise_frac * n) distinct positions replaced by tokens
    uniform on [0, alphabet).  Returns uint32[n]."""
    s = (np.arange(n, dtype=np.int64) % period).astype(np.uint32)
    k = int(math.floor(noise_frac * n))
    pos = distinct_positions(seed, n, k, stream=1)
    s[pos] = uniform_int(seed, k, 0, alphabet - 1, stream=2).astype(np.uint32)
    return s


def config1_window(n: int = 4096, seed: int = 1) -> np.ndarray:
    """Single window: 50-task loop body, 5% noise over an alphabet of 1,000."""
    return periodic_window(n, 50, 0.05, 1000, seed)


def config3_windows(n_windows: int = 512, lo: int = 1024, hi: int = 262144, seed0: int = 3):
    """Batched windows: log-uniform lengths in [lo, hi], period U{3..5000},
    5% noise over an alphabet of 1,000; window w uses seed seed0 + w.
    Returns (tokens uint32[sum L], offsets uint64[n_windows + 1], periods)."""
    lens, periods, parts = [], [], []
    for w in range(n_windows):
        seed = seed0 + w
        u = uniform01(seed, 1, stream=10)
        L = int(log_uniform_int(u, lo, hi)[0])
        P = int(uniform_int(seed, 1, 3, 5000, stream=11)[0])
        lens.append(L)
        periods.append(P)
        parts.append(periodic_window(L, P, 0.05, 1000, seed))
    off = np.zeros(n_windows + 1, dtype=np.uint64)
    off[1:] = np.cumsum(np.array(lens, dtype=np.uint64))
    tokens = np.concatenate(parts) if parts else np.zeros(0, dtype=np.uint32)
    return tokens, off, np.array(periods, dtype=np.int64)


def config4_windows(n: int = 1 << 24, seed: int = 4):
    """Adversarial pair: window A = a constant run, a period-2 run and a
    period-3 run in equal thirds (m = floor(n/3)); window B = n uniform u32."""
    m = n // 3
    a = np.empty(n, dtype=np.uint32)
    a[:m] = 0
    j = np.arange(m, 2 * m, dtype=np.int64)
    a[m:2 * m] = (1 + ((j - m) % 2)).astype(np.uint32)
    j = np.arange(2 * m, n, dtype=np.int64)
    a[2 * m:] = (3 + ((j - 2 * m) % 3)).astype(np.uint32)
    b = (splitmix64(seed, n, stream=3) >> np.uint64(32)).astype(np.uint32)
    return a, b


# --------------------------------------------------------------------------
# Task descriptors
# --------------------------------------------------------------------------

@dataclass
class TaskStream:
    """Structure-of-arrays task descriptors.

    task_id[N]     u32   task (function) identifier
    arg_off[N + 1] u32   CSR offsets of each task's region arguments, in issue order
    region[M]      u32   logical region id of each argument
    field_mask[M]  u64   fields of the region the argument touches
    priv[M]        u8    privilege (0 read, 1 write, 2 read-write, 3 reduce)
    """
    task_id: np.ndarray
    arg_off: np.ndarray
    region: np.ndarray
    field_mask: np.ndarray
    priv: np.ndarray

    @property
    def n_tasks(self) -> int:
        return int(self.task_id.shape[0])


def _descriptor_pool(count: int, seed: int, stream: int):
    tid = (splitmix64(seed, count, stream) >> np.uint64(32)).astype(np.uint32)
    nargs = uniform_int(seed, count, 1, 8, stream + 1)
    off = np.zeros(count + 1, dtype=np.int64)
    off[1:] = np.cumsum(nargs)
    m = int(off[-1])
    region = (splitmix64(seed, m, stream + 2) >> np.uint64(32)).astype(np.uint32)
    mask = splitmix64(seed, m, stream + 3)
    priv = uniform_int(seed, m, 0, 3, stream + 4).astype(np.uint8)
    return tid, nargs, off, region, mask, priv


def config2_tasks(n: int = 1 << 20, seed: int = 2, noise_frac: float = 0.01,
                  pool_size: int = 1 << 16) -> TaskStream:
    """Nested loop task stream: position j has o = j mod 3000, b = o div 120,
    q = o mod 120; q < 119 issues inner task (q mod 7) of 7 fixed descriptors,
    q = 119 issues body b's "check" task (a fixed descriptor whose first region
    is base + b).  floor(noise_frac * n) distinct positions are replaced by a
    descriptor drawn uniformly from a pool of ``pool_size`` random ones."""
    n_inner, n_check = 7, 25
    total = n_inner + n_check + pool_size
    tid, nargs, off, region, mask, priv = _descriptor_pool(total, seed, stream=20)
    # check descriptors share one task id and differ only in the first region
    check_tid = tid[n_inner]
    base_region = np.uint32(0x40000000)
    for b in range(n_check):
        d = n_inner + b
        tid[d] = check_tid
        region[off[d]] = base_region + np.uint32(b)
    j = np.arange(n, dtype=np.int64)
    o = j % 3000
    b = o // 120
    q = o % 120
    d = np.where(q < 119, q % 7, n_inner + b).astype(np.int64)
    k = int(math.floor(noise_frac * n))
    pos = distinct_positions(seed, n, k, stream=30)
    d[pos] = n_inner + n_check + uniform_int(seed, k, 0, pool_size - 1, stream=31)
    return tasks_from_pool(d, tid, nargs, off, region, mask, priv)


def tasks_from_pool(d, tid, nargs, off, region, mask, priv) -> TaskStream:
    """Materialise the SoA stream that issues pool descriptors d[0], d[1], ..."""
    na = nargs[d]
    arg_off = np.zeros(d.shape[0] + 1, dtype=np.int64)
    arg_off[1:] = np.cumsum(na)
    m = int(arg_off[-1])
    src = np.repeat(off[:-1][d] - arg_off[:-1], na) + np.arange(m, dtype=np.int64)
    return TaskStream(task_id=tid[d].astype(np.uint32),
                      arg_off=arg_off.astype(np.uint32),
                      region=region[src].astype(np.uint32),
                      field_mask=mask[src].astype(np.uint64),
                      priv=priv[src].astype(np.uint8))


def jacobi_tasks(iters: int = 4) -> TaskStream:
    """The Jacobi main-loop stream of Fig. 1b: DOT(R,x,t1) SUB(b,t1,t2)
    DIV(t2,d,x') with x alternating between two regions x1 and x2.  The first
    two arguments are inputs (read), the third the output (write)."""
    R, b, d, x1, x2, t1, t2 = 1, 2, 3, 4, 5, 6, 7
    DOT, SUB, DIV = 100, 101, 102
    seq = []
    for it in range(iters):
        xin, xout = (x1, x2) if it % 2 == 0 else (x2, x1)
        seq += [(DOT, (R, xin, t1)), (SUB, (b, t1, t2)), (DIV, (t2, d, xout))]
    tid = np.array([t for t, _ in seq], dtype=np.uint32)
    arg_off = np.arange(0, 3 * len(seq) + 1, 3, dtype=np.uint32)
    region = np.array([r for _, a in seq for r in a], dtype=np.uint32)
    mask = np.ones(region.shape[0], dtype=np.uint64)
    priv = np.array([0, 0, 1] * len(seq), dtype=np.uint8)
    return TaskStream(tid, arg_off, region, mask, priv)


# --------------------------------------------------------------------------
# Matching workload
# --------------------------------------------------------------------------

def match_stream(n: int = 1 << 26, seed: int = 5) -> np.ndarray:
    """A token stream made of back-to-back periodic segments (period U{3..5000},
    length log-uniform in [4096, 2^20], 5% noise over 1,000 tokens)."""
    out = np.empty(n, dtype=np.uint32)
    pos, w = 0, 0
    while pos < n:
        s = seed * 1000003 + w
        L = int(log_uniform_int(uniform01(s, 1, stream=40), 4096, 1 << 20)[0])
        P = int(uniform_int(s, 1, 3, 5000, stream=41)[0])
        L = min(L, n - pos)
        out[pos:pos + L] = periodic_window(L, P, 0.05, 1000, s)
        pos += L
        w += 1
    return out


def match_patterns(stream: np.ndarray, n_patterns: int = 10000, lo: int = 5, hi: int = 2000,
                   seed: int = 5):
    """Candidate traces to match: lengths log-uniform in [lo, hi]; even-numbered
    patterns are copies of the stream at random offsets (guaranteed hits), odd
    ones are drawn from the stream's alphabet at random.
    Returns (tokens uint32[sum len], offsets uint64[n_patterns + 1])."""
    lens = log_uniform_int(uniform01(seed, n_patterns, stream=50), lo, hi)
    hi_eff = max(1, int(stream.shape[0]))
    lens = np.minimum(lens, hi_eff)
    starts = uniform_int(seed, n_patterns, 0, max(0, hi_eff - 1), stream=51)
    parts = []
    for p in range(n_patterns):
        L = int(lens[p])
        if p % 2 == 0:
            st = int(min(starts[p], hi_eff - L))
            parts.append(stream[st:st + L].copy())
        else:
            parts.append(uniform_int(seed * 7919 + p, L, 0, 999, stream=52).astype(np.uint32))
    off = np.zeros(n_patterns + 1, dtype=np.uint64)
    off[1:] = np.cumsum(lens.astype(np.uint64))
    return np.concatenate(parts).astype(np.uint32), off


def served_requests(duration_s: float = 30.0, rate: float = 2000.0, lo: int = 4096,
                    hi: int = 1 << 20, seed: int = 5):
    """Poisson analysis requests: arrival times (s) and window lengths
    log-uniform in [lo, hi]; request r's tokens are periodic_window(L_r, P_r,
    0.05, 1000, seed') with P_r uniform on 3..5000.  Returns (arrival, L, P)."""
    mean = rate * duration_s
    cap = int(mean + 10 * math.sqrt(mean) + 16)
    gaps = -np.log1p(-uniform01(seed, cap, stream=60)) / rate
    t = np.cumsum(gaps)
    k = int(np.searchsorted(t, duration_s))
    t = t[:k]
    L = log_uniform_int(uniform01(seed, k, stream=61), lo, hi)
    P = uniform_int(seed, k, 3, 5000, stream=62)
    return t, L, P


def served_window(r: int, L: int, P: int, seed: int = 5) -> np.ndarray:
    """Tokens of served request r (see served_requests)."""
    return periodic_window(int(L), int(P), 0.05, 1000, seed * 1000033 + r)


# --------------------------------------------------------------------------
# Trace replay inputs
# --------------------------------------------------------------------------

def replay_stream(n: int = 1 << 20, seed: int = 6) -> np.ndarray:
    """A task stream whose loop structure changes over time: back-to-back
    phases (length log-uniform in [2^14, 2^17]), each a period-P loop
    (P uniform on 20..600) with 1% noise over 2^16 tokens.  uint32[n]."""
    out = np.empty(n, dtype=np.uint32)
    pos, w = 0, 0
    while pos < n:
        s = seed * 1000003 + w
        L = int(log_uniform_int(uniform01(s, 1, stream=70), 1 << 14, 1 << 17)[0])
        P = int(uniform_int(s, 1, 20, 600, stream=71)[0])
        L = min(L, n - pos)
        out[pos:pos + L] = periodic_window(L, P, 0.01, 1 << 16, s)
        pos += L
        w += 1
    return out


def replay_random_traces(n: int, n_traces: int, seed: int, lo: int = 1, hi: int = 300):
    """Candidate traces as random slices of a length-n stream: lengths
    log-uniform in [lo, min(hi, n)], starts uniform, ingestion tasks uniform
    on [0, n + n // 8] (some never enter).  Returns (start, length, ingest)
    as uint32 arrays."""
    hi = max(lo, min(hi, n))
    L = log_uniform_int(uniform01(seed, n_traces, stream=80), lo, hi).astype(np.int64)
    u = uniform01(seed, n_traces, stream=81)
    start = np.floor(u * (n - L + 1)).astype(np.int64)
    ingest = uniform_int(seed, n_traces, 0, n + n // 8, stream=82)
    return start.astype(np.uint32), L.astype(np.uint32), ingest.astype(np.uint32)


def quality_windows(count: int = 1 << 16, n: int = 20, seed: int = 9):
    """Short windows for the comparison with the exact optimum: half random
    strings over alphabets of 2..4 tokens, half periodic (period U{2..6} over
    4 tokens) with 10% of positions redrawn.  Returns uint32[count * n]."""
    out = np.empty((count, n), dtype=np.uint32)
    kind = uniform_int(seed, count, 0, 1, stream=90)
    sigma = uniform_int(seed, count, 2, 4, stream=91)
    per = uniform_int(seed, count, 2, 6, stream=92)
    u = uniform01(seed, count * n, stream=93).reshape(count, n)
    body = uniform_int(seed, count * 6, 0, 3, stream=94).reshape(count, 6)
    noise = uniform01(seed, count * n, stream=95).reshape(count, n)
    redraw = uniform_int(seed, count * n, 0, 3, stream=96).reshape(count, n)
    j = np.arange(n)
    for w in range(count):
        if kind[w] == 0:
            out[w] = np.floor(u[w] * sigma[w]).astype(np.uint32)
        else:
            s = body[w, j % per[w]]
            out[w] = np.where(noise[w] < 0.1, redraw[w], s).astype(np.uint32)
    return out.reshape(-1)


def analysis_ready_ops(submit, slice_len, node: int, seed: int = 10, ops_per_token: float = 0.05,
                       jitter: int = 400):
    """Operation count at which node `node` has each asynchronous analysis
    back: submit op + slice_len * ops_per_token * (1 + node / 2) (nodes
    differ in speed) + a uniform jitter in [0, jitter).  int64 array."""
    submit = np.asarray(submit, dtype=np.int64)
    L = np.asarray(slice_len, dtype=np.float64)
    j = uniform_int(seed * 7 + node, len(submit), 0, max(0, jitter - 1), stream=100)
    return submit + np.ceil(L * ops_per_token * (1.0 + node / 2.0)).astype(np.int64) + j
