#!/usr/bin/env python3
"""Benchmark of the GPU trace finder: analysed tokens per second.

One step = the whole hot path over one window of synthetic task descriptors:
FNV-1a task hashing (Alg. 1 Hash) -> suffix array by prefix doubling -> LCP
-> Alg. 2 candidates, ordering, greedy non-overlapping selection (min trace
length 5) -> Aho-Corasick match of the traces found against the window's
token stream (Sec. 4.3).  The window is 2^20 tasks with nested loop periods
7 / 120 / 3000 and 1% of positions replaced by one of 2^16 random
descriptors (1-8 region arguments each).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]

Prints one JSON line.  `value` is device-timed throughput with the
descriptors resident in HBM (L2 flushed between steps); `e2e` is the same
step through the library's API with host (pinned) inputs copied in and the
step's result (selected intervals and traces; the match list stays on the
device for the replayer) copied back inside the timed region, each step's
input copy double-buffered against the previous step's work (`e2e.serial`:
the same without overlap); `roofline` reports the dominant kernel's
algorithmic bytes per launch over its event-timed launch duration against
the measured HBM copy bandwidth.  With N > 1 (torchrun) every rank analyses
its own window (weak scaling; windows are independent, no collective on
the data path).  `--impl reference` times the CPU oracle instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "analyzed tokens/s (SA+LCP+repeats) batched vs plain, % HBM roofline; p99 ms"
UNIT = "tokens/s"
MIN_LEN = 5
N_TASKS = 1 << 20
WORKLOAD = ("one window of 2^20 hashed task descriptors (nested periods 7/120/3000, 1% noise "
            "from 2^16 descriptors, 1-8 region args): hash -> SA -> LCP -> Alg. 2 repeats "
            "(min_len 5) -> Aho-Corasick match of the traces found against the window")

# Algorithmic bytes moved per unit of work, per kernel (unit = the element
# count the library records for each launch).  rs_pass: read and write one
# (u64 key, u32 value) pair; round (a doubling round over its list entries):
# the survey's 36 bytes per active suffix and round (read the entry, gather
# the rank h ahead, write the new rank, the key traffic of a sort); split
# (settling sorted pairs): read a pair, write a rank and a list entry; hash:
# descriptor bytes in, 8 out (per task, at the workload's mean of 4.5
# arguments).  The greedy loop and the automaton
# passes are chains of dependent accesses (latency-bound) and have no entry.
BYTES_PER_UNIT = {"rs_pass": 24, "rs_pass_keys": 16, "round": 36, "split": 24, "rs_hist": 12,
                  "hash_tasks": 16 + 4.5 * 13,
                  "plcp": 24, "rep.cand_gen": 36, "rep.compact": 16}
# (Launches sized for an upper bound -- the doubling rounds, their big-group
# sorts and splits -- have their recorded units corrected by the library to
# the exact counts once those are read, so every entry's units are exact.)


# The suffix-array + LCP path: prefix doubling (rank init, doubling rounds
# with their radix sorts and rank refreshes) and the Phi/PLCP LCP.
SA_LCP_KERNELS = ("init_keys", "key_or", "sa_dict", "wsb", "rs_hist", "rs_offsets", "rs_pass", "rs_pass_keys",
                  "round", "split", "list_compact", "minor", "phi", "plcp", "lcp_perm")


def sa_lcp_bytes(lcp, win_off, w: int) -> tuple[float, list]:
    """Algorithmic bytes of the SA+LCP path for one call (all windows):
    rank init n(w+28); per doubling round r >= 1, 36 bytes per active suffix,
    where A_r = #{i : max LCP of i with its SA neighbours >= 2^(r-1)} (a
    property of the input, not of the implementation); SA write 4n; LCP
    n(28+2w).  `lcp` is the pair-convention LCP (LCP[i] of SA[i], SA[i+1]),
    zero across window boundaries."""
    import torch
    n = int(lcp.numel())
    lc = lcp.to(torch.int64)
    if win_off is not None:
        # the pair straddling a window boundary has LCP 0 by definition
        ends = torch.as_tensor([int(x) - 1 for x in win_off[1:-1]], dtype=torch.int64, device=lc.device)
        lc[ends] = 0
    lc[n - 1] = 0
    left = torch.cat([torch.zeros(1, dtype=torch.int64, device=lc.device), lc[:-1]])
    mx = torch.maximum(left, lc)
    a_r = []
    h = 1
    while True:
        a = int((mx >= h).sum())
        if a == 0:
            break
        a_r.append(a)
        h <<= 1
    total = n * (w + 28) + 36 * sum(a_r) + 4 * n + n * (28 + 2 * w)
    return float(total), a_r


class _Range:
    """NVTX range around each timed step (lets a profiler select exactly the
    steady-state launches); a no-op where NVTX is unavailable."""

    def __enter__(self):
        try:
            import torch
            torch.cuda.nvtx.range_push("step")
            self.ok = True
        except Exception:
            self.ok = False
        return self

    def __exit__(self, *a):
        if self.ok:
            import torch
            torch.cuda.nvtx.range_pop()


def traffic_for(workload: str, kernel: str, launches_per_step: float):
    """DRAM bytes per launch of `kernel` from the committed ncu figures
    (profiles/traffic.txt: bytes per step of the kernel's launches), or None
    when there are none or the kernel's source changed since they were
    taken."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    if not os.path.exists(path):
        return None
    for line in open(path):
        f = line.split()
        if len(f) != 5 or line.startswith("#") or f[0] != workload or f[1] != kernel:
            continue
        h = hashlib.sha256()
        for rel in f[3].split(","):  # one or more source files, hashed in order
            src = os.path.join(ROOT, rel)
            if not os.path.exists(src):
                return None
            h.update(open(src, "rb").read())
        if h.hexdigest() != f[4]:
            return None
        return float(f[2]) / launches_per_step if launches_per_step else None
    return None


def tuning_summary(apo) -> list:
    """Radix-sort shapes chosen so far: [log2 size class, key bits, threads,
    pairs per thread, digit bits, trial ms of the chosen / default shape]."""
    return [[t["size_log2"], t["key_bits"], t["threads"], t["items"], t["digit_bits"],
             round(t["best_ms"], 4), round(t["default_ms"], 4)] for t in apo.sort_tuning_read()]


def sa_lcp_roofline(prof: dict, steps: int, b_alg: float, a_r: list, peak: float, peak_kind: str,
                    traffic_step=None) -> dict:
    """The SA+LCP path against the HBM roofline, over the summed event time
    of its kernels: `achieved`/`frac` from its algorithmic bytes per call
    (work efficiency), `dram_achieved`/`dram_frac` from the DRAM bytes ncu
    measured for the same launches (`traffic`, per step; null when the
    kernels' sources changed since)."""
    ms = sum(prof[k][1] for k in SA_LCP_KERNELS if k in prof) / steps
    launches = sum(prof[k][0] for k in SA_LCP_KERNELS if k in prof) / steps
    ach = b_alg / (ms / 1e3) / 1e9 if ms > 0 else None
    dram = traffic_step / (ms / 1e3) / 1e9 if (traffic_step and ms > 0) else None
    return {"bound": "hbm", "unit": "GB/s", "kernels": list(SA_LCP_KERNELS), "launches_per_step": launches,
            "ms_per_step": ms, "algorithmic_bytes": b_alg, "active_per_round": a_r, "achieved": ach,
            "peak": peak, "peak_kind": peak_kind, "frac": (ach / peak) if ach else None,
            "traffic": traffic_step, "dram_achieved": dram, "dram_frac": (dram / peak) if dram else None}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--n-tasks", type=int, default=N_TASKS)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default="window", choices=["window", "batched", "served", "match", "finder", "replay", "quality",
                                                     "config4"],
                    help="window: the full path on one 2^20-task window (default); batched: "
                         "SA+LCP+repeats over 512 uneven windows in one call vs one call per window")
    ap.add_argument("--windows", type=int, default=512)
    ap.add_argument("--duration", type=float, default=30.0, help="served: seconds of arrivals")
    ap.add_argument("--rate", type=float, default=2000.0, help="served: mean requests per second")
    ap.add_argument("--lanes", type=int, default=2, help="served: batches in flight")
    ap.add_argument("--no-forms", action="store_true",
                    help="window workload: skip the short batched and served measurements")
    ap.add_argument("--sort-tuning", type=int, default=0, choices=range(0, 8),
                    help="0: radix-sort shapes timed per size class on first use; 1: default shape "
                         "only; 2 + k: shape k only")
    return ap.parse_args()


def env_ranks():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class Clocks:
    """nvidia-smi samples (200 ms) while the timed region runs."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                       "-lms", "200", "-i", str(device)], stdout=self.f,
                                      stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self) -> dict:
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        rows = [r.strip().split(",") for r in self.f.read().splitlines() if r.strip()]
        os.unlink(self.f.name)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except (ValueError, IndexError):
                continue
            for k, nm in enumerate(names):
                if len(r) > 5 + k and r[5 + k].strip().lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def oracle_window_step(ts):
    """The oracle, as it stands, on one window: hash the descriptors, then
    SA, LCP and Alg. 2's repeats (the metric's stages).  Returns the seconds
    taken and the number of traces."""
    import oracle
    t0 = time.perf_counter()
    tok = oracle.hash_tasks(ts)
    r = oracle.find_repeats(tok, MIN_LEN)
    return time.perf_counter() - t0, int(r.trace_len.shape[0])


def cpu_baseline(n_tasks: int) -> dict:
    """The oracle, as it stands, single-threaded, on the bench's own window
    (same seed and size): one step of hashing, SA, LCP and repeats.  The
    GPU step also matches the traces against the window; the oracle's naive
    matching of the same traces takes over a minute per window, so it is
    left out of the sample (the GPU side does more work than this sample)."""
    import workloads as W
    ts = W.config2_tasks(n_tasks, seed=2)
    dt, nt = oracle_window_step(ts)
    return {"value": n_tasks / dt, "unit": UNIT, "cores": 1, "kind": "oracle", "same_config": True,
            "sample": f"one step (hash, SA, LCP, Alg. 2 repeats: {nt} traces) on the bench's own {n_tasks}-task "
                      f"window, {dt:.2f} s single-threaded; the GPU step's matching stage is not in the sample"}


def batched_cpu_baseline(toks, off) -> dict:
    """The oracle, as it stands, over the batched workload's windows: every
    host core through a thread pool over independent windows (the oracle is
    a C library called through ctypes, which releases the GIL), and one
    core on a prefix of the windows."""
    import os
    from concurrent.futures import ThreadPoolExecutor

    import oracle
    wins = [toks[int(off[w]):int(off[w + 1])] for w in range(len(off) - 1)]
    t0 = time.perf_counter()
    one, k = 0, 0
    while k < len(wins) and one < (1 << 21):
        oracle.find_repeats(wins[k], MIN_LEN)
        one += len(wins[k])
        k += 1
    dt1 = time.perf_counter() - t0
    cores = os.cpu_count() or 1
    t0 = time.perf_counter()
    with ThreadPoolExecutor(cores) as ex:
        list(ex.map(lambda x: oracle.find_repeats(x, MIN_LEN), wins))
    dt = time.perf_counter() - t0
    total = int(off[-1])
    return {"value": total / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"SA, LCP and Alg. 2 repeats of all {len(wins)} windows ({total} tokens), one window per "
                      f"task on a pool of {cores} threads: {dt:.2f} s",
            "one_core": {"value": one / dt1, "unit": UNIT, "cores": 1,
                         "sample": f"the first {k} windows ({one} tokens): {dt1:.2f} s"}}


def run_reference(args, rank, world):
    """The oracle on the bench's own window (2^20 tasks, same seed), one
    window per step: hashing, SA, LCP and Alg. 2's repeats, single-threaded
    (about 4-5 s per step).  The GPU step also matches the traces it found
    against the window; the oracle's naive matching of those traces alone
    takes over a minute, so the reference step leaves it out."""
    if rank != 0:
        return
    import workloads as W
    n = args.n_tasks
    ts = W.config2_tasks(n, seed=2)
    times = []
    for k in range(args.warmup + args.steps):
        dt, _ = oracle_window_step(ts)
        if k >= args.warmup:
            times.append(dt)
    tot = sum(times)
    value = n * len(times) / tot
    sample = (f"each step: hash, SA, LCP and Alg. 2 repeats of the bench's own {n}-task window "
              "(the GPU step also matches the traces; not in the oracle step), single-threaded oracle")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / len(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
        "data": "synthetic", "config": {"workload": WORKLOAD, "n_tokens": n, "min_len": MIN_LEN,
                                        "same_config": True,
                                        "stages": "hash, SA, LCP, repeats (the GPU step adds matching)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))


def run_batched(args, rank, world, local, emit=True, plain_steps=3):
    """512 windows of log-uniform length 1,024..262,144 (period U{3..5000},
    5% noise over 1,000 tokens): SA + LCP + Alg. 2 repeats for all of them in
    one batched call, against one call per window (plain)."""
    import numpy as np
    import torch

    import workloads as W
    from paper_2406_18111_gb300 import Apo
    dev = torch.device("cuda", local)
    apo = Apo(local)
    apo.sort_tuning(args.sort_tuning)
    toks, off, _ = W.config3_windows(args.windows, seed0=3 + 100000 * rank)
    t = torch.from_numpy(toks.view(np.int32)).to(dev)
    total = int(off[-1])
    stream = torch.cuda.current_stream()
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    for _ in range(args.warmup):
        r = apo.find_repeats_batched(t, off, MIN_LEN, stages=False)
    torch.cuda.synchronize()

    def timed(fn, steps):
        tot = 0.0
        for _ in range(steps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            with _Range():
                fn()
            b.record(stream)
            b.synchronize()
            tot += a.elapsed_time(b)
        return tot / steps

    clocks = Clocks(local)
    l0 = sum(v[0] for v in apo.profile_read().values())
    ms = timed(lambda: apo.find_repeats_batched(t, off, MIN_LEN, stages=False), args.steps)
    n_launch = sum(v[0] for v in apo.profile_read().values()) - l0
    apo.profile_reset()
    apo.profile(True)
    ms_prof = timed(lambda: apo.find_repeats_batched(t, off, MIN_LEN, stages=False), args.steps)
    prof = apo.profile_read()
    apo.profile(False)

    # the same call replayed as a CUDA graph (apo_graph_mode): the first
    # call records and captures, the timed ones replay
    ga = Apo(local)
    ga.sort_tuning(args.sort_tuning)
    ga.graph_mode(True)
    for _ in range(max(2, args.warmup)):
        ga.find_repeats_batched(t, off, MIN_LEN, stages=False, reuse=True)
    torch.cuda.synchronize()
    st0 = ga.graph_stats()
    ms_graph = timed(lambda: ga.find_repeats_batched(t, off, MIN_LEN, stages=False, reuse=True), args.steps)
    st1 = ga.graph_stats()
    graph = {"value": total * world / (ms_graph / 1e3), "unit": UNIT, "ms_per_step": ms_graph,
             "replays_in_timed_steps": st1["replays"] - st0["replays"], "captures": st1["captures"],
             "discarded": st1["discarded"],
             "form": "the whole batched call as one CUDA graph launch (recorded host reads, checked on the device)"}
    ga.close()

    def plain():
        for w in range(args.windows):
            a, b = int(off[w]), int(off[w + 1])
            apo.find_repeats(t[a:b], MIN_LEN, stages=False)
    plain_steps = max(1, min(plain_steps, args.steps))
    ms_plain = timed(plain, plain_steps)
    clk = clocks.stop()
    peak, peak_kind = peaks()

    def kernel_roof(name):
        la, kms, units = prof[name]
        bpu = BYTES_PER_UNIT.get(name)
        r = {"kernel": name, "bound": "hbm", "unit": "GB/s", "peak": peak, "peak_kind": peak_kind,
             "launches_per_step": la / args.steps, "share_of_step": kms / args.steps / ms_prof,
             "traffic": traffic_for("batched", name, la / args.steps) if la else None,
             "traffic_unit": "bytes per launch (ncu dram__bytes_read.sum + dram__bytes_write.sum)"}
        if bpu is not None and kms > 0:
            ach = bpu * units / (kms / 1e3) / 1e9
            r.update({"achieved": ach, "frac": ach / peak, "algorithmic_bytes_per_launch": bpu * units / la,
                      "ms_per_launch": kms / la})
        return r
    name = max((k for k in prof if k in BYTES_PER_UNIT), key=lambda k: prof[k][1])
    roof = kernel_roof(name)
    kernels = {k: {"launches_per_step": v[0] / args.steps, "ms_per_step": v[1] / args.steps}
               for k, v in sorted(prof.items(), key=lambda kv: -kv[1][1])}
    full = apo.find_repeats_batched(t, off, MIN_LEN, stages=True)
    b_alg, a_r = sa_lcp_bytes(full.lcp, off, 4)
    sa_lcp = sa_lcp_roofline(prof, args.steps, b_alg, a_r, peak, peak_kind, traffic_for("batched", "sa_lcp", 1.0))
    del full
    out = ({
            "metric": METRIC, "value": total * world / (ms / 1e3), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": f"batched: {args.windows} windows, log-uniform 1,024..262,144 tokens, "
                                   "periods U{3..5000}, 5% noise; SA+LCP+repeats (min_len 5)",
                       "n_tokens": total, "windows": args.windows, "min_len": MIN_LEN,
                       "l2": "flushed between steps"},
            "plain": {"value": total / (ms_plain / 1e3), "unit": UNIT, "ms_per_step": ms_plain,
                      "form": "one apo_find_repeats call per window, same stream", "steps": plain_steps},
            "batched_over_plain": ms_plain / ms, "graph": graph,
            "gpu_launches": n_launch, "roofline": roof, "sa_lcp_roofline": sa_lcp, "clocks": clk,
            "kernels": kernels, "sort_tuning": tuning_summary(apo)})
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = batched_cpu_baseline(toks, off)
    if emit and rank == 0:
        print(json.dumps(out))
    return out


def _served_latency(lat_ms, tokens, span, n_req, duration, rate):
    import numpy as np
    return {"rate_per_s": rate, "requests": n_req, "offered_tokens_per_s": tokens / duration,
            "value": tokens / span, "unit": UNIT, "p50_ms": float(np.percentile(lat_ms, 50)),
            "p99_ms": float(np.percentile(lat_ms, 99))}


def _serve_arrivals(srv, reqs, t_arr):
    """Submit reqs[k] at t_arr[k] seconds from now (a feeder thread), then
    wait for every result."""
    import threading
    ids = [None] * len(reqs)
    t0 = time.perf_counter()

    def feeder():
        for k, S in enumerate(reqs):
            delay = t_arr[k] - (time.perf_counter() - t0)
            if delay > 0:
                time.sleep(delay)
            ids[k] = srv.submit(S)
    th = threading.Thread(target=feeder)
    th.start()
    th.join()
    return [srv.wait(i) for i in ids]


def _served_run(srv, pool, t_arr, duration, rate):
    import numpy as np
    reqs = [pool[k % len(pool)] for k in range(len(t_arr))]
    res = _serve_arrivals(srv, reqs, t_arr)
    lat = np.array([r.t_done - r.t_submit for r in res]) * 1e3
    tokens = sum(r.n for r in res)
    span = max(r.t_done for r in res) - min(r.t_submit for r in res)
    out = _served_latency(lat, tokens, span, len(res), duration, rate)
    out["mean_batch_windows"] = float(np.mean([r.batch_windows for r in res]))
    return out


def _plain_run(apo, dev, pool, t_arr, duration, rate):
    """The same arrivals through one apo_find_repeats call per request, in
    arrival order, from one host thread: each request's tokens copied in from
    pinned memory, analysed, its selection and traces read back; latency from
    its arrival to its results on the host."""
    import numpy as np
    import torch
    stage = torch.empty(max(len(S) for S in pool), dtype=torch.int32).pin_memory()
    lat, tokens = [], 0
    t0 = time.perf_counter()
    for k, ta in enumerate(t_arr):
        delay = ta - (time.perf_counter() - t0)
        if delay > 0:
            time.sleep(delay)
        S = pool[k % len(pool)]
        n = len(S)
        stage[:n].numpy()[:] = S.view(np.int32)
        t = stage[:n].to(dev, non_blocking=True)
        r = apo.find_repeats(t, MIN_LEN, stages=False)
        for x in (r.sel_start, r.sel_len, r.sel_trace, r.trace_len, r.trace_start):
            x.cpu()
        lat.append((time.perf_counter() - t0 - ta) * 1e3)
        tokens += n
    span = time.perf_counter() - t0 - t_arr[0]
    return _served_latency(np.array(lat), tokens, span, len(t_arr), duration, rate)


def run_served(args, rank, world, local, emit=True, sweep=True):
    """Config 5's serving: Poisson analysis requests (mean `rate`/s for
    `duration` s, window lengths log-uniform 4,096..2^20 tokens, periodic
    content with 5% noise) submitted in real time to a continuous-batching
    server; p50/p99 latency from submission to results and tokens/s served.
    With sweep: the rate doubled until the server saturates (tokens/s served
    below 90% of those offered), and the same arrivals at the base rate
    through one plain apo_find_repeats call per request."""
    import numpy as np
    import torch

    import workloads as W
    from paper_2406_18111_gb300 import Apo, Server
    t_arr, L, P = W.served_requests(args.duration, args.rate, seed=5 + rank)
    pool_n = 256  # distinct windows, replayed by the arrivals
    pool = [W.served_window(k, int(L[k]), int(P[k])) for k in range(min(pool_n, len(L)))]
    srv = Server(local, min_len=MIN_LEN, token_bytes=4, max_batch_tokens=1 << 24, max_batch_windows=256,
                 lanes=args.lanes)
    # Warm-up, untimed: every pool window once, then one second of the same
    # arrival process, so that the lanes' first-use work (workspace growth,
    # the radix-sort shape trials of each batch size class) is done before
    # the measured arrivals.
    for i in [srv.submit(S) for S in pool]:
        srv.wait(i)
    t_w, _, _ = W.served_requests(1.0, args.rate, seed=1005 + rank)
    _serve_arrivals(srv, [pool[k % len(pool)] for k in range(len(t_w))], t_w)
    clocks = Clocks(local)
    main_run = _served_run(srv, pool, t_arr, args.duration, args.rate)
    sweep_runs, plain = [], None
    if sweep:
        step_s = 2.0
        t_w, _, _ = W.served_requests(0.5, args.rate * 8, seed=2005 + rank)  # the larger batches' first use
        _serve_arrivals(srv, [pool[k % len(pool)] for k in range(len(t_w))], t_w)
        for mult in (2, 4, 8):
            rate = args.rate * mult
            ts, _, _ = W.served_requests(step_s, rate, seed=3005 + 10 * mult + rank)
            r = _served_run(srv, pool, ts, step_s, rate)
            sweep_runs.append(r)
            if r["value"] < 0.9 * r["offered_tokens_per_s"]:
                break
    clk = clocks.stop()
    srv.close()
    if sweep:
        apo = Apo(local)
        dev = torch.device("cuda", local)
        for S in pool[:8]:  # first-use work of the plain form
            apo.find_repeats(torch.from_numpy(S.view(np.int32)).to(dev), MIN_LEN, stages=False)
        torch.cuda.synchronize(dev)
        step_s = 2.0
        ts = t_arr[t_arr < step_s]
        plain = _plain_run(apo, dev, pool, ts, step_s, args.rate)
        plain["form"] = ("one apo_find_repeats call per request in arrival order, one host thread: "
                         "copy in from pinned memory, analyse, read the selection back")
        apo.close()
    runs = [main_run] + sweep_runs
    best = max(runs, key=lambda r: r["value"])
    out = ({
            "metric": METRIC, "value": main_run["value"], "unit": UNIT, "n_gpus": world,
            "steps": main_run["requests"], "warmup": len(pool), "ms_per_step": None, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": f"served: Poisson {args.rate}/s for {args.duration} s, windows log-uniform "
                                   "4,096..2^20 tokens, periods U{3..5000}, 5% noise; SA+LCP+repeats "
                                   "(min_len 5), continuous batching",
                       "requests": main_run["requests"], "offered_tokens_per_s": main_run["offered_tokens_per_s"],
                       "lanes": args.lanes, "max_batch_tokens": 1 << 24, "distinct_windows": len(pool)},
            "p50_ms": main_run["p50_ms"], "p99_ms": main_run["p99_ms"],
            "mean_batch_windows": main_run["mean_batch_windows"], "clocks": clk})
    if sweep:
        out["sweep"] = sweep_runs
        out["saturated"] = {"value": best["value"], "unit": UNIT, "rate_per_s": best["rate_per_s"],
                            "p99_ms": best["p99_ms"]}
        out["plain"] = plain
        out["served_over_plain"] = best["value"] / plain["value"] if plain and plain["value"] else None
    if emit and rank == 0:
        print(json.dumps(out))
    return out


def run_finder(args, rank, world, local, emit=True):
    """Alg. 1's online TraceFinder with Sec. 4.4's ruler-function sampling
    (history buffer 5000 tokens, unit 250) over a stream of 2^20 hashed task
    descriptors pushed in chunks of 1000 as fast as the host issues them;
    every analysis is an asynchronous request of the served form."""
    import numpy as np
    import torch

    import workloads as W
    from paper_2406_18111_gb300 import Apo, Finder, Server
    dev = torch.device("cuda", local)
    apo = Apo(local)
    n = args.n_tasks
    ts = W.config2_tasks(n, seed=2 + rank)
    dts = [torch.from_numpy(np.ascontiguousarray(a).view(dt)).to(dev)
           for a, dt in ((ts.task_id, np.int32), (ts.arg_off, np.int32), (ts.region, np.int32),
                         (ts.field_mask, np.int64), (ts.priv, np.uint8))]
    tok = apo.hash_tasks(*dts).cpu().numpy().view(np.uint64)
    unit, buffer, chunk = 250, 5000, 1000
    srv = Server(local, min_len=MIN_LEN, token_bytes=8, max_batch_tokens=1 << 22, max_batch_windows=256,
                 lanes=args.lanes)
    warm = Finder(srv, buffer_tokens=buffer, unit=unit)  # first-use work (workspace, shape trials)
    warm.push(tok[:200000])
    warm.drain()
    warm.close()
    clocks = Clocks(local)
    f = Finder(srv, buffer_tokens=buffer, unit=unit)
    res = []
    t0 = time.perf_counter()
    for a in range(0, n, chunk):
        f.push(tok[a:a + chunk])
        while True:
            r = f.poll()
            if r is None:
                break
            res.append(r)
    t_push = time.perf_counter() - t0
    res += f.drain()
    wall = time.perf_counter() - t0
    clk = clocks.stop()
    st = f.stats()
    f.close()
    srv.close()
    lat = np.array([r.t_done - r.t_submit for r in res]) * 1e3
    import math
    out = {"metric": "online trace finder: stream tokens/s (ruler-sampled analyses, Sec. 4.4)",
           "value": n * world / wall, "unit": UNIT, "n_gpus": world, "steps": len(res), "warmup": 1,
           "ms_per_step": float(np.mean(lat)), "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "u64", "data": "synthetic",
           "config": {"workload": f"{n} hashed task descriptors (config-2 structure) pushed {chunk} at a time; "
                                  f"history buffer {buffer}, unit {unit}; analyses on the served form "
                                  f"({args.lanes} lanes)",
                      "analyses": st["analyses"], "analysed_tokens": st["analysed_tokens"],
                      "analysed_per_token": st["analysed_tokens"] / n,
                      "log2_buffer_over_unit": math.log2(buffer / unit)},
           "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
           "push_s": t_push, "wall_s": wall, "traces_found": int(sum(len(r.trace_len) for r in res)),
           "clocks": clk}
    if emit and rank == 0:
        print(json.dumps(out))
    return out


def run_replay(args, rank, world, local, emit=True, cpu_leg=True):
    """Alg. 1's TraceReplayer (Sec. 4.3) over a 2^20-task stream whose loop
    structure changes over time: the candidate traces are what the online
    finder (ruler sampling, buffer 5000, unit 250; this library's served
    form) reports over that stream, each ingested one analysis period after
    its analysis point.  Replay decisions for the whole stream per step."""
    import numpy as np
    import torch

    import workloads as W
    from paper_2406_18111_gb300 import Apo, Finder, Server
    dev = torch.device("cuda", local)
    apo = Apo(local)
    apo.sort_tuning(args.sort_tuning)
    n = args.n_tasks
    S = W.replay_stream(n, seed=6 + rank)
    unit, buffer = 250, 5000
    srv = Server(local, min_len=MIN_LEN, token_bytes=4, max_batch_tokens=1 << 22, max_batch_windows=256,
                 lanes=args.lanes)
    f = Finder(srv, buffer_tokens=buffer, unit=unit)
    st_l, ln_l, ig_l = [], [], []
    for a in range(0, n, 1 << 16):
        f.push(S[a:a + (1 << 16)])
    for r in f.drain():
        st_l.append(np.asarray(r.trace_start, dtype=np.uint64))
        ln_l.append(np.asarray(r.trace_len, dtype=np.uint32))
        ig_l.append(np.full(len(r.trace_len), (r.index + 1) * unit, dtype=np.uint64))
    f.close()
    srv.close()
    h_st = np.concatenate(st_l).astype(np.uint32)
    h_ln = np.concatenate(ln_l).astype(np.uint32)
    h_ig = np.minimum(np.concatenate(ig_l), 0xffffffff).astype(np.uint32)
    P = int(h_st.shape[0])
    params = dict(count_cap=8, half_life=1000, bonus=(17, 16), window=5000)
    d_S = torch.from_numpy(S.view(np.int32)).to(dev)
    d_st, d_ln, d_ig = (torch.from_numpy(x.view(np.int32)).to(dev) for x in (h_st, h_ln, h_ig))
    for _ in range(max(3, args.warmup)):
        rep = apo.replay(d_S, d_st, d_ln, d_ig, curve=True, **params)
    counts = rep[5]
    stream = torch.cuda.current_stream()
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    clocks = Clocks(local)
    steps = max(1, min(args.steps, 10))
    tot = 0.0
    for _ in range(steps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        with _Range():
            apo.replay(d_S, d_st, d_ln, d_ig, curve=True, **params)
        b.record(stream)
        b.synchronize()
        tot += a.elapsed_time(b)
    ms = tot / steps
    # per-kernel times from separate profiled steps (events around every launch)
    apo.profile_reset()
    apo.profile(True)
    for _ in range(steps):
        flush.zero_()
        apo.replay(d_S, d_st, d_ln, d_ig, curve=True, **params)
    torch.cuda.synchronize()
    prof = apo.profile_read()
    apo.profile(False)
    # end to end: host stream and traces in, replays out
    pin = [torch.from_numpy(x.view(np.int32)).pin_memory() for x in (S, h_st, h_ln, h_ig)]
    dst = [torch.empty_like(x, device=dev) for x in pin]
    tot_e2e, d2h = 0.0, 0
    for _ in range(steps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for d_, h_ in zip(dst, pin):
            d_.copy_(h_, non_blocking=True)
        e, l, t, _, _, _ = apo.replay(dst[0], dst[1], dst[2], dst[3], traced=False, **params)
        out = [x.cpu() for x in (e, l, t)]
        b.record(stream)
        b.synchronize()
        tot_e2e += a.elapsed_time(b)
        d2h = sum(x.numel() * 4 for x in out)
    clk = clocks.stop()
    ms_e2e = tot_e2e / steps
    kernels = {k: {"launches_per_step": v[0] / steps, "ms_per_step": v[1] / steps}
               for k, v in sorted(prof.items(), key=lambda kv: -kv[1][1])}
    ksum = sum(v["ms_per_step"] for v in kernels.values()) or 1.0
    top = next(iter(kernels.items())) if kernels else ("", {"ms_per_step": 0.0, "launches_per_step": 0})
    out = {"metric": "replayed stream tasks/s (TraceReplayer, Alg. 1 / Sec. 4.3, whole stream per step)",
           "value": n * world / (ms / 1e3), "unit": UNIT, "n_gpus": world, "steps": steps,
           "warmup": max(3, args.warmup), "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "u32", "data": "synthetic",
           "config": {"workload": f"{n}-task stream of changing loops (periods 20..600, 1% noise); "
                                  f"{P} traces from the online finder (buffer {buffer}, unit {unit}), "
                                  f"ingested one period after their analysis point",
                      "n_tasks": n, "traces": P, **{k: v for k, v in params.items()},
                      "l2": "flushed between steps"},
           "e2e": {"value": n * world / (ms_e2e / 1e3), "unit": UNIT,
                   "h2d_bytes_per_step": int(sum(x.numel() * 4 for x in pin)), "d2h_bytes_per_step": d2h},
           "replays": counts[0], "traced_fraction": counts[1] / n, "pieces": counts[2],
           "occurrences": counts[3], "appearances": counts[4], "undecided": counts[5],
           "selection_rounds": counts[6],
           "top_kernel": {"kernel": top[0], "share_of_kernel_time": top[1]["ms_per_step"] / ksum},
           "kernels": kernels, "clocks": clk}
    if cpu_leg and rank == 0:
        import oracle
        t0 = time.perf_counter()
        o = oracle.replay(S.astype(np.uint64), h_st, h_ln, h_ig, 0, params["count_cap"], params["half_life"],
                          params["bonus"])
        dt = time.perf_counter() - t0
        out["cpu_baseline"] = {"value": n / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
                               "sample": f"the whole step (the same stream and traces), {dt:.2f} s "
                                         f"single-threaded; {len(o.end)} replays"}
    if emit and rank == 0:
        print(json.dumps(out))
    return out


def run_quality(args, rank, world, local, emit=True):
    """Alg. 2 against the exact optimum of Sec. 3's problem (traces required
    to repeat) on 2^16 windows of 20 tokens, min length 2: the optimum by
    exhaustive search (apo_optimum_batched, timed: windows/s), Alg. 2 by the
    batched form on the same windows, and how far the heuristic falls short."""
    import numpy as np
    import torch

    import workloads as W
    from paper_2406_18111_gb300 import Apo
    dev = torch.device("cuda", local)
    apo = Apo(local)
    count, n, m = 1 << 16, 20, 2
    q = W.quality_windows(count, n, seed=9 + rank)
    off = np.arange(count + 1, dtype=np.uint64) * n
    dq = torch.from_numpy(q.view(np.int32)).to(dev)
    for _ in range(max(1, args.warmup)):
        best, ws_, wl, wc = apo.optimum_batched(dq, off, m)
    stream = torch.cuda.current_stream()
    clocks = Clocks(local)
    steps = max(1, min(args.steps, 5))
    tot = 0.0
    for _ in range(steps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        best, ws_, wl, wc = apo.optimum_batched(dq, off, m)
        b.record(stream)
        b.synchronize()
        tot += a.elapsed_time(b)
    clk = clocks.stop()
    ms = tot / steps
    opt = best.cpu().numpy().astype(np.int64)
    r = apo.find_repeats_batched(dq, off, m)
    sel_start = r.sel_start.cpu().numpy().view(np.uint32).astype(np.int64)
    sel_len = r.sel_len.cpu().numpy().view(np.uint32).astype(np.int64)
    sel_off = np.asarray(r.sel_off, dtype=np.int64)
    raw = np.zeros(count, np.int64)
    feas = np.zeros(count, np.int64)
    qq = q.reshape(count, n)
    for w in range(count):
        groups = {}
        for k in range(sel_off[w], sel_off[w + 1]):
            a, l = int(sel_start[k]), int(sel_len[k])
            groups.setdefault(qq[w, a:a + l].tobytes(), []).append(l)
            raw[w] += l
        feas[w] = sum(sum(v) for v in groups.values() if len(v) >= 2)
    gap = opt[:, 0] - feas
    out = {"metric": "exact Sec. 3 optimum: windows/s (exhaustive search, one thread per window)",
           "value": count * world / (ms / 1e3), "unit": "windows/s", "n_gpus": world, "steps": steps,
           "warmup": max(1, args.warmup), "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "u32", "data": "synthetic",
           "config": {"workload": f"{count} windows of {n} tokens (half random over 2..4 tokens, half periodic "
                                  f"with 10% noise), min length {m}", "windows": count, "n": n, "min_len": m},
           "study": {"optimum_coverage_mean": float(opt[:, 0].mean() / n),
                     "alg2_coverage_mean": float(raw.mean() / n),
                     "alg2_repeated_coverage_mean": float(feas.mean() / n),
                     "alg2_optimal_fraction": float((gap == 0).mean()),
                     "gap_mean_tokens": float(gap.mean()), "gap_max_tokens": int(gap.max()),
                     "gap_histogram": {str(g): int((gap == g).sum()) for g in range(0, int(gap.max()) + 1)
                                       if int((gap == g).sum())}},
           "clocks": clk}
    if rank == 0:
        import oracle
        k = 50
        t0 = time.perf_counter()
        for w in range(k):
            oracle.optimum(qq[w].astype(np.uint64), m)
        dt = time.perf_counter() - t0
        out["cpu_baseline"] = {"value": k / dt, "unit": "windows/s", "cores": 1, "kind": "oracle",
                               "sample": f"the first {k} windows, {dt:.2f} s single-threaded (plain enumeration)"}
    if emit and rank == 0:
        print(json.dumps(out))
    return out


def run_config4(args, rank, world, local, emit=True):
    """The adversarial pair at 2^24 tokens each: window A (a constant run, a
    period-2 run and a period-3 run in equal thirds: 23 doubling rounds) and
    window B (uniform random u32): SA, LCP and Alg. 2 repeats per window,
    device-resident tokens, L2 flushed between steps."""
    import numpy as np
    import torch

    import workloads as W
    from paper_2406_18111_gb300 import Apo
    dev = torch.device("cuda", local)
    apo = Apo(local)
    apo.sort_tuning(args.sort_tuning)
    a_np, b_np = W.config4_windows(1 << 24, seed=4 + rank)
    stream = torch.cuda.current_stream()
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    peak, peak_kind = peaks()
    out = {"config": {"workload": "config 4: two windows of 2^24 u32 tokens: A = constant / period-2 / "
                                  "period-3 thirds, B = uniform random; SA+LCP+repeats (min_len 5)",
                      "l2": "flushed between steps"}}
    steps = max(1, min(args.steps, 3))
    for name, S in (("A", a_np), ("B", b_np)):
        t = torch.from_numpy(S.view(np.int32)).to(dev)
        for _ in range(max(1, min(args.warmup, 2))):
            r = apo.find_repeats(t, MIN_LEN, stages=False)
        torch.cuda.synchronize()
        tot = 0.0
        for _ in range(steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            r = apo.find_repeats(t, MIN_LEN, stages=False)
            e1.record(stream)
            e1.synchronize()
            tot += e0.elapsed_time(e1)
        ms = tot / steps
        apo.profile_reset()
        apo.profile(True)
        for _ in range(steps):
            flush.zero_()
            apo.find_repeats(t, MIN_LEN, stages=False)
        torch.cuda.synchronize()
        prof = apo.profile_read()
        apo.profile(False)
        full = apo.find_repeats(t, MIN_LEN, stages=True)
        b_alg, a_r = sa_lcp_bytes(full.lcp, None, 4)
        rounds = full.rounds
        del full
        out[name] = {"value": S.shape[0] * world / (ms / 1e3), "unit": UNIT, "ms_per_step": ms,
                     "rounds": rounds, "selected": int(r.sel_start.shape[0]),
                     "sa_lcp_roofline": sa_lcp_roofline(prof, steps, b_alg, a_r, peak, peak_kind)}
        del t
    if emit and rank == 0:
        print(json.dumps(out))
    return out


def run_match(args, rank, world, local, emit=True):
    """Aho-Corasick matching (Sec. 4.3) of 10,000 candidate traces (lengths
    log-uniform 5..2000; half copied from the stream, half random) against a
    2^26-token stream of periodic segments: stream tokens per second, with
    the automaton built inside every timed call."""
    import numpy as np
    import torch

    import workloads as W
    from paper_2406_18111_gb300 import Apo
    dev = torch.device("cuda", local)
    apo = Apo(local)
    apo.sort_tuning(args.sort_tuning)
    stream_np = W.match_stream(1 << 26, seed=5 + rank)
    pt, off = W.match_patterns(stream_np, 10000, 5, 2000, seed=5 + rank)
    st = torch.from_numpy(stream_np.view(np.int32)).to(dev)
    ptd = torch.from_numpy(pt.view(np.int32)).to(dev)
    cap = [1 << 20]
    for _ in range(max(1, args.warmup)):
        e, i = apo.match_candidates(ptd, off, st, cap=cap[0])
        cap[0] = max(cap[0], int(e.shape[0] * 1.1) + 1)
    matches = int(e.shape[0])
    stream = torch.cuda.current_stream()
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    clocks = Clocks(local)
    tot = 0.0
    steps = max(1, min(args.steps, 10))
    for _ in range(steps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        apo.match_candidates(ptd, off, st, cap=cap[0])
        b.record(stream)
        b.synchronize()
        tot += a.elapsed_time(b)
    clk = clocks.stop()
    ms = tot / steps
    # per-kernel times from separate profiled steps (events around every launch)
    apo.profile_reset()
    apo.profile(True)
    for _ in range(steps):
        flush.zero_()
        apo.match_candidates(ptd, off, st, cap=cap[0])
    torch.cuda.synchronize()
    prof = apo.profile_read()
    apo.profile(False)
    n = int(stream_np.shape[0])
    kernels = {k: {"launches_per_step": v[0] / steps, "ms_per_step": v[1] / steps}
               for k, v in sorted(prof.items(), key=lambda kv: -kv[1][1])}
    out = {"metric": "matched stream tokens/s (Aho-Corasick, build included)", "value": n * world / (ms / 1e3),
           "unit": UNIT, "n_gpus": world, "steps": steps, "warmup": args.warmup, "ms_per_step": ms,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
           "data": "synthetic",
           "config": {"workload": "2^26-token stream of periodic segments; 10,000 patterns, lengths "
                                  "log-uniform 5..2000, half stream substrings, half random",
                      "n_tokens": n, "patterns": 10000, "pattern_tokens": int(off[-1]),
                      "matches": matches, "l2": "flushed between steps"},
           "clocks": clk, "kernels": kernels}
    if emit and rank == 0:
        print(json.dumps(out))
    return out


def main():
    args = parse()
    rank, world, local = env_ranks()
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.workload in ("batched", "served", "match", "finder", "replay", "quality", "config4"):
        import torch
        torch.cuda.set_device(local)
        if world > 1:
            import torch.distributed as dist
            dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        import __graft_entry__
        if rank == 0:
            __graft_entry__.build()
        if world > 1:
            torch.distributed.barrier()
        if args.workload == "served":
            return run_served(args, rank, world, local)
        if args.workload == "match":
            return run_match(args, rank, world, local)
        if args.workload == "finder":
            return run_finder(args, rank, world, local)
        if args.workload == "replay":
            return run_replay(args, rank, world, local)
        if args.workload == "quality":
            return run_quality(args, rank, world, local)
        if args.workload == "config4":
            return run_config4(args, rank, world, local)
        return run_batched(args, rank, world, local)
    import numpy as np
    import torch
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import __graft_entry__
    if rank == 0:
        __graft_entry__.build()
    if world > 1:
        torch.distributed.barrier()
    import workloads as W
    from paper_2406_18111_gb300 import Apo
    dev = torch.device("cuda", local)
    apo = Apo(local)
    apo.sort_tuning(args.sort_tuning)
    n = args.n_tasks
    ts = W.config2_tasks(n, seed=2 + rank)
    host = [torch.from_numpy(np.ascontiguousarray(a).view(dt)).pin_memory()
            for a, dt in ((ts.task_id, np.int32), (ts.arg_off, np.int32), (ts.region, np.int32),
                          (ts.field_mask, np.int64), (ts.priv, np.uint8))]
    dts = [h.to(dev) for h in host]
    h2d_bytes = sum(h.numel() * h.element_size() for h in host)
    tok = torch.empty(n, dtype=torch.int64, device=dev)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)  # > 129 MB L2
    stream = torch.cuda.current_stream()
    cap = [8 * n]

    def step(inputs):
        apo.hash_tasks(*inputs, out=tok)
        r = apo.find_repeats(tok, MIN_LEN, stages=False, sa_lcp=True)
        e, i = apo.match_candidates(tok, None, tok, cap=cap[0], pat_start=r.trace_start,
                                    pat_len=r.trace_len, src_sa=r.sa, src_lcp=r.lcp)
        return r, e, i

    r = None
    for _ in range(args.warmup):
        r, e, i = step(dts)
        cap[0] = max(cap[0], int(e.shape[0] * 1.25) + 1)
    torch.cuda.synchronize()
    stats = {"candidates": None, "selected": int(r.sel_start.shape[0]), "traces": int(r.trace_len.shape[0]),
             "matches": int(e.shape[0]), "rounds": r.rounds}

    def launches():
        return sum(v[0] for v in apo.profile_read().values())

    def timed(inputs_fn, out_fn=None):
        total = 0.0
        for _ in range(args.steps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            with _Range():
                res = step(inputs_fn())
                if out_fn is not None:
                    out_fn(res)
            b.record(stream)
            b.synchronize()
            total += a.elapsed_time(b)
        return total / args.steps

    # 1. device-resident inputs
    clocks = Clocks(local)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    l0 = launches()
    t_wall = time.perf_counter()
    ms = timed(lambda: dts)
    torch.cuda.synchronize()
    t_wall = time.perf_counter() - t_wall
    n_launch = launches() - l0
    if world > 1:
        torch.distributed.barrier()
    # 2. the same steps with per-kernel event timing (roofline)
    apo.profile_reset()
    apo.profile(True)
    ms_prof = timed(lambda: dts)
    prof = apo.profile_read()
    apo.profile(False)
    # 3. end to end: pinned host inputs in, results back to the host
    d2h = [0]
    pinned_out = {}

    def to_host(res):
        # the step's result: the selected intervals and the traces R (the
        # match list stays on the device for the replayer; its count reaches
        # the host inside the call)
        r_, e_, i_ = res
        nb = 0
        for name, t in (("ss", r_.sel_start), ("sl", r_.sel_len), ("st", r_.sel_trace),
                        ("tl", r_.trace_len), ("ts", r_.trace_start)):
            buf = pinned_out.get(name)
            if buf is None or buf.numel() < t.numel():
                buf = torch.empty(max(1, int(t.numel() * 1.25)), dtype=t.dtype, pin_memory=True)
                pinned_out[name] = buf
            buf[:t.numel()].copy_(t, non_blocking=True)
            nb += t.numel() * t.element_size()
        d2h[0] = nb

    def h2d():
        for d_, h_ in zip(dts, host):
            d_.copy_(h_, non_blocking=True)
        return dts

    ms_e2e_serial = timed(h2d, to_host)

    # 4. end to end with the input copies double-buffered: step k+1's
    # descriptors are copied on a second stream while step k runs (every
    # step still copies its own inputs in and its result out, all inside one
    # timed region, L2 flush included)
    def e2e_pipelined(steps):
        xs, cs = torch.cuda.Stream(device=dev), torch.cuda.Stream(device=dev)
        bufs = [dts, [torch.empty_like(x) for x in dts]]
        copied = [torch.cuda.Event(), torch.cuda.Event()]
        freed = [torch.cuda.Event(), torch.cuda.Event()]
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()

        def copy_in(k):
            b = k % 2
            with torch.cuda.stream(cs):
                if k >= 2:
                    cs.wait_event(freed[b])
                for d_, h_ in zip(bufs[b], host):
                    d_.copy_(h_, non_blocking=True)
                copied[b].record(cs)

        t0.record(cs)
        copy_in(0)
        for k in range(steps):
            if k + 1 < steps:
                copy_in(k + 1)
            b = k % 2
            with torch.cuda.stream(xs):
                xs.wait_event(copied[b])
                flush.zero_()
                with _Range():
                    res = step(bufs[b])
                freed[b].record(xs)
                to_host(res)
        t1.record(xs)
        t1.synchronize()
        return t0.elapsed_time(t1) / steps

    ms_e2e = e2e_pipelined(args.steps)
    # 4. the same step with the repeat finding in graph mode (a repeated
    # window shape on the same buffers: one CUDA graph launch per call, the
    # recorded host reads checked on the device); hashing and matching eager
    ga = Apo(local)
    ga.graph_mode(True)

    def gstep(inputs):
        ga.hash_tasks(*inputs, out=tok)
        r = ga.find_repeats(tok, MIN_LEN, stages=False, sa_lcp=True, reuse=True)
        return ga.match_candidates(tok, None, tok, cap=cap[0], pat_start=r.trace_start,
                                   pat_len=r.trace_len, src_sa=r.sa, src_lcp=r.lcp)
    for _ in range(max(3, args.warmup)):
        gstep(dts)
    torch.cuda.synchronize()
    g0 = ga.graph_stats()
    gt = 0.0
    for _ in range(args.steps):
        flush.zero_()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        gstep(dts)
        ev1.record(stream)
        ev1.synchronize()
        gt += ev0.elapsed_time(ev1)
    ms_graph = gt / args.steps
    g1 = ga.graph_stats()
    ga.close()
    clk = clocks.stop()

    mst = torch.tensor([ms, ms_e2e, ms_e2e_serial, ms_graph], dtype=torch.float64, device=dev)
    if world > 1:
        torch.distributed.all_reduce(mst, op=torch.distributed.ReduceOp.MAX)
    ms, ms_e2e, ms_e2e_serial, ms_graph = float(mst[0]), float(mst[1]), float(mst[2]), float(mst[3])
    value = n * world / (ms / 1e3)
    e2e_value = n * world / (ms_e2e / 1e3)

    # roofline of the dominant kernel with a byte model (the kernels without
    # one are latency-bound chains: the greedy loop, automaton passes)
    peak, peak_kind = peaks()
    top = max(prof.items(), key=lambda kv: kv[1][1])
    dom = max(((k, v) for k, v in prof.items() if k in BYTES_PER_UNIT), key=lambda kv: kv[1][1])
    name, (la, kms, units) = dom
    bpu = BYTES_PER_UNIT.get(name)
    roof = {"kernel": name, "bound": "hbm", "unit": "GB/s", "peak": peak, "peak_kind": peak_kind,
            "launches_per_step": la / args.steps, "share_of_step": kms / args.steps / ms_prof,
            "traffic": traffic_for("window", name, la / args.steps) if la else None,
            "traffic_unit": "bytes per launch (ncu dram__bytes_read.sum + dram__bytes_write.sum)"}
    if bpu is not None and kms > 0:
        ach = bpu * units / (kms / 1e3) / 1e9
        roof.update({"achieved": ach, "frac": ach / peak, "algorithmic_bytes_per_launch": bpu * units / la,
                     "ms_per_launch": kms / la})
    else:
        roof.update({"achieved": None, "frac": None})
    roof["top_kernel"] = {"kernel": top[0], "share_of_step": top[1][1] / args.steps / ms_prof,
                          "bound": "hbm" if top[0] in BYTES_PER_UNIT else "latency"}
    kernels = {k: {"launches_per_step": v[0] / args.steps, "ms_per_step": v[1] / args.steps}
               for k, v in sorted(prof.items(), key=lambda kv: -kv[1][1])}

    full = apo.find_repeats(tok, MIN_LEN, stages=True)
    b_alg, a_r = sa_lcp_bytes(full.lcp, None, 8)
    sa_lcp = sa_lcp_roofline(prof, args.steps, b_alg, a_r, peak, peak_kind, traffic_for("window", "sa_lcp", 1.0))
    del full

    if rank != 0:
        return
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(n)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n_tokens": n, "min_len": MIN_LEN,
                   "l2": "flushed between steps (512 MiB write, outside the step events)",
                   "parallelism": f"replicas x{world}"},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d_bytes,
                "d2h_bytes_per_step": d2h[0], "ms_per_step": ms_e2e,
                "copies": "step k+1's inputs copied on a second stream while step k runs (two input buffers)",
                "serial": {"value": n * world / (ms_e2e_serial / 1e3), "ms_per_step": ms_e2e_serial,
                           "copies": "each step's copy in, step, copy out, one after another"}},
        "gpu_launches": n_launch,
        "roofline": roof,
        "sa_lcp_roofline": sa_lcp,
        "cpu_baseline": cpu,
        "clocks": clk,
        "wall_s_timed": t_wall,
        "ms_per_step_profiled": ms_prof,
        "graph": {"value": n * world / (ms_graph / 1e3), "unit": UNIT, "ms_per_step": ms_graph,
                  "replays_in_timed_steps": g1["replays"] - g0["replays"],
                  "discarded": g1["discarded"] - g0["discarded"],
                  "form": "the same step with apo_find_repeats in graph mode (one CUDA graph launch per "
                          "call, recorded host reads checked on the device); hashing and matching eager"},
        "step_stats": stats,
        "kernels": kernels,
        "sort_tuning": tuning_summary(apo),
    }
    if world == 1 and not args.no_forms:
        # The batched and served forms, measured briefly on their own
        # workloads; their own modes (--workload) give the full runs.
        import copy
        a2 = copy.copy(args)
        a2.steps, a2.warmup = min(args.steps, 5), 2
        bt = run_batched(a2, rank, world, local, emit=False, plain_steps=1)
        line["batched"] = {k: bt[k] for k in ("value", "unit", "ms_per_step", "config", "plain",
                                               "batched_over_plain", "graph", "roofline", "sa_lcp_roofline")}
        a3 = copy.copy(args)
        a3.duration = 30.0  # config 5's arrival process
        sv = run_served(a3, rank, world, local, emit=False)
        line["served"] = {k: sv[k] for k in ("value", "unit", "p50_ms", "p99_ms", "config", "mean_batch_windows",
                                              "sweep", "saturated", "plain", "served_over_plain")}
        fd = run_finder(args, rank, world, local, emit=False)
        line["finder"] = {k: fd[k] for k in ("metric", "value", "unit", "p50_ms", "p99_ms", "config")}
        line["batched"]["cpu_baseline"] = bt.get("cpu_baseline")
        c4 = run_config4(a2, rank, world, local, emit=False)
        line["config4"] = c4
        mt = run_match(a2, rank, world, local, emit=False)
        line["match"] = {k: mt[k] for k in ("metric", "value", "unit", "ms_per_step", "config")}
        rp = run_replay(a2, rank, world, local, emit=False, cpu_leg=False)
        line["replay"] = {k: rp[k] for k in ("metric", "value", "unit", "ms_per_step", "e2e", "replays",
                                              "traced_fraction", "top_kernel", "config")}
    print(json.dumps(line))


if __name__ == "__main__":
    main()
