"""GPU trace finder: Python binding of libapo (argument marshalling only).

Every step of the analysis runs in the CUDA kernels of ``libapo.so`` behind
the C ABI declared in ``include/apo.h``; this module only moves torch
tensors' device pointers and sizes across it.  There is no CPU fallback: if
the library is missing, or no GPU is present, calls raise.

    from paper_2406_18111_gb300 import Apo
    apo = Apo(device=0)
    tokens = apo.hash_tasks(task_id, arg_off, region, field_mask, priv)   # Alg. 1 Hash
    res = apo.find_repeats(tokens, min_len=5)                              # Alg. 2
    end, pid = apo.match_candidates(pat_tokens, pat_off, stream_tokens)    # Sec. 4.3
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libapo.so")

APO_OK, APO_EINVAL, APO_ENOMEM, APO_ECAPACITY, APO_ECUDA, APO_ETIMEOUT, APO_EDEVICE = 0, -1, -2, -3, -4, -5, -6
APO_EAGAIN = -7
_NAMES = {0: "APO_OK", -1: "APO_EINVAL", -2: "APO_ENOMEM", -3: "APO_ECAPACITY", -4: "APO_ECUDA",
          -5: "APO_ETIMEOUT", -6: "APO_EDEVICE", -7: "APO_EAGAIN"}

# Every symbol include/apo.h declares.
EXPORTS = ("apo_create", "apo_destroy", "apo_last_error", "apo_version", "apo_hash_tasks",
           "apo_find_repeats", "apo_find_repeats_batched", "apo_match_candidates",
           "apo_profile_enable", "apo_profile_reset",
           "apo_profile_read", "apo_greedy_select_noalloc", "apo_server_create", "apo_server_submit",
           "apo_server_poll", "apo_server_wait", "apo_server_release", "apo_server_now",
           "apo_server_destroy", "apo_sort_tuning", "apo_sort_tuning_read", "apo_finder_create",
           "apo_finder_push", "apo_finder_poll", "apo_finder_stats", "apo_finder_destroy",
           "apo_replay", "apo_optimum_batched", "apo_graph_mode", "apo_graph_stats",
           "apo_find_repeats_workspace", "apo_set_workspace", "apo_server_memory")

# Largest window apo_greedy_select_noalloc accepts (positions of its fixed bitmap).
NOALLOC_MAX_WINDOW = 1 << 22

_P = ctypes.c_void_p
_U64 = ctypes.c_uint64
_U32 = ctypes.c_uint32


class ApoError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_NAMES.get(code, code)}: {msg}")
        self.code = code


class apo_tasks(ctypes.Structure):
    _fields_ = [("n_tasks", _U64), ("task_id", _P), ("arg_off", _P), ("region", _P),
                ("field_mask", _P), ("priv", _P)]


class apo_window(ctypes.Structure):
    _fields_ = [("n", _U64), ("tokens", _P), ("token_bytes", ctypes.c_int)]


class apo_repeats_params(ctypes.Structure):
    _fields_ = [("min_len", _U32), ("flags", _U32)]


class apo_repeats_out(ctypes.Structure):
    _fields_ = [("sa", _P), ("lcp", _P), ("cand_len", _P), ("cand_id", _P), ("cand_start", _P),
                ("cand_accepted", _P), ("cand_cap", _U64), ("sel_start", _P), ("sel_len", _P),
                ("sel_trace", _P), ("sel_cap", _U64), ("trace_len", _P), ("trace_start", _P),
                ("trace_cap", _U64), ("counts", _P), ("cand_off", _P), ("sel_off", _P),
                ("trace_off", _P)]


class apo_server_config(ctypes.Structure):
    _fields_ = [("min_len", _U32), ("token_bytes", ctypes.c_int), ("max_batch_tokens", _U64),
                ("max_batch_windows", _U32), ("lanes", _U32), ("hbm_budget", _U64)]


class apo_request_result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("n", _U64), ("n_selected", _U64), ("n_traces", _U64),
                ("sel_start", _P), ("sel_len", _P), ("sel_trace", _P), ("trace_len", _P),
                ("trace_start", _P), ("t_submit", ctypes.c_double), ("t_start", ctypes.c_double),
                ("t_done", ctypes.c_double), ("batch_windows", _U64)]


class apo_windows(ctypes.Structure):
    _fields_ = [("n_windows", _U64), ("tokens", _P), ("token_bytes", ctypes.c_int), ("win_off", _P)]


class apo_patterns(ctypes.Structure):
    _fields_ = [("n_patterns", _U64), ("tokens", _P), ("token_bytes", ctypes.c_int),
                ("pat_off", _P), ("pat_start", _P), ("pat_len", _P), ("src_sa", _P), ("src_lcp", _P),
                ("src_n", _U64)]


_lib = None


class apo_replay_traces(ctypes.Structure):
    _fields_ = [("n_traces", _U64), ("start", _P), ("len", _P), ("ingest", _P)]


class apo_replay_params(ctypes.Structure):
    _fields_ = [("max_trace_len", _U32), ("count_cap", _U32), ("half_life", _U32), ("bonus_num", _U32),
                ("bonus_den", _U32), ("window", _U32)]


class apo_replay_out(ctypes.Structure):
    _fields_ = [("rep_end", _P), ("rep_len", _P), ("rep_trace", _P), ("rep_cap", _U64), ("traced", _P),
                ("curve", _P), ("counts", _P)]


def lib():
    """Load libapo.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "`python -m paper_2406_18111_gb300.build` (needs nvcc)")
        L = ctypes.CDLL(LIB_PATH)
        L.apo_create.argtypes = [ctypes.POINTER(_P), ctypes.c_int]
        L.apo_destroy.argtypes = [_P]
        L.apo_last_error.restype = ctypes.c_char_p
        L.apo_last_error.argtypes = []
        L.apo_version.argtypes = []
        L.apo_hash_tasks.argtypes = [_P, ctypes.POINTER(apo_tasks), _P, _P]
        L.apo_find_repeats.argtypes = [_P, ctypes.POINTER(apo_window),
                                       ctypes.POINTER(apo_repeats_params),
                                       ctypes.POINTER(apo_repeats_out), _P]
        L.apo_find_repeats_batched.argtypes = [_P, ctypes.POINTER(apo_windows),
                                               ctypes.POINTER(apo_repeats_params),
                                               ctypes.POINTER(apo_repeats_out), _P]
        L.apo_match_candidates.argtypes = [_P, ctypes.POINTER(apo_patterns), _P, _U64, _P, _P, _U64,
                                           ctypes.POINTER(_U64), _P]
        L.apo_profile_enable.argtypes = [_P, ctypes.c_int]
        L.apo_profile_reset.argtypes = [_P]
        L.apo_profile_read.argtypes = [_P, ctypes.c_int, ctypes.c_char_p, ctypes.c_size_t,
                                       ctypes.POINTER(_U64), ctypes.POINTER(ctypes.c_double),
                                       ctypes.POINTER(_U64)]
        L.apo_greedy_select_noalloc.argtypes = [_P, _P, _U64, _U64, _P, _P, _P]
        L.apo_find_repeats_workspace.argtypes = [_P, ctypes.POINTER(apo_windows), ctypes.POINTER(_U64)]
        L.apo_set_workspace.argtypes = [_P, _P, _U64]
        L.apo_server_create.argtypes = [ctypes.POINTER(_P), ctypes.c_int, ctypes.POINTER(apo_server_config)]
        L.apo_server_submit.argtypes = [_P, _P, _U64, ctypes.POINTER(_U64)]
        L.apo_server_poll.argtypes = [_P, _U64, ctypes.POINTER(apo_request_result)]
        L.apo_server_wait.argtypes = [_P, _U64, ctypes.POINTER(apo_request_result)]
        L.apo_server_release.argtypes = [_P, _U64]
        L.apo_server_now.argtypes = [_P]
        L.apo_server_memory.argtypes = [_P, ctypes.POINTER(_U64), ctypes.POINTER(_U64), ctypes.POINTER(_U64)]
        L.apo_server_destroy.argtypes = [_P]
        L.apo_sort_tuning.argtypes = [_P, ctypes.c_int]
        _I = ctypes.POINTER(ctypes.c_int)
        _D = ctypes.POINTER(ctypes.c_double)
        _U = ctypes.POINTER(_U32)
        L.apo_sort_tuning_read.argtypes = [_P, ctypes.c_int, _U, _U, _U, _I, _I, _I, _D, _D]
        L.apo_finder_create.argtypes = [ctypes.POINTER(_P), _P, ctypes.POINTER(apo_finder_config)]
        L.apo_finder_push.argtypes = [_P, _P, _U64, ctypes.POINTER(_U64)]
        L.apo_finder_poll.argtypes = [_P, ctypes.c_int, ctypes.POINTER(apo_finder_result)]
        L.apo_finder_stats.argtypes = [_P, ctypes.POINTER(_U64), ctypes.POINTER(_U64), ctypes.POINTER(_U64)]
        L.apo_finder_destroy.argtypes = [_P]
        L.apo_graph_mode.argtypes = [_P, ctypes.c_int]
        L.apo_graph_stats.argtypes = [_P, ctypes.POINTER(_U64), ctypes.POINTER(_U64), ctypes.POINTER(_U64)]
        L.apo_optimum_batched.argtypes = [_P, ctypes.POINTER(apo_windows), _U32, _P, _P, _P, _P, _P]
        L.apo_replay.argtypes = [_P, _P, _U64, ctypes.c_int, ctypes.POINTER(apo_replay_traces),
                                 ctypes.POINTER(apo_replay_params), ctypes.POINTER(apo_replay_out), _P]
        for f in EXPORTS:
            if f not in ("apo_last_error", "apo_server_now"):
                getattr(L, f).restype = ctypes.c_int
        L.apo_server_now.restype = ctypes.c_double
        _lib = L
    return _lib


def _check(code: int):
    if code != APO_OK:
        raise ApoError(code, lib().apo_last_error().decode(errors="replace"))


def _ptr(t) -> int:
    return 0 if t is None else int(t.data_ptr())


def _stream_handle(stream) -> int:
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


def _token_bytes(t) -> int:
    import torch
    if t.dtype in (torch.int32, getattr(torch, "uint32", torch.int32)):
        return 4
    if t.dtype in (torch.int64, getattr(torch, "uint64", torch.int64)):
        return 8
    raise TypeError(f"tokens must be 32- or 64-bit integers, got {t.dtype}")


@dataclass
class Repeats:
    """Outputs of Alg. 2 on one window (device tensors, unsigned values held
    in int32 bit patterns)."""
    sa: object
    lcp: object
    cand_len: object
    cand_id: object
    cand_start: object
    cand_accepted: object
    sel_start: object
    sel_len: object
    sel_trace: object
    trace_len: object
    trace_start: object
    rounds: int


@dataclass
class BatchRepeats:
    """Outputs of a batched call, concatenated window by window (starts are
    window-relative, sel_trace indexes the window's traces); the *_off host
    arrays give each window's range."""
    sa: object
    lcp: object
    cand_len: object
    cand_id: object
    cand_start: object
    cand_accepted: object
    sel_start: object
    sel_len: object
    sel_trace: object
    trace_len: object
    trace_start: object
    rounds: int
    win_off: np.ndarray
    cand_off: np.ndarray
    sel_off: np.ndarray
    trace_off: np.ndarray


class Apo:
    """A library context bound to one CUDA device."""

    def __init__(self, device: int = 0):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("libapo needs a CUDA GPU; none is available")
        self.device = device
        h = _P()
        _check(lib().apo_create(ctypes.byref(h), device))
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            lib().apo_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -------------------------------------------------------------- workspace
    def find_repeats_workspace(self, win_off) -> int:
        """Device bytes a repeat call over these windows needs (win_off on
        the host; [0, n] for one window of n tokens)."""
        wo = np.ascontiguousarray(np.asarray(win_off, dtype=np.uint64))
        ws = apo_windows(wo.shape[0] - 1, None, 4, wo.ctypes.data)
        out = _U64()
        _check(lib().apo_find_repeats_workspace(self._h, ctypes.byref(ws), ctypes.byref(out)))
        return int(out.value)

    def set_workspace(self, buf=None):
        """Take the repeat calls' scratch from a caller-owned device buffer
        (a uint8 tensor, kept alive by the caller), or from the context's own
        scratch again (None)."""
        if buf is None:
            _check(lib().apo_set_workspace(self._h, None, 0))
        else:
            _check(lib().apo_set_workspace(self._h, _ptr(buf), int(buf.numel() * buf.element_size())))

    # -------------------------------------------------------------- Alg. 1 Hash
    def hash_tasks(self, task_id, arg_off, region, field_mask, priv, out=None, stream=None):
        """Tokens (int64 tensor holding u64 bit patterns) of N task descriptors."""
        import torch
        n = int(task_id.shape[0])
        if out is None:
            out = torch.empty(n, dtype=torch.int64, device=task_id.device)
        t = apo_tasks(n, _ptr(task_id), _ptr(arg_off), _ptr(region), _ptr(field_mask), _ptr(priv))
        _check(lib().apo_hash_tasks(self._h, ctypes.byref(t), _ptr(out), _stream_handle(stream)))
        return out

    # -------------------------------------------------------------- Alg. 2
    def find_repeats(self, tokens, min_len: int, stages: bool = True, stream=None,
                     sa_lcp: bool = False, reuse: bool = False) -> Repeats:
        """Alg. 2 on one window of device tokens (int32 = u32, int64 = u64).
        stages: also return SA, LCP and the candidates; sa_lcp: SA and LCP
        only (what match_candidates can reuse).  With reuse, the output
        buffers are kept for the next call of the same sizes (the returned
        tensors are then overwritten by it), so that repeated calls hand the
        library the same arguments (graph mode)."""
        import torch
        n = int(tokens.shape[0])
        dev = tokens.device
        u32 = torch.int32
        M = max(1, 2 * (n - 1))
        K = max(1, n // max(1, min_len))
        bkey = ("one", n, int(min_len), bool(stages), bool(sa_lcp), str(dev))
        bufs = getattr(self, "_bufs", {}).get(bkey) if reuse else None
        if bufs is None:
            bufs = (torch.empty(max(1, n), dtype=u32, device=dev) if stages or sa_lcp else None,
                    torch.empty(max(1, n), dtype=u32, device=dev) if stages or sa_lcp else None,
                    torch.empty(M, dtype=u32, device=dev) if stages else None,
                    torch.empty(M, dtype=u32, device=dev) if stages else None,
                    torch.empty(M, dtype=u32, device=dev) if stages else None,
                    torch.empty(M, dtype=torch.uint8, device=dev) if stages else None,
                    *(torch.empty(K, dtype=u32, device=dev) for _ in range(5)))
            if reuse:
                if not hasattr(self, "_bufs"):
                    self._bufs = {}
                self._bufs[bkey] = bufs
        sa, lcp, cl, ci, cs, ca, ss, sl, st, tl, ts = bufs
        counts = (ctypes.c_uint64 * 4)()
        o = apo_repeats_out(_ptr(sa), _ptr(lcp), _ptr(cl), _ptr(ci), _ptr(cs), _ptr(ca),
                            M if stages else 0, _ptr(ss), _ptr(sl), _ptr(st), K, _ptr(tl), _ptr(ts), K,
                            ctypes.cast(counts, _P), None, None, None)
        w = apo_window(n, _ptr(tokens), _token_bytes(tokens))
        p = apo_repeats_params(int(min_len), 0)
        _check(lib().apo_find_repeats(self._h, ctypes.byref(w), ctypes.byref(p), ctypes.byref(o),
                                      _stream_handle(stream)))
        m, k, t, rounds = (int(x) for x in counts)

        def cut(x, c):
            return None if x is None else x[:c]
        return Repeats(cut(sa, n), cut(lcp, n), cut(cl, m), cut(ci, m), cut(cs, m), cut(ca, m),
                       ss[:k], sl[:k], st[:k], tl[:t], ts[:t], rounds)

    def find_repeats_batched(self, tokens, win_off, min_len: int, stages: bool = True,
                             stream=None, reuse: bool = False) -> "BatchRepeats":
        """Alg. 2 on many windows at once: tokens holds the windows back to
        back, window w = tokens[win_off[w]:win_off[w+1]] (win_off on the host).
        With reuse, the output buffers are kept for the next call of the same
        sizes (the returned tensors are then overwritten by it), so that
        repeated calls hand the library the same arguments (graph mode)."""
        import torch
        wo = np.ascontiguousarray(np.asarray(win_off, dtype=np.uint64))
        W = wo.shape[0] - 1
        n = int(tokens.shape[0])
        dev = tokens.device
        u32 = torch.int32
        M = max(1, 2 * n)
        K = max(1, n // max(1, min_len))
        bkey = (n, W, int(min_len), bool(stages), str(dev))
        bufs = getattr(self, "_bufs", {}).get(bkey) if reuse else None
        if bufs is None:
            bufs = (torch.empty(max(1, n), dtype=u32, device=dev) if stages else None,
                    torch.empty(max(1, n), dtype=u32, device=dev) if stages else None,
                    torch.empty(M, dtype=u32, device=dev) if stages else None,
                    torch.empty(M, dtype=u32, device=dev) if stages else None,
                    torch.empty(M, dtype=u32, device=dev) if stages else None,
                    torch.empty(M, dtype=torch.uint8, device=dev) if stages else None,
                    *(torch.empty(K, dtype=u32, device=dev) for _ in range(5)))
            if reuse:
                if not hasattr(self, "_bufs"):
                    self._bufs = {}
                self._bufs[bkey] = bufs
        sa, lcp, cl, ci, cs, ca, ss, sl, st, tl, ts = bufs
        counts = (ctypes.c_uint64 * 4)()
        offs = [np.zeros(W + 1, dtype=np.uint64) for _ in range(3)]
        o = apo_repeats_out(_ptr(sa), _ptr(lcp), _ptr(cl), _ptr(ci), _ptr(cs), _ptr(ca),
                            M if stages else 0, _ptr(ss), _ptr(sl), _ptr(st), K, _ptr(tl), _ptr(ts), K,
                            ctypes.cast(counts, _P), *[x.ctypes.data_as(_P).value for x in offs])
        w = apo_windows(W, _ptr(tokens), _token_bytes(tokens), wo.ctypes.data_as(_P).value)
        p = apo_repeats_params(int(min_len), 0)
        _check(lib().apo_find_repeats_batched(self._h, ctypes.byref(w), ctypes.byref(p), ctypes.byref(o),
                                              _stream_handle(stream)))
        m, k, t, rounds = (int(x) for x in counts)

        def cut(x, c):
            return None if x is None else x[:c]
        return BatchRepeats(cut(sa, n), cut(lcp, n), cut(cl, m), cut(ci, m), cut(cs, m), cut(ca, m),
                            ss[:k], sl[:k], st[:k], tl[:t], ts[:t], rounds, wo, *offs)

    # -------------------------------------------------------------- Sec. 4.3
    def match_candidates(self, pat_tokens, pat_off, stream_tokens, cap: int | None = None,
                         stream=None, pat_start=None, pat_len=None, src_sa=None, src_lcp=None):
        """All (end, pattern id) occurrences in stream_tokens, sorted.  Patterns
        are either a host CSR (pat_off) over pat_tokens, or device slices
        (pat_start, pat_len, with pat_off None) of pat_tokens; for slices,
        src_sa / src_lcp (the suffix and LCP arrays of pat_tokens, as
        find_repeats returns them) let the automaton be read off them."""
        import torch
        n = int(stream_tokens.shape[0])
        if cap is None:
            cap = max(1, 4 * n)
        end = torch.empty(max(1, cap), dtype=torch.int32, device=stream_tokens.device)
        pid = torch.empty(max(1, cap), dtype=torch.int32, device=stream_tokens.device)
        cnt = _U64(0)
        if pat_off is not None:
            po = np.ascontiguousarray(np.asarray(pat_off, dtype=np.uint64))
            p = apo_patterns(po.shape[0] - 1, _ptr(pat_tokens), _token_bytes(pat_tokens),
                             po.ctypes.data_as(_P).value, None, None)
        else:
            p = apo_patterns(int(pat_start.shape[0]), _ptr(pat_tokens), _token_bytes(pat_tokens),
                             None, _ptr(pat_start), _ptr(pat_len), _ptr(src_sa), _ptr(src_lcp),
                             int(pat_tokens.shape[0]) if src_sa is not None else 0)
        code = lib().apo_match_candidates(self._h, ctypes.byref(p), _ptr(stream_tokens), n, _ptr(end),
                                          _ptr(pid), cap, ctypes.byref(cnt), _stream_handle(stream))
        if code == APO_ECAPACITY:
            return self.match_candidates(pat_tokens, pat_off, stream_tokens, int(cnt.value), stream,
                                         pat_start, pat_len, src_sa, src_lcp)
        _check(code)
        c = int(cnt.value)
        return end[:c], pid[:c]

    def replay(self, stream_tokens, start, length, ingest, max_trace_len: int = 0, count_cap: int = 0,
               half_life: int = 0, bonus=(1, 1), window: int = 0, traced: bool = True, curve: bool = False,
               rep_cap: int | None = None, stream=None):
        """Alg. 1's TraceReplayer over stream_tokens (device): trace q is
        stream_tokens[start[q] : start[q] + length[q]] and enters the trie at
        task ingest[q] (all device u32 tensors).  Returns (end, len, trace)
        of the replays, the traced flags (u8 per task) or None, the curve
        (traced tasks among the last `window`) or None, and the counts."""
        import torch
        n = int(stream_tokens.shape[0])
        dev = stream_tokens.device
        cap = max(1, n if rep_cap is None else rep_cap)
        end = torch.empty(cap, dtype=torch.int32, device=dev)
        ln = torch.empty(cap, dtype=torch.int32, device=dev)
        tr = torch.empty(cap, dtype=torch.int32, device=dev)
        tf = torch.empty(max(1, n), dtype=torch.uint8, device=dev) if traced else None
        cv = torch.empty(max(1, n), dtype=torch.int32, device=dev) if curve else None
        counts = np.zeros(8, dtype=np.uint64)
        t = apo_replay_traces(int(start.shape[0]), _ptr(start), _ptr(length), _ptr(ingest))
        p = apo_replay_params(max_trace_len, count_cap, half_life, bonus[0], bonus[1], window)
        o = apo_replay_out(_ptr(end), _ptr(ln), _ptr(tr), cap, _ptr(tf), _ptr(cv), counts.ctypes.data_as(_P).value)
        _check(lib().apo_replay(self._h, _ptr(stream_tokens), n, _token_bytes(stream_tokens), ctypes.byref(t),
                                ctypes.byref(p), ctypes.byref(o), _stream_handle(stream)))
        r = int(counts[0])
        return (end[:r], ln[:r], tr[:r], None if tf is None else tf[:n], None if cv is None else cv[:n],
                [int(x) for x in counts])

    def optimum_batched(self, tokens, win_off, min_len: int, stream=None):
        """Sec. 3's optimum (traces required to repeat) for every window of
        the concatenated device tokens (host offsets win_off): per window
        (coverage, intervals, |T|) as an int32 [W, 3] tensor, and the
        witness intervals (start, len) at each window's offset with their
        counts."""
        import torch
        wo = np.ascontiguousarray(np.asarray(win_off, dtype=np.uint64))
        W = wo.shape[0] - 1
        dev = tokens.device
        best = torch.empty((max(1, W), 3), dtype=torch.int32, device=dev)
        n = int(tokens.shape[0])
        ws_ = torch.empty(max(1, n), dtype=torch.int32, device=dev)
        wl = torch.empty(max(1, n), dtype=torch.int32, device=dev)
        wc = torch.empty(max(1, W), dtype=torch.int32, device=dev)
        w = apo_windows(W, _ptr(tokens), _token_bytes(tokens), wo.ctypes.data_as(_P).value)
        _check(lib().apo_optimum_batched(self._h, ctypes.byref(w), min_len, _ptr(best), _ptr(ws_), _ptr(wl),
                                         _ptr(wc), _stream_handle(stream)))
        return best[:W], ws_[:n], wl[:n], wc[:W]

    def graph_mode(self, enable: bool = True):
        """Replay batched calls with unchanged arguments as CUDA graphs
        (apo_graph_mode); results are the same as without."""
        _check(lib().apo_graph_mode(self._h, int(bool(enable))))

    def graph_stats(self) -> dict:
        a, b, c = _U64(0), _U64(0), _U64(0)
        _check(lib().apo_graph_stats(self._h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
        return {"replays": int(a.value), "captures": int(b.value), "discarded": int(c.value)}

    # -------------------------------------------------------------- sort tuning
    def sort_tuning(self, mode: int):
        """0: time the radix-sort shapes per size class and key width on first
        use (default); 1: always the default shape; 2 + k: always shape k."""
        _check(lib().apo_sort_tuning(self._h, int(mode)))

    def sort_tuning_read(self) -> list:
        """The shapes chosen so far, one dict per (size class, key bits)."""
        out = []
        i = 0
        while True:
            sl, kb, tn = _U32(0), _U32(0), _U32(0)
            th, it, db = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_int(0)
            bm, dm = ctypes.c_double(0), ctypes.c_double(0)
            if lib().apo_sort_tuning_read(self._h, i, ctypes.byref(sl), ctypes.byref(kb), ctypes.byref(tn),
                                          ctypes.byref(th), ctypes.byref(it), ctypes.byref(db),
                                          ctypes.byref(bm), ctypes.byref(dm)) != APO_OK:
                break
            out.append({"size_log2": sl.value, "key_bits": kb.value, "trial_n": tn.value,
                        "threads": th.value, "items": it.value, "digit_bits": db.value,
                        "best_ms": bm.value, "default_ms": dm.value})
            i += 1
        return out

    # -------------------------------------------------------------- instrumentation
    def profile(self, enable_timing: bool = True):
        _check(lib().apo_profile_enable(self._h, int(enable_timing)))

    def profile_reset(self):
        _check(lib().apo_profile_reset(self._h))

    def profile_read(self) -> dict:
        """{kernel: (launches, ms, units)} for every kernel launched so far."""
        out = {}
        name = ctypes.create_string_buffer(64)
        i = 0
        while True:
            la, un, ms = _U64(0), _U64(0), ctypes.c_double(0)
            if lib().apo_profile_read(self._h, i, name, 64, ctypes.byref(la), ctypes.byref(ms),
                                      ctypes.byref(un)) != APO_OK:
                break
            if la.value:
                out[name.value.decode()] = (int(la.value), float(ms.value), int(un.value))
            i += 1
        return out


@dataclass
class ServedResult:
    n: int
    sel_start: np.ndarray
    sel_len: np.ndarray
    sel_trace: np.ndarray
    trace_len: np.ndarray
    trace_start: np.ndarray
    t_submit: float
    t_start: float
    t_done: float
    batch_windows: int


class apo_finder_config(ctypes.Structure):
    _fields_ = [("buffer_tokens", _U64), ("unit", _U64)]


class apo_finder_result(ctypes.Structure):
    _fields_ = [("index", _U64), ("slice_start", _U64), ("slice_len", _U64), ("status", ctypes.c_int),
                ("n_traces", _U64), ("trace_len", _P), ("trace_start", _P), ("t_submit", ctypes.c_double),
                ("t_done", ctypes.c_double)]


@dataclass
class FinderResult:
    index: int
    slice_start: int
    slice_len: int
    trace_len: np.ndarray
    trace_start: np.ndarray
    t_submit: float
    t_done: float


class Finder:
    """Alg. 1's online TraceFinder with Sec. 4.4's ruler-function sampling
    (apo_finder_*): push tokens as they are issued; every `unit` tokens the
    most recent unit * 2^ruler(i) tokens (at most `buffer_tokens`) go to the
    server as one asynchronous analysis; poll returns them in order."""

    def __init__(self, server: "Server", buffer_tokens: int = 5000, unit: int = 250):
        self.server = server
        h = _P()
        cfg = apo_finder_config(buffer_tokens, unit)
        _check(lib().apo_finder_create(ctypes.byref(h), server._h, ctypes.byref(cfg)))
        self._h = h

    def push(self, tokens) -> int:
        a = np.ascontiguousarray(np.asarray(tokens).astype(self.server._dt, copy=False))
        subs = _U64(0)
        _check(lib().apo_finder_push(self._h, a.ctypes.data_as(_P).value, a.shape[0], ctypes.byref(subs)))
        return int(subs.value)

    def poll(self, wait: bool = False):
        """The next analysis in order, or None (still running / none left)."""
        r = apo_finder_result()
        code = lib().apo_finder_poll(self._h, int(wait), ctypes.byref(r))
        if code in (APO_EAGAIN, APO_ECAPACITY):
            return None
        _check(code)
        _check(r.status)
        k = int(r.n_traces)
        tl = (np.ctypeslib.as_array(ctypes.cast(r.trace_len, ctypes.POINTER(ctypes.c_uint32)), shape=(k,)).copy()
              if k else np.zeros(0, np.uint32))
        ts = (np.ctypeslib.as_array(ctypes.cast(r.trace_start, ctypes.POINTER(ctypes.c_uint64)), shape=(k,)).copy()
              if k else np.zeros(0, np.uint64))
        return FinderResult(int(r.index), int(r.slice_start), int(r.slice_len), tl, ts, r.t_submit, r.t_done)

    def drain(self) -> list:
        out = []
        while True:
            r = self.poll(wait=True)
            if r is None:
                return out
            out.append(r)

    def stats(self) -> dict:
        a, b, c = _U64(0), _U64(0), _U64(0)
        _check(lib().apo_finder_stats(self._h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
        return {"pushed": int(a.value), "analyses": int(b.value), "analysed_tokens": int(c.value)}

    def close(self):
        if getattr(self, "_h", None):
            lib().apo_finder_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous batching of repeat-finding requests (apo_server_*): submit
    host token windows at any time; lanes batch whatever is waiting, up to
    max_batch_tokens tokens and max_batch_windows requests, and run them on
    the GPU, several batches in flight at once."""

    def __init__(self, device: int = 0, min_len: int = 5, token_bytes: int = 4,
                 max_batch_tokens: int = 1 << 24, max_batch_windows: int = 512, lanes: int = 2,
                 hbm_budget: int = 0):
        self.token_bytes = token_bytes
        self._dt = np.uint32 if token_bytes == 4 else np.uint64
        h = _P()
        cfg = apo_server_config(min_len, token_bytes, max_batch_tokens, max_batch_windows, lanes, hbm_budget)
        _check(lib().apo_server_create(ctypes.byref(h), device, ctypes.byref(cfg)))
        self._h = h

    def memory(self) -> dict:
        """The pool's size and the bytes batches in flight hold (now, most at once)."""
        b, h, m = _U64(), _U64(), _U64()
        _check(lib().apo_server_memory(self._h, ctypes.byref(b), ctypes.byref(h), ctypes.byref(m)))
        return {"budget": int(b.value), "held": int(h.value), "held_max": int(m.value)}

    @staticmethod
    def footprint(n_tokens: int, token_bytes: int = 4, min_len: int = 5) -> int:
        """Bytes one request of n_tokens takes from the pool when it is
        batched alone (tokens, outputs, analysis scratch)."""
        wo = np.array([0, n_tokens], dtype=np.uint64)
        ws = apo_windows(1, None, token_bytes, wo.ctypes.data)
        out = _U64()
        _check(lib().apo_find_repeats_workspace(None, ctypes.byref(ws), ctypes.byref(out)))
        al = lambda b: (b + 255) & ~255  # noqa: E731
        return al(n_tokens * token_bytes + 16) + al(5 * (n_tokens // max(min_len, 1) + 1) * 4) + al(int(out.value))

    def submit(self, tokens) -> int:
        a = np.ascontiguousarray(np.asarray(tokens).astype(self._dt, copy=False))
        rid = _U64(0)
        _check(lib().apo_server_submit(self._h, a.ctypes.data_as(_P).value, a.shape[0], ctypes.byref(rid)))
        return int(rid.value)

    @staticmethod
    def _arr(p, k):
        if k == 0:
            return np.zeros(0, np.uint32)
        return np.ctypeslib.as_array(ctypes.cast(p, ctypes.POINTER(ctypes.c_uint32)), shape=(k,)).copy()

    def _take(self, rid, r) -> ServedResult:
        _check(r.status)
        out = ServedResult(int(r.n), self._arr(r.sel_start, r.n_selected), self._arr(r.sel_len, r.n_selected),
                           self._arr(r.sel_trace, r.n_selected), self._arr(r.trace_len, r.n_traces),
                           self._arr(r.trace_start, r.n_traces), r.t_submit, r.t_start, r.t_done,
                           int(r.batch_windows))
        _check(lib().apo_server_release(self._h, rid))
        return out

    def poll(self, rid: int):
        r = apo_request_result()
        code = lib().apo_server_poll(self._h, rid, ctypes.byref(r))
        if code == APO_EAGAIN:
            return None
        _check(code)
        return self._take(rid, r)

    def wait(self, rid: int) -> ServedResult:
        r = apo_request_result()
        _check(lib().apo_server_wait(self._h, rid, ctypes.byref(r)))
        return self._take(rid, r)

    def now(self) -> float:
        return float(lib().apo_server_now(self._h))

    def close(self):
        if getattr(self, "_h", None):
            lib().apo_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def greedy_select_noalloc(cand_len, cand_start, n: int, accepted, accepted_count, stream=None):
    """apo_greedy_select_noalloc, for callers that cannot allocate device
    memory (see include/apo.h): accepted[k] = 1 iff the interval
    [cand_start[k], cand_start[k] + cand_len[k]) meets no interval accepted
    before it, visiting the m candidates in the order given; cand_len must not
    increase along that order (apo_find_repeats's candidate order satisfies
    this), and *accepted_count receives the number accepted, or 0xffffffff
    (-1 as int32) when a length increases.

    All tensors are caller-owned buffers on one CUDA device: cand_len and
    cand_start int32 with m entries each, accepted uint8 with at least m,
    accepted_count int32 with at least 1, all contiguous.  Anything else is
    refused with ValueError before the library is called, so that no kernel
    reads or writes past a buffer.  The call runs with that device current and
    only enqueues the work on `stream`."""
    import torch
    named = (("cand_len", cand_len), ("cand_start", cand_start), ("accepted", accepted),
             ("accepted_count", accepted_count))
    for name, t in named:
        if not isinstance(t, torch.Tensor):
            raise ValueError(f"greedy_select_noalloc: {name} must be a torch.Tensor")
        if t.dim() != 1 or not t.is_contiguous():
            raise ValueError(f"greedy_select_noalloc: {name} must be a contiguous 1-D tensor")
    want = {"cand_len": torch.int32, "cand_start": torch.int32, "accepted": torch.uint8,
            "accepted_count": torch.int32}
    for name, t in named:
        if t.dtype != want[name]:
            raise ValueError(f"greedy_select_noalloc: {name} must be {want[name]}, got {t.dtype}")
    m = int(cand_len.shape[0])
    if int(cand_start.shape[0]) != m:
        raise ValueError(f"greedy_select_noalloc: cand_start has {cand_start.shape[0]} entries, cand_len {m}")
    if int(accepted.shape[0]) < m:
        raise ValueError(f"greedy_select_noalloc: accepted holds {accepted.shape[0]} entries, need {m}")
    if int(accepted_count.shape[0]) < 1:
        raise ValueError("greedy_select_noalloc: accepted_count needs one entry")
    if int(n) < 0:
        raise ValueError("greedy_select_noalloc: n must be >= 0")
    devs = {t.device for _, t in named}
    if len(devs) != 1 or next(iter(devs)).type != "cuda":
        raise ValueError(f"greedy_select_noalloc: all tensors must be on one CUDA device, got {sorted(map(str, devs))}")
    with torch.cuda.device(next(iter(devs))):
        _check(lib().apo_greedy_select_noalloc(_ptr(cand_len), _ptr(cand_start), m, int(n), _ptr(accepted),
                                               _ptr(accepted_count), _stream_handle(stream)))


def as_u32(t) -> np.ndarray:
    """Device int32 tensor (u32 bit patterns) -> numpy uint32."""
    return t.cpu().numpy().view(np.uint32)


def as_u64(t) -> np.ndarray:
    """Device int64 tensor (u64 bit patterns) -> numpy uint64."""
    return t.cpu().numpy().view(np.uint64)
