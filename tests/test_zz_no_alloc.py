"""apo_greedy_select_noalloc, the entry point for callers that cannot
allocate device memory (a runtime that owns all device memory, or a path that
must not pay for cudaMalloc's device-wide synchronisation).  Its output must
equal the accepted flags apo_find_repeats computes for the same candidates,
on two calls in a row (the second call reuses the fixed scratch array the
first one left behind).  Kept in its own file so that it is collected last."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


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


def _window(S):
    import torch
    return torch.from_numpy(np.ascontiguousarray(S, dtype=np.uint32).view(np.int32)).cuda()


def test_noalloc_greedy_matches_find_repeats(apo):
    import torch
    from paper_2406_18111_gb300 import greedy_select_noalloc
    windows = [W.config1_window(), W.periodic_window(200003, 977, 0.05, 1000, seed=31)]
    for S in windows:  # two calls in a row, different windows
        t = _window(S)
        r = apo.find_repeats(t, 5)
        m = int(r.cand_len.shape[0])
        assert m > 0
        acc = torch.full((m,), 7, dtype=torch.uint8, device=t.device)
        cnt = torch.full((1,), -1, dtype=torch.int32, device=t.device)
        greedy_select_noalloc(r.cand_len, r.cand_start, int(S.shape[0]), acc, cnt)
        torch.cuda.synchronize()
        assert torch.equal(acc, r.cand_accepted)
        assert int(cnt.item()) == int(r.cand_accepted.sum().item()) == int(r.sel_start.shape[0])


def _noalloc(cl, cs, n):
    import torch
    from paper_2406_18111_gb300 import greedy_select_noalloc
    m = int(cl.shape[0])
    acc = torch.full((max(m, 1),), 7, dtype=torch.uint8, device="cuda")
    cnt = torch.full((1,), -2, dtype=torch.int32, device="cuda")
    greedy_select_noalloc(cl, cs, n, acc[:m], cnt)
    torch.cuda.synchronize()
    return acc[:m], int(cnt.item())


def test_noalloc_window_sizes_in_sequence(apo):
    """A window at the fixed maximum, then a small one, then the large one
    again: no marks left from a larger window leak into a smaller one, and
    the full bitmap is used correctly."""
    from paper_2406_18111_gb300 import NOALLOC_MAX_WINDOW
    big = W.periodic_window(NOALLOC_MAX_WINDOW, 4999, 0.05, 1000, seed=37)
    small = W.config1_window()
    for S in (big, small, big):
        t = _window(S)
        r = apo.find_repeats(t, 5)
        acc, cnt = _noalloc(r.cand_len, r.cand_start, int(S.shape[0]))
        assert acc.equal(r.cand_accepted)
        assert cnt == int(r.cand_accepted.sum().item()) == int(r.sel_start.shape[0])


def test_noalloc_batch_boundary_and_empty(apo):
    """Hand-built candidate lists of exactly 1024 and 1025 entries (the
    kernel's batch size and one past it) against the oracle's greedy; no
    candidates at all gives a count of 0."""
    import torch
    import oracle
    n = 5000
    for m in (1024, 1025, 1):
        ln = np.sort(W.uniform_int(60 + m, m, 1, 40))[::-1].astype(np.uint32)
        st = (W.uniform_int(70 + m, m, 0, n - 41)).astype(np.uint32)
        want = oracle.greedy(n, ln, st)
        cl = torch.from_numpy(ln.view(np.int32).copy()).cuda()
        cs = torch.from_numpy(st.view(np.int32).copy()).cuda()
        acc, cnt = _noalloc(cl, cs, n)
        assert np.array_equal(acc.cpu().numpy(), want), m
        assert cnt == int(want.sum())
    z = torch.zeros(0, dtype=torch.int32, device="cuda")
    acc, cnt = _noalloc(z, z, n)
    assert cnt == 0


def test_noalloc_flags_increasing_length(apo):
    """A list whose lengths increase breaks the precondition; the count says so."""
    import torch
    cl = torch.tensor([3, 5, 2], dtype=torch.int32, device="cuda")
    cs = torch.tensor([0, 10, 20], dtype=torch.int32, device="cuda")
    _, cnt = _noalloc(cl, cs, 100)
    assert cnt == -1


def test_noalloc_rejects_oversized_window(apo):
    import torch
    from paper_2406_18111_gb300 import NOALLOC_MAX_WINDOW, ApoError, greedy_select_noalloc
    z = torch.zeros(4, dtype=torch.int32, device="cuda")
    acc = torch.zeros(4, dtype=torch.uint8, device="cuda")
    with pytest.raises(ApoError, match="exceeds the fixed maximum"):
        greedy_select_noalloc(z, z, NOALLOC_MAX_WINDOW + 1, acc, z[:1])
