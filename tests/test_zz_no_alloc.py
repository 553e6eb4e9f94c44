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


def test_noalloc_rejects_oversized_window(apo):
    import torch
    from paper_2406_18111_gb300 import NOALLOC_MAX_WINDOW, ApoError, greedy_select_noalloc
    z = torch.zeros(4, dtype=torch.int32, device="cuda")
    acc = torch.zeros(4, dtype=torch.uint8, device="cuda")
    with pytest.raises(ApoError, match="exceeds the fixed maximum"):
        greedy_select_noalloc(z, z, NOALLOC_MAX_WINDOW + 1, acc, z[:1])
