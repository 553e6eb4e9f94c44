"""The workspace query and the caller-owned workspace of the repeat calls.

CPU: apo_find_repeats_workspace through the C ABI (it needs no GPU or
context): a positive size that grows with the tokens and the window count,
and refusals of malformed arguments.  GPU: calls with a caller workspace of
exactly the queried size give the same bytes as with the context's own
scratch; one byte too few is refused before any launch; detaching returns
to the context's own scratch."""
import ctypes

import numpy as np
import pytest

import workloads as W


def _query(win_off):
    import paper_2406_18111_gb300 as P
    wo = np.ascontiguousarray(np.asarray(win_off, dtype=np.uint64))
    ws = P.apo_windows(wo.shape[0] - 1, None, 4, wo.ctypes.data)
    out = ctypes.c_uint64()
    rc = P.lib().apo_find_repeats_workspace(None, ctypes.byref(ws), ctypes.byref(out))
    return rc, int(out.value)


def test_workspace_query_through_the_abi():
    import paper_2406_18111_gb300 as P
    sizes = []
    for n in (1, 1000, 1 << 16, 1 << 20, 1 << 24):
        rc, b = _query([0, n])
        assert rc == P.APO_OK and b > 0
        sizes.append(b)
    assert sizes == sorted(sizes) and sizes[-1] > 100 * (1 << 24)  # a few hundred bytes per token
    rc1, one = _query([0, 1 << 20])
    rc2, many = _query(np.linspace(0, 1 << 20, 513).astype(np.uint64))
    assert rc1 == rc2 == P.APO_OK and many >= one
    rc, _ = _query([0, 1 << 31])
    assert rc == P.APO_EINVAL
    out = ctypes.c_uint64()
    assert P.lib().apo_find_repeats_workspace(None, None, ctypes.byref(out)) == P.APO_EINVAL


@pytest.mark.gpu
def test_caller_workspace_gives_the_same_results():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2406_18111_gb300 import Apo, ApoError, as_u32
    a = Apo(0)
    S = W.config1_window(1 << 16, seed=7)
    t = torch.from_numpy(S.view(np.int32)).cuda()
    toks, off, _ = W.config3_windows(16)
    tb = torch.from_numpy(toks.view(np.int32)).cuda()
    want1 = a.find_repeats(t, 5)
    wantb = a.find_repeats_batched(tb, off, 5)
    need = max(a.find_repeats_workspace([0, S.shape[0]]), a.find_repeats_workspace(off))
    buf = torch.empty(need, dtype=torch.uint8, device="cuda")
    a.set_workspace(buf)
    for _ in range(2):  # twice: the second call reuses the attached look-back words
        got1 = a.find_repeats(t, 5)
        gotb = a.find_repeats_batched(tb, off, 5)
        for f in ("sa", "lcp", "cand_len", "cand_start", "sel_start", "sel_len", "trace_len", "trace_start"):
            assert np.array_equal(as_u32(getattr(got1, f)), as_u32(getattr(want1, f))), f
            assert np.array_equal(as_u32(getattr(gotb, f)), as_u32(getattr(wantb, f))), f
    small = torch.empty(a.find_repeats_workspace(off) - 1, dtype=torch.uint8, device="cuda")
    a.set_workspace(small)
    with pytest.raises(ApoError, match="APO_ENOMEM"):
        a.find_repeats_batched(tb, off, 5)
    a.set_workspace(None)
    again = a.find_repeats_batched(tb, off, 5)
    assert np.array_equal(as_u32(again.sel_start), as_u32(wantb.sel_start))
    a.close()
