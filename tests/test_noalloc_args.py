"""greedy_select_noalloc refuses malformed buffers before the library is
called (no GPU needed): a wrong dtype, a short or non-contiguous buffer, or
tensors off a CUDA device would otherwise become out-of-bounds device reads
or writes."""
import pytest

torch = pytest.importorskip("torch")

from paper_2406_18111_gb300 import greedy_select_noalloc  # noqa: E402


def _args(m=8):
    return dict(cand_len=torch.zeros(m, dtype=torch.int32), cand_start=torch.zeros(m, dtype=torch.int32),
                accepted=torch.zeros(m, dtype=torch.uint8), accepted_count=torch.zeros(1, dtype=torch.int32))


def _call(a, n=100):
    greedy_select_noalloc(a["cand_len"], a["cand_start"], n, a["accepted"], a["accepted_count"])


@pytest.mark.parametrize("name,bad,match", [
    ("cand_len", torch.zeros(8, dtype=torch.int64), "must be torch.int32"),
    ("cand_start", torch.zeros(8, dtype=torch.float32), "must be torch.int32"),
    ("accepted", torch.zeros(8, dtype=torch.int32), "must be torch.uint8"),
    ("accepted_count", torch.zeros(1, dtype=torch.int64), "must be torch.int32"),
    ("cand_start", torch.zeros(7, dtype=torch.int32), "cand_start has 7 entries"),
    ("accepted", torch.zeros(7, dtype=torch.uint8), "accepted holds 7 entries"),
    ("accepted_count", torch.zeros(0, dtype=torch.int32), "needs one entry"),
    ("cand_len", torch.zeros(16, dtype=torch.int32)[::2], "contiguous 1-D"),
    ("accepted", torch.zeros(2, 4, dtype=torch.uint8), "contiguous 1-D"),
    ("cand_len", [0] * 8, "torch.Tensor"),
])
def test_malformed_buffers_are_refused(name, bad, match):
    a = _args()
    a[name] = bad
    with pytest.raises(ValueError, match=match):
        _call(a)


def test_host_tensors_are_refused():
    with pytest.raises(ValueError, match="one CUDA device"):
        _call(_args())


def test_negative_window_is_refused():
    with pytest.raises(ValueError, match="n must be"):
        _call(_args(), n=-1)
