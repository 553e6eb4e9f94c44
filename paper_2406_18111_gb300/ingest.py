"""Deterministic ingestion of asynchronous analyses across nodes (Sec. 4.5).

Every node issues the same task stream (control replication) and runs its
own asynchronous analyses, which finish at different times on different
nodes.  For all nodes to replay the same traces at the same tasks, the
result of analysis j is ingested when operation submit_j + lag_j is reached,
on every node; a node whose result is not ready there waits for it.  At
each ingestion the nodes agree (one max-reduction of a "waited" flag) on
whether anyone waited, and if so every node multiplies the lag of the next
analysis by `growth`.  The lags settle where no node waits, so ingestion is
deterministic without stalling the stream.  The agreed points are the
`ingest` times the replayer (apo_replay) takes.

The reduction is passed in: torch.distributed.all_reduce (gloo or NCCL)
between processes, or any callable with the same meaning.
"""
from __future__ import annotations

from collections import deque


class AgreedIngestion:
    """One node's side of the protocol.  Call submitted(j, op) when analysis
    j (numbered 0, 1, ... in submission order) is launched at operation op,
    next_point() for the operation at which the oldest pending analysis is
    ingested, and ingest(waited) when that operation is reached (waited:
    this node had to wait for the result); every node makes the same calls
    in the same order, since they issue the same stream."""

    def __init__(self, lag0: int, growth: int = 2, reduce_max=None):
        if lag0 < 1 or growth < 1:
            raise ValueError("lag0 >= 1 and growth >= 1")
        self.lag = int(lag0)
        self.growth = int(growth)
        self.reduce_max = reduce_max or (lambda v: v)
        self.pending = deque()  # (j, submit op)
        self.points = []        # (j, ingestion op, agreed waited, lag)

    def submitted(self, j: int, op: int) -> None:
        self.pending.append((int(j), int(op)))

    def next_point(self):
        """Operation at which the oldest pending analysis is ingested, or None."""
        if not self.pending:
            return None
        return self.pending[0][1] + self.lag

    def ingest(self, waited: bool) -> bool:
        """Ingest the oldest pending analysis; returns whether any node waited."""
        j, s = self.pending.popleft()
        p = s + self.lag
        anyone = bool(self.reduce_max(1 if waited else 0))
        self.points.append((j, p, anyone, self.lag))
        if anyone:
            self.lag *= self.growth
        return anyone


def torch_reduce_max(group=None):
    """A reduce_max over torch.distributed ranks."""
    import torch
    import torch.distributed as dist

    def f(v: int) -> int:
        t = torch.tensor([int(v)], dtype=torch.int64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
        return int(t.item())
    return f


def simulate_node(submit, ready, lag0: int, growth: int = 2, reduce_max=None):
    """Drive one node through a stream: analyses submitted at submit[j],
    ready on this node at ready[j]; returns the agreed ingestion points
    [(j, op, anyone waited, lag)] and this node's own waits."""
    ing = AgreedIngestion(lag0, growth, reduce_max)
    waits = []
    for j, s in enumerate(submit):
        # ingestions due before this submission
        while ing.next_point() is not None and ing.next_point() <= s:
            k = ing.pending[0][0]
            w = ready[k] > ing.next_point()
            waits.append(w)
            ing.ingest(w)
        ing.submitted(j, s)
    while ing.next_point() is not None:
        k = ing.pending[0][0]
        w = ready[k] > ing.next_point()
        waits.append(w)
        ing.ingest(w)
    return ing.points, waits
