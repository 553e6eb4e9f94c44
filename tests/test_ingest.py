"""Agreed ingestion of asynchronous analyses across nodes (Sec. 4.5) on CPU
ranks: gloo processes stand in for the nodes.  Every node must ingest every
analysis at the same operation, equal to the sequential recurrence of the
oracle over all nodes' completion times, and the lags must settle."""
import os
import socket

import numpy as np
import pytest

import oracle
import workloads as W


def _schedule(n_ops=200_000, unit=250, buffer=5000):
    sched = oracle.ruler_schedule(n_ops, unit, buffer)
    submit = [i * unit for i, _, _ in sched]
    lens = [l for _, _, l in sched]
    return submit, lens


def test_single_node_equals_recurrence():
    from paper_2406_18111_gb300.ingest import simulate_node
    submit, lens = _schedule()
    ready = W.analysis_ready_ops(submit, lens, node=0)
    pts, waits = simulate_node(submit, ready, lag0=250)
    want, wwait, wlag = oracle.ingestion_points(submit, [ready], 250)
    assert [p for _, p, _, _ in pts] == want
    assert [w for _, _, w, _ in pts] == wwait == waits
    assert [l for _, _, _, l in pts] == wlag


def test_recurrence_by_hand():
    # lag 10, doubling: analysis 0 (submitted at 0) ingested at 10 but ready
    # at 15 on node 1 -> waited, lag 20; analysis 1 (at 5) -> 25, ready at
    # 20/12 -> no wait; analysis 2 (at 30) -> 50
    pts, waited, lags = oracle.ingestion_points([0, 5, 30], [[3, 20, 31], [15, 12, 49]], 10)
    assert pts == [10, 25, 50] and waited == [True, False, False] and lags == [10, 20, 20]


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import torch
    import torch.distributed as dist
    from paper_2406_18111_gb300.ingest import simulate_node, torch_reduce_max
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        submit, lens = _schedule()
        ready = W.analysis_ready_ops(submit, lens, node=rank)
        pts, waits = simulate_node(submit, ready, lag0=250, reduce_max=torch_reduce_max())
        mine = torch.tensor([p for _, p, _, _ in pts], dtype=torch.int64)
        allp = [torch.zeros_like(mine) for _ in range(world)]
        dist.all_gather(allp, mine)
        q.put((rank, [t.tolist() for t in allp], [l for _, _, _, l in pts], sum(waits)))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_nodes_agree_on_ingestion(world):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=180) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    submit, lens = _schedule()
    readies = [W.analysis_ready_ops(submit, lens, node=r) for r in range(world)]
    want, waited, lags = oracle.ingestion_points(submit, readies, 250)
    for rank, allp, mylags, nwait in res:
        for other in allp:
            assert other == want  # every node ingests every analysis at the same op
        assert mylags == lags
    # the lags settle: no node waits in the second half of the stream
    assert not any(waited[len(waited) // 2:])
    assert lags[-1] > 250  # some early wait raised the lag


def test_agreed_points_make_replays_identical():
    # the same stream and traces on two nodes: ingesting each analysis when
    # the node has it gives different replays, the agreed points identical ones
    S = W.replay_stream(1 << 15, seed=6)
    unit = 250
    res = oracle.online_traces(S, unit, 5000, 5)
    submit = [i * unit for i, _, _, _, _ in res]
    lens = [l for _, _, l, _, _ in res]
    readies = [W.analysis_ready_ops(submit, lens, node=r, jitter=2000) for r in range(2)]
    pts, _, _ = oracle.ingestion_points(submit, readies, unit)

    def replay_with(times):
        st = np.concatenate([ts for *_, ts in res]).astype(np.uint64)
        ln = np.concatenate([tl for *_, tl, _ in res]).astype(np.uint64)
        ig = np.concatenate([np.full(len(r[3]), t, np.uint64) for r, t in zip(res, times)])
        return oracle.replay(S.astype(np.uint64), st, ln, ig, 0, 8, 1000, (17, 16))

    local = [replay_with(r) for r in readies]
    assert not np.array_equal(local[0].end, local[1].end) or not np.array_equal(local[0].trace, local[1].trace)
    agreed = [replay_with(pts) for _ in range(2)]
    assert np.array_equal(agreed[0].end, agreed[1].end) and np.array_equal(agreed[0].trace, agreed[1].trace)
