"""Multi-GPU runs of bench.py are replicas (independent solves; no collective on the data
path). Its host-side rank logic — rendezvous from the torchrun environment, the barriers
around the timed region and the max over ranks of the timed span — is checked here with
two gloo ranks on the CPU."""
import importlib.util
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench", os.path.join(ROOT, "bench.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


def _rank(rank, ws, port, q):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(ws), LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    b = _bench()
    got_ws, got_rank, local = b.dist_setup()
    b.barrier(got_ws)
    span = 1.0 + rank                      # rank r "took" 1 + r seconds
    mx = b.max_over_ranks(span, got_ws)
    b.barrier(got_ws)
    import torch.distributed as dist
    dist.destroy_process_group()
    q.put((got_rank, got_ws, local, mx))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_gloo_ranks_share_the_max_span():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    out = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[0] for o in out] == [0, 1]
    assert all(o[1] == 2 for o in out)
    assert all(o[3] == 2.0 for o in out)      # both ranks report the slowest rank's span


def test_single_process_needs_no_rendezvous():
    b = _bench()
    env = {k: os.environ.pop(k) for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK") if k in os.environ}
    try:
        assert b.dist_setup() == (1, 0, 0)
        assert b.max_over_ranks(3.5, 1) == 3.5
    finally:
        os.environ.update(env)
