"""The benchmark's multi-process host logic on the CPU: two gloo ranks.

The solves themselves need a GPU; what runs here is the rendezvous
(dist_init), the max-over-ranks timing that every rank agrees on, and the
reference arm's rule that only rank 0 works and prints.
"""
import importlib.util
import io
import os
import socket
import sys
from contextlib import redirect_stdout

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, q):
    os.environ.update(RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE=str(ws), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    b = _bench()
    r, w, local, dist = b.dist_init()
    assert (r, w, local) == (rank, ws, rank) and dist.get_backend() == "gloo"
    got = b.max_over_ranks(10.0 + 5.0 * rank, dist)  # rank 1 is the slow one
    # the reference arm: rank 0 alone prints its line; the other ranks return 0 at once
    out = io.StringIO()
    if rank != 0:
        with redirect_stdout(out):
            rc = b.run_reference(None, rank, ws)
        assert rc == 0 and out.getvalue() == ""
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, got))


def test_two_gloo_ranks_agree_on_max_time():
    torch = pytest.importorskip("torch")
    mp = torch.multiprocessing.get_context("spawn")
    q = mp.Queue()
    port = _free_port()
    procs = [mp.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
    got = sorted(q.get(timeout=5) for _ in range(2))
    assert got == [(0, 15.0), (1, 15.0)]


def test_single_process_needs_no_rendezvous(monkeypatch):
    monkeypatch.delenv("WORLD_SIZE", raising=False)
    b = _bench()
    assert b.dist_init() == (0, 1, 0, None)
    assert b.max_over_ranks(3.5, None) == 3.5
