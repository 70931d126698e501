"""Host logic of the multi-GPU (independent replicas) path, on CPU with gloo ranks."""
import os
import socket

import pytest
import torch.multiprocessing as mp

from paper_2108_01438_gb300 import replicas


def test_assign_covers_every_scan_once_and_balances_bytes():
    sizes = [replicas.scan_bytes(w, d, d) for w, d in
             [(256, 1024), (2048, 2048), (512, 1024), (1024, 2048), (768, 1024), (384, 2048), (1536, 1024)]]
    for ws in (1, 2, 3, 4):
        parts = replicas.assign(sizes, ws)
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(sizes)))
        loads = [sum(sizes[i] for i in p) for p in parts]
        assert max(loads) - min(loads) <= max(sizes)
    assert replicas.assign(sizes, 2) == replicas.assign(list(sizes), 2)
    with pytest.raises(ValueError):
        replicas.assign(sizes, 0)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, ws, port, sizes, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    mine = replicas.assign(sizes, ws)[rank]
    t = replicas.max_over_ranks(1.0 + rank * 0.5)
    dist.barrier()
    q.put((rank, mine, t))
    dist.destroy_process_group()


def test_two_gloo_ranks_partition_and_reduce_max():
    sizes = [5, 9, 2, 7, 7, 1, 3]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, sizes, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, a0, t0), (r1, a1, t1) = res
    assert sorted(a0 + a1) == list(range(len(sizes))) and not set(a0) & set(a1)
    assert t0 == t1 == 1.5


def test_max_over_ranks_without_process_group():
    assert replicas.max_over_ranks(3.25) == 3.25
