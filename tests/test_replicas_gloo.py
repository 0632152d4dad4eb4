"""Multi-process replica bookkeeping of bench.py on CPU (gloo, world size 2):
barrier, max over ranks, and distinct RNG streams per rank (lattice_id = rank)."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    import oracle
    import torch.distributed as dist

    w, r, loc = bench.dist_setup()
    d = bench.Dist(w, r, loc, use_cuda=False)
    d.barrier()
    m = d.max(float(10 + r))
    dims = [4, 4, 2, 2]
    U = oracle.init_links(dims, 1, seed=3, lattice_id=r)   # one stream per replica
    p = oracle.update_chain(U, dims, 5.7, 3, r, 0, 2, 1, 1)[-1]
    import torch

    t = torch.tensor([p], dtype=torch.float64)
    out = [torch.zeros(1, dtype=torch.float64) for _ in range(w)]
    dist.all_gather(out, t)
    q.put((r, m, [float(x.item()) for x in out]))
    d.close()


def test_two_replicas_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    assert res[0][1] == res[1][1] == 11.0            # max over ranks
    assert res[0][2] == res[1][2]                    # both ranks gathered the same pair
    assert res[0][2][0] != res[0][2][1]              # distinct lattice_id streams
