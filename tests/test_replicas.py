"""The multi-GPU form is independent replicas (no data-path collective):
the host-side plumbing -- process group, barrier, max over ranks of the
timing, disjoint member seeds -- run as two gloo ranks on the CPU."""
import os
import socket

import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(ws), RANK=str(rank),
                      LOCAL_RANK=str(rank))
    from paper_2205_04148_gb300 import replicas
    w, r, loc = replicas.init("gloo")
    replicas.barrier()
    m = replicas.max_over_ranks(1.5 + rank, device="cpu")
    seeds = [replicas.member_seed(r, k) for k in range(24)]
    replicas.barrier()
    replicas.finish()
    out.put((r, w, loc, m, seeds))


def test_two_gloo_ranks():
    ws, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, ws, port, q)) for r in range(ws)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(ws))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[0] for r in res] == [0, 1] and all(r[1] == 2 for r in res)
    assert all(r[3] == 2.5 for r in res)                 # the slowest rank's time
    assert not set(res[0][4]) & set(res[1][4])           # members of the ranks differ


def test_single_rank_is_plain():
    from paper_2205_04148_gb300 import replicas
    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        os.environ.pop(k, None)
    assert replicas.world() == (1, 0, 0)
    assert replicas.max_over_ranks(3.0) == 3.0
    replicas.barrier()
