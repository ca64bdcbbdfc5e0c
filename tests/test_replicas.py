"""Multi-rank host logic of the replica layout, on CPU with the gloo backend (world size 2).

Covers what the benchmark does across ranks -- per-rank poses, barrier, max over ranks, whole-job
rate -- and host-side failure detection: a rank that dies between steps is noticed by the other
rank through a short process-group timeout on its next collective, without any GPU involvement.
"""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _env(rank, world, port):
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    sys.path.insert(0, ROOT)


def _worker_ok(rank, world, port, q):
    _env(rank, world, port)
    from paper_2006_14726_b300.replicas import Replicas
    import synth
    r = Replicas.from_env("gloo", timeout_s=30)
    r.barrier()
    t = r.max_over_ranks(1.0 + rank)            # rank 1 is the slower one
    rate = r.whole_job_rate(100.0, t)
    poses = synth.LARGE.client_poses(2, seed_offset=r.pose_seed_offset())
    q.put((rank, t, rate, poses[0].eye))
    r.close()


def _worker_dies(rank, world, port, q):
    _env(rank, world, port)
    from paper_2006_14726_b300.replicas import Replicas
    r = Replicas.from_env("gloo", timeout_s=5)
    r.barrier()                                  # step 1 completes on both ranks
    if rank == 1:
        os._exit(3)                              # rank 1 leaves between steps
    try:
        r.max_over_ranks(2.0)                    # rank 0's next collective must fail, not hang
        q.put((rank, "no error"))
    except Exception as e:                       # noqa: BLE001
        q.put((rank, type(e).__name__))


def _run(fn, world=2, timeout=90):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=fn, args=(r, world, port, q)) for r in range(world)]
    for p in ps:
        p.start()
    for p in ps:
        p.join(timeout)
    alive = [p for p in ps if p.is_alive()]
    for p in alive:
        p.kill()
    assert not alive, "a rank hung"
    out = []
    while not q.empty():
        out.append(q.get())
    return out, [p.exitcode for p in ps]


def test_two_ranks_barrier_max_and_rate():
    out, codes = _run(_worker_ok)
    assert codes == [0, 0]
    res = {r[0]: r for r in out}
    assert res[0][1] == res[1][1] == 2.0           # max over ranks
    assert res[0][2] == res[1][2] == 2 * 100.0 / 2.0  # whole-job units / slowest time
    assert tuple(res[0][3]) != tuple(res[1][3])    # each rank traces its own poses


def test_dead_rank_is_detected_on_the_host():
    out, codes = _run(_worker_dies)
    assert codes[1] == 3
    res = dict(out)
    assert res.get(0) not in (None, "no error")
