"""Multi-rank ensemble sharding on CPU (gloo, world size 2).

Each rank advances its shard of an ensemble with the oracle and the FP64
accumulators are gathered; the result must equal a single-process run bit for
bit, because a system's evolution depends only on its own descriptor."""
import os
import socket

import numpy as np
import pytest

import synth


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _systems():
    out = []
    for k, n in enumerate([8, 12, 16, 10, 8, 14]):
        out.append(synth.system("D2Q9", n=n, a=0.002 * (k - 2), seed=1 + k % 2, system_id=k))
    return out


def _run_one(s, steps=12, every=4):
    from oracle import lbm, observables as ob
    from tests.helpers import params_of
    p = params_of(s)
    rec = ob.Recorder(p, every=every)
    f = lbm.run(lbm.initial_state(p), 0, steps, p, callback=rec)
    return {"acc": rec.acc, "f_sum": f.sum(axis=0)}


def _worker(rank, world, port, outdir):
    import torch.distributed as dist
    from paper_1202_4748_gb300 import shard
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    systems = _systems()
    mine = shard.partition(systems, world)[rank]
    local = {k: _run_one(systems[k]) for k in mine}
    res = shard.gather(local, len(systems))
    if rank == 0:
        np.save(os.path.join(outdir, "acc.npy"), np.stack([r["acc"][-1] for r in res]))
        np.save(os.path.join(outdir, "fsum.npy"), np.concatenate([r["f_sum"].ravel() for r in res]))
    dist.barrier()
    dist.destroy_process_group()


def test_partition_balances_and_covers():
    from paper_1202_4748_gb300 import shard
    systems = synth.ensemble("fss_160", "D3Q19")
    for world in (1, 2, 3, 8):
        parts = shard.partition(systems, world)
        assert sorted(k for p in parts for k in p) == list(range(len(systems)))
        loads = [sum(systems[k]["nx"] ** 3 for k in p) for p in parts]
        assert max(loads) - min(loads) <= 64 ** 3


def test_two_ranks_equal_one_process(tmp_path):
    import torch.multiprocessing as mp
    port = _free_port()
    mp.spawn(_worker, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    acc = np.load(os.path.join(tmp_path, "acc.npy"))
    fsum = np.load(os.path.join(tmp_path, "fsum.npy"))
    ref = [_run_one(s) for s in _systems()]
    assert np.array_equal(acc, np.stack([r["acc"][-1] for r in ref]))
    assert np.array_equal(fsum, np.concatenate([r["f_sum"].ravel() for r in ref]))


def _failing_worker(rank, world, port, outdir):
    import datetime
    import time
    import torch.distributed as dist
    from paper_1202_4748_gb300 import shard
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=10))
    systems = _systems()
    mine = shard.partition(systems, world)[rank]
    if rank == 1:
        os._exit(3)                       # leaves between steps, no collective in flight
    local = {k: _run_one(systems[k], steps=4) for k in mine}
    t0 = time.time()
    try:
        shard.gather(local, len(systems))
        outcome = "completed"
    except Exception as exc:              # the survivor must see an error, not hang
        outcome = type(exc).__name__
    with open(os.path.join(outdir, "rank0.txt"), "w") as fh:
        fh.write("%s %.2f" % (outcome, time.time() - t0))


def test_a_rank_that_leaves_makes_the_gather_fail_not_hang(tmp_path):
    """Failure detection on the host: when one rank exits before the final
    gather, the surviving rank's gather ends with an error within the process
    group's 10 s timeout instead of waiting forever."""
    import multiprocessing
    ctx = multiprocessing.get_context("spawn")
    port = _free_port()
    procs = [ctx.Process(target=_failing_worker, args=(r, 2, port, str(tmp_path))) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    alive = [p for p in procs if p.is_alive()]
    for p in alive:
        p.kill()
    assert not alive, "a rank hung"
    assert procs[1].exitcode == 3
    outcome, secs = open(os.path.join(tmp_path, "rank0.txt")).read().split()
    assert outcome != "completed"
    assert float(secs) < 60.0
