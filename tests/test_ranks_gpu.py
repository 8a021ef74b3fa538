"""The library itself under ensemble sharding: two ranks (gloo, one process
each, both on cuda:0) advance their partition() shares of a small D3Q19
ensemble through lb.Ensemble and gather the results; the gathered
observables and populations must equal a single-process run of the whole
ensemble bit for bit.  A system's trajectory depends only on its own
descriptor (the noise is keyed by site, step and system_id), not on which
rank or batch advances it; the ranks share no device memory and none of
their kernels waits on the other's (the only exchange is the host gather)."""
import os
import socket

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

FIELDS = ("n", "sum_m", "sum_m2", "sum_abs_m", "sum_m4", "sum_e", "sum_e2")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _systems():
    shapes = [(16, 16, 16), (12, 8, 20), (24, 24, 8), (8, 8, 8), (20, 12, 12), (32, 16, 8)]
    out = []
    for k, (nx, ny, nz) in enumerate(shapes):
        s = synth.system("D3Q19", "guo", n=nx, a=-0.002 + 0.001 * k, kT=1e-4, seed=1 + k % 3, system_id=k)
        s.update(nx=nx, ny=ny, nz=nz)
        out.append(s)
    return out


def _advance(lb, systems, precision, steps=20, every=5):
    res = {}
    if not systems:
        return res
    ens = lb.Ensemble([s for _, s in systems], precision=precision, obs_every=every)
    ens.init(amplitude=0.01)
    ens.step(steps)
    for i, (k, _) in enumerate(systems):
        levels, glob = ens.observables(i)
        res[k] = {"obs": np.array([[lv[f] for f in FIELDS] for lv in levels]),
                  "mass": np.array([glob["mass0"], glob["mass"]]), "f": ens.read_fields(i)}
    ens.close()
    return res


def _worker(rank, world, port, outdir, precision):
    import torch
    import torch.distributed as dist
    import paper_1202_4748_gb300 as lb
    from paper_1202_4748_gb300 import shard
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    torch.cuda.set_device(0)
    systems = _systems()
    mine = shard.partition(systems, world)[rank]
    res = shard.gather(_advance(lb, [(k, systems[k]) for k in mine], precision), len(systems))
    if rank == 0:
        np.savez(os.path.join(outdir, "gathered.npz"),
                 **{"%s_%d" % (name, k): r[name] for k, r in enumerate(res) for name in ("obs", "mass", "f")})
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_two_ranks_of_the_library_equal_one_process(tmp_path, precision):
    import torch.multiprocessing as mp
    import paper_1202_4748_gb300 as lb
    from paper_1202_4748_gb300 import shard
    systems = _systems()
    parts = shard.partition(systems, 2)
    assert all(parts) and sorted(parts[0] + parts[1]) == list(range(len(systems)))
    mp.spawn(_worker, args=(2, _free_port(), str(tmp_path), precision), nprocs=2, join=True)
    got = np.load(os.path.join(tmp_path, "gathered.npz"))
    ref = _advance(lb, list(enumerate(systems)), precision)
    for k in range(len(systems)):
        for name in ("obs", "mass", "f"):
            assert np.array_equal(got["%s_%d" % (name, k)], ref[k][name]), (k, name)
