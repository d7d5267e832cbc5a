"""Energy sharding across processes (world size 2, gloo on CPU): every energy is owned exactly once,
and the per-rank partial integrals summed by one all-reduce equal the single-process integral."""
import os
import socket

import numpy as np

from paper_1702_05167_gb300 import sharding


def test_shards_partition_the_grid():
    for n, R in ((64, 1), (64, 2), (65, 4), (3, 8)):
        owned = np.concatenate([sharding.shard(n, r, R) for r in range(R)])
        assert sorted(owned.tolist()) == list(range(n))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    E = np.linspace(-5.5, 5.5, 64)
    f = np.stack([np.exp(-E ** 2), np.cos(E) ** 2], axis=1)      # stand-ins for T(E), sum Im G^<
    own = sharding.shard(len(E), rank, world)
    part = sharding.partial_integral(E, f[own], own)
    tot = sharding.allreduce_sum(part)
    q.put((rank, tot.tolist(), len(own)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_allreduce_matches_serial():
    import torch.multiprocessing as mp
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
    E = np.linspace(-5.5, 5.5, 64)
    f = np.stack([np.exp(-E ** 2), np.cos(E) ** 2], axis=1)
    trap = getattr(np, "trapezoid", None) or np.trapz
    serial = np.array([trap(f[:, 0], E), trap(f[:, 1], E)])
    assert sum(n for _, _, n in res) == 64
    for _, tot, _ in res:
        np.testing.assert_allclose(tot, serial, rtol=1e-13)


def test_interleaved_grids_are_disjoint():
    E = np.linspace(-6, 6, 32)
    g = [sharding.interleaved_grid(E, r, 4) for r in range(4)]
    allE = np.concatenate(g)
    assert len(np.unique(np.round(allE, 12))) == 128


def test_a_one_energy_grid_is_not_shifted():
    E = np.array([0.25])
    for r in range(3):
        assert np.array_equal(sharding.interleaved_grid(E, r, 3), E)
