"""Walker sharding and the one cross-rank reduction, on CPU ranks (gloo,
world size 2).  The multi-rank path is covered on the host: the data path
has no collective to emulate."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2504_06087_gb300 import replicas


def test_walker_blocks_partition_the_range():
    for total in (0, 1, 7, 4096, 4099):
        for world in (1, 2, 3, 8):
            blocks = [replicas.walker_block(total, r, world) for r in range(world)]
            assert blocks[0][0] == 0
            for (s0, c0), (s1, _) in zip(blocks, blocks[1:]):
                assert s0 + c0 == s1
            assert sum(c for _, c in blocks) == total
            assert max(c for _, c in blocks) - min(c for _, c in blocks) <= 1
    with pytest.raises(ValueError):
        replicas.walker_block(10, 2, 2)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, e_all, out_q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        start, cnt = replicas.walker_block(len(e_all), rank, world)
        mom = replicas.energy_moments(torch.as_tensor(e_all[start:start + cnt]))
        out_q.put((rank, mom))
    finally:
        dist.destroy_process_group()


def test_energy_moments_all_reduce_over_two_ranks():
    rng = np.random.default_rng(3)
    e = rng.normal(-300.0, 2.0, size=1001)
    e[[5, 600]] = np.nan                          # walkers on a node
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, e, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    ok = np.isfinite(e)
    for r in (0, 1):
        m = res[r]
        assert m["n"] == ok.sum() and m["n_nonfinite"] == 2
        np.testing.assert_allclose(m["mean"], e[ok].mean(), rtol=1e-14)
        np.testing.assert_allclose(m["variance"], e[ok].var(), rtol=1e-9)


def test_moments_without_a_process_group_are_local():
    e = torch.tensor([1.0, 2.0, float("nan"), 4.0])
    m = replicas.energy_moments(e)
    assert m["n"] == 3 and m["n_nonfinite"] == 1
    np.testing.assert_allclose(m["mean"], 7.0 / 3.0)
