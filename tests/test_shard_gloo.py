"""Chains split over two processes (gloo, CPU): each rank runs its own chain
range with the FP64 oracle, and the resolve over both ranks equals one run of
all the chains.  Checks the range split and the reduction used on GPUs
(paper_2409_07148_gb300/shard.py)."""
import os
import socket

import numpy as np
import pytest

from paper_2409_07148_gb300 import shard


def test_chain_range_covers_every_chain_once():
    for n, w in ((10, 3), (1 << 20, 8), (7, 7), (1000, 1)):
        got = [shard.chain_range(r, w, n) for r in range(w)]
        ids = np.concatenate([np.arange(a, a + c) for a, c in got])
        assert np.array_equal(ids, np.arange(n))
        assert max(c for _, c in got) - min(c for _, c in got) <= 1
    with pytest.raises(ValueError):
        shard.chain_range(2, 2, 10)
    with pytest.raises(ValueError):
        shard.chain_range(0, 4, 3)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, n_total, steps, out_dir):
    import torch
    import torch.distributed as dist
    from oracle import oracle as O
    from paper_2409_07148_gb300 import scenes
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sc = scenes.cornell(width=16, height=16, depth=2)
    first, count = shard.chain_range(rank, world, n_total)
    ch = O.Chains(O.Scene(sc), sc.D, sc.width, sc.height, seed=11, chain_begin=first, n_chains=count)
    ch.advance(steps)
    img, J = shard.resolve_all(torch.from_numpy(ch.accum.copy()), ch.J)
    if rank == 0:
        np.save(os.path.join(out_dir, "img.npy"), img.numpy())
        np.save(os.path.join(out_dir, "J.npy"), np.array([J]))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_resolve_to_the_single_run(tmp_path):
    import torch.multiprocessing as mp
    from oracle import oracle as O
    from paper_2409_07148_gb300 import scenes
    n_total, steps = 96, 40
    mp.start_processes(_rank, args=(2, _free_port(), n_total, steps, str(tmp_path)), nprocs=2, join=True,
                       start_method="spawn")
    img = np.load(tmp_path / "img.npy")
    J = int(np.load(tmp_path / "J.npy")[0])
    sc = scenes.cornell(width=16, height=16, depth=2)
    one = O.Chains(O.Scene(sc), sc.D, sc.width, sc.height, seed=11, chain_begin=0, n_chains=n_total)
    one.advance(steps)
    assert J == one.J and J > 0
    ref = one.accum[:, :, :3] / one.J
    assert np.abs(img - ref).max() <= 1e-12 * max(1.0, np.abs(ref).max())
