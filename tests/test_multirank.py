"""The multi-process path of bench.py on CPU: two gloo ranks, each with its own
seeded stream (oracle on a tiny table), combined by the bench's reduction."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_main(rank, world, port, out):
    import sys
    import torch.distributed as dist
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from oracle import ct_oracle as O
    from paper_2507_18413_gb300 import inputs as G
    seed = bench.rank_seed(7, rank)
    dom_lo, dom_size, tup = G.tiny_table(seed=seed)
    tup = O.retained_tuples(tup, dom_lo, dom_size)
    rng = G.Rng(seed)
    masks = [np.ones(d, bool) for d in dom_size]
    props = 0
    for k in range(20 + 5 * rank):
        new, _ = G.remove_random_values(rng, masks, 1)
        st, out_m, _ = O.gac_table(tup, dom_lo, new)
        props += 1
        masks = out_m if st == O.OK else [np.ones(d, bool) for d in dom_size]
    ms = 10.0 + rank
    tmax, psum = bench.reduce_over_ranks(ms, props, world, "cpu")
    out[rank] = (tmax, psum, int(tup.sum()))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_reduce_like_the_bench():
    world = 2
    ctx = mp.get_context("spawn")
    manager = ctx.Manager()
    out = manager.dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    assert out[0][0] == out[1][0] == 11.0          # slowest rank's time
    assert out[0][1] == out[1][1] == 20 + 25       # propagations of all ranks
    assert out[0][2] != out[1][2]                  # each rank has its own stream


def test_single_rank_reduction_is_identity():
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    assert bench.reduce_over_ranks(3.5, 7, 1, "cpu") == (3.5, 7.0)
    assert bench.rank_seed(5, 0) != bench.rank_seed(5, 1)
