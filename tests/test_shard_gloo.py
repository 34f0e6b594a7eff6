"""Host-side multi-rank logic on CPU: world_size 2 over gloo.

The ranks run the benchmark's own shard, walk and gather functions
(paper_2606_27604_b300.shard), with the FP64 oracle as the walk, under the
instances' global numbers (the GPU path takes the same numbers):
  * strong sharding: one batch cut into contiguous instance ranges and one
    all_gather must equal a single-process walk of the batch, bit for bit;
  * weak sharding: each rank's own batch walked as its slice of a stacked
    global batch must equal a single-process walk of the stacked batch;
and the job time is the slowest rank's."""
import os
import socket

import numpy as np
import pytest

from paper_2606_27604_b300.shard import shard_range


def test_shard_ranges_cover_exactly():
    for n in (0, 1, 7, 100, 4096):
        for world in (1, 2, 3, 8):
            ranges = [shard_range(n, r, world) for r in range(world)]
            assert ranges[0][0] == 0 and ranges[-1][1] == n
            for (b0, e0), (b1, e1) in zip(ranges, ranges[1:]):
                assert e0 == b1
            sizes = [e - b for b, e in ranges]
            assert max(sizes) - min(sizes) <= 1


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _oracle_walk_fn(nbins=16, seed=3):
    """A walk function for walk_and_gather: the FP64 oracle on CPU, under the
    instances' global numbers, as the GPU walk takes them (instance_offset)."""
    import torch
    import oracle

    def fn(xs, begin):
        r = oracle.walk(xs.alpha, xs.sigma_t, xs.g, xs.w, xs.n_paths, xs.thickness_mm, xs.n_rel,
                        oracle.OracleOpts(nbins=nbins, seed=seed),
                        inst_ids=np.arange(begin, begin + xs.n_inst))
        return torch.from_numpy(r["R"]), torch.from_numpy(r["bins"])
    return fn


def _batch(seed=4):
    from paper_2606_27604_b300 import inputs
    return inputs.uneven_batch(n_inst=9, param_seed=seed, log2_min=8, log2_max=10)


def _worker(rank, world, port, out_path):
    # the shard, walk and gather steps of the benchmark's multi-GPU modes
    import torch.distributed as dist
    from paper_2606_27604_b300.shard import (gather_instances, max_over_ranks, shard_batch,
                                             walk_and_gather)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    fn = _oracle_walk_fn()
    # strong: one batch cut into contiguous instance ranges, one all_gather
    x = _batch()
    xs, begin = shard_batch(x, rank, world)
    full = walk_and_gather(fn, xs, begin, x.n_inst)
    # weak: every rank walks its own batch as instances rank*n .. rank*n + n - 1
    # of a global batch; no exchange during the walk (gathered here only to check)
    xw = _batch(seed=10 + rank)
    local = walk_and_gather(fn, xw, rank * xw.n_inst, xw.n_inst * world, gather=False)
    weak = gather_instances(local, xw.n_inst * world)
    t = max_over_ranks(float(rank + 1))
    if rank == 0:
        np.save(out_path, full.numpy())
        np.save(out_path + ".weak.npy", weak.numpy())
        np.save(out_path + ".t.npy", np.array([t]))
    dist.destroy_process_group()


def test_two_rank_walk_equals_single_process(tmp_path):
    import torch.multiprocessing as mp
    import oracle
    from paper_2606_27604_b300 import inputs
    out = str(tmp_path / "full.npy")
    mp.start_processes(_worker, args=(2, _free_port(), out), nprocs=2, join=True,
                       start_method="spawn")
    fn = _oracle_walk_fn()
    # strong sharding: the gathered table equals one process walking the batch
    x = _batch()
    R, bins = fn(x, 0)
    np.testing.assert_array_equal(np.load(out), np.concatenate([R[:, None], bins], axis=1))
    # weak sharding: equals one process walking the stacked batches
    xa, xb = _batch(seed=10), _batch(seed=11)
    stacked = inputs.WalkInputs(*(np.concatenate([getattr(xa, k), getattr(xb, k)], axis=-1)
                                  for k in ("alpha", "sigma_t", "g", "w", "n_paths",
                                            "thickness_mm")), n_rel=xa.n_rel)
    R, bins = fn(stacked, 0)
    np.testing.assert_array_equal(np.load(out + ".weak.npy"),
                                  np.concatenate([R[:, None], bins], axis=1))
    assert np.load(out + ".t.npy")[0] == 2.0
