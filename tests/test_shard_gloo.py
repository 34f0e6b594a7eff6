"""Host-side multi-rank logic on CPU: world_size 2 over gloo.

Each rank walks its contiguous range of instances with the FP64 oracle
under the instances' global numbers (the GPU path takes the same numbers);
the gathered result must equal a single-process walk of the whole batch,
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


def _worker(rank, world, port, out_path):
    import torch
    import torch.distributed as dist
    import oracle
    from paper_2606_27604_b300 import inputs
    from paper_2606_27604_b300.shard import gather_instances, max_over_ranks, shard_range
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    x = inputs.uneven_batch(n_inst=9, param_seed=4, log2_min=8, log2_max=10)
    b, e = shard_range(x.n_inst, rank, world)
    xs = x.subset(np.arange(b, e))
    r = oracle.walk(xs.alpha, xs.sigma_t, xs.g, xs.w, xs.n_paths, xs.thickness_mm, x.n_rel,
                    oracle.OracleOpts(nbins=16, seed=3), inst_ids=np.arange(b, e))
    local = torch.from_numpy(np.concatenate([r["R"][:, None], r["bins"]], axis=1))
    full = gather_instances(local, x.n_inst)
    t = max_over_ranks(float(rank + 1))
    if rank == 0:
        np.save(out_path, full.numpy())
        np.save(out_path + ".t.npy", np.array([t]))
    dist.destroy_process_group()


def test_two_rank_walk_equals_single_process(tmp_path):
    import torch.multiprocessing as mp
    import oracle
    from paper_2606_27604_b300 import inputs
    out = str(tmp_path / "full.npy")
    mp.start_processes(_worker, args=(2, _free_port(), out), nprocs=2, join=True,
                       start_method="spawn")
    got = np.load(out)
    x = inputs.uneven_batch(n_inst=9, param_seed=4, log2_min=8, log2_max=10)
    r = oracle.walk(x.alpha, x.sigma_t, x.g, x.w, x.n_paths, x.thickness_mm, x.n_rel,
                    oracle.OracleOpts(nbins=16, seed=3))
    np.testing.assert_array_equal(got, np.concatenate([r["R"][:, None], r["bins"]], axis=1))
    assert np.load(out + ".t.npy")[0] == 2.0
