"""World-size-2 host logic on the CPU (gloo): photon-range sharding and the
integer tally sum reproduce a single-process run bit for bit; the step time
is the maximum over ranks."""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2604_13929_gb300 import shard


def test_photon_ranges_partition_the_ids():
    for world in (1, 2, 3, 8):
        for n in (0, 1, 7, 100, 1001):
            got = [shard.photon_range(r, world, n) for r in range(world)]
            ids = [i for f, c in got for i in range(f, f + c)]
            assert ids == list(range(n))
    with pytest.raises(ValueError):
        shard.photon_range(2, 2, 10)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, n_total, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from oracle import oracle as orc
    from paper_2604_13929_gb300 import inputs
    mask = inputs.random_mask((12, 10, 8), 0.6, 2)
    first, count = shard.photon_range(rank, world, n_total)
    r = orc.run(mask, 0.6, 0.02, 0.7, count, 5, pid_begin=first, n_threads=1)
    field, R, T, A, depth = shard.allreduce_u64([r["field"], r["R"], r["T"], r["A"], r["depth"]],
                                               dist)
    t = shard.max_over_ranks(float(rank + 1), dist)
    if rank == 0:
        np.savez(os.path.join(out_dir, "merged.npz"), field=field, R=R, T=T, A=A, depth=depth,
                 t=t)
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_sum_to_one_run(tmp_path):
    n_total = 3001
    port = _free_port()
    mp.start_processes(_worker, args=(2, port, n_total, str(tmp_path)), nprocs=2,
                       start_method="spawn")
    m = np.load(tmp_path / "merged.npz")
    from oracle import oracle as orc
    from paper_2604_13929_gb300 import inputs
    mask = inputs.random_mask((12, 10, 8), 0.6, 2)
    ref = orc.run(mask, 0.6, 0.02, 0.7, n_total, 5, n_threads=1)
    for k in ("field", "R", "T", "A", "depth"):
        assert np.array_equal(m[k], ref[k]), k
    assert float(m["t"]) == 2.0
