"""Multi-rank path sharding on CPU (gloo, world size 2).

Paths are independent and keyed by their global index, so N ranks run
replicas over disjoint path ranges with no collective on the data path; the
only cross-rank operations are the barrier and the max-over-ranks timing
reduction that bench.py performs.  Checked here with the oracle as the
per-rank solver."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as tmp

from workloads import LANGEVIN_32, path_range


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from oracle import magnus
    w = LANGEVIN_32.with_(d=8, ax=-3.0, bx=3.0, av=-3.0, bv=3.0, n_fine=64, paths=3)
    # weak scaling: rank r owns global paths [r P, (r+1) P)
    wr = w.with_(path_offset=rank * w.paths)
    U = magnus.solve(wr, 2, 4)
    np.save(os.path.join(out_dir, f"rank{rank}.npy"), U)
    # barrier + max-over-ranks of the elapsed time
    t = torch.tensor([float(rank + 1)])
    dist.barrier()
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    np.save(os.path.join(out_dir, f"tmax{rank}.npy"), t.numpy())
    dist.destroy_process_group()


def test_two_rank_replicas_match_one_process(tmp_path):
    world = 2
    tmp.spawn(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    from oracle import magnus
    w = LANGEVIN_32.with_(d=8, ax=-3.0, bx=3.0, av=-3.0, bv=3.0, n_fine=64, paths=6)
    full = magnus.solve(w, 2, 4)
    got = np.concatenate([np.load(tmp_path / f"rank{r}.npy") for r in range(world)])
    np.testing.assert_array_equal(got, full)
    for r in range(world):
        assert float(np.load(tmp_path / f"tmax{r}.npy")[0]) == 2.0


@pytest.mark.parametrize("paths,world", [(10, 3), (4096, 8), (1, 2), (0, 4)])
def test_path_ranges_partition(paths, world):
    seen = []
    for r in range(world):
        a, b = path_range(paths, r, world)
        assert 0 <= a <= b <= paths
        seen.extend(range(a, b))
    assert seen == list(range(paths))
