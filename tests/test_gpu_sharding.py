"""Two ranks (processes, gloo) each solve their own block of global paths through the
library on the same GPU, as the bench's replicas do on separate GPUs: the context's
path offset keys every Brownian path by its global index, so the concatenated rank
results equal one process's solve of all paths bit for bit.  The ranks never wait on
each other's kernels: the only cross-rank operations are the host-side barrier and
the max-over-ranks timing reduction."""
import os
import socket

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as tmp  # noqa: E402

from workloads import LANGEVIN_TRIG_128, path_range  # noqa: E402

PATHS = 301          # not divisible by the world size: ranks own 151 and 150 paths
WORLD = 2


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _workload():
    return LANGEVIN_TRIG_128.with_(d=64, n_fine=1024, paths=PATHS)


def _worker(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import paper_2207_09776_b300 as msk
    msk.load_library()
    a, b = path_range(PATHS, rank, world)
    w = _workload().with_(path_offset=a, paths=b - a)
    s = msk.Solver(w, device=0)
    u32, st = s.magnus(3, 8, precision=msk.MSK_F32, status=True)
    u64 = s.magnus(3, 8, precision=msk.MSK_F64)
    torch.cuda.synchronize()
    np.save(os.path.join(out_dir, f"f32_{rank}.npy"), u32.cpu().numpy())
    np.save(os.path.join(out_dir, f"f64_{rank}.npy"), u64.cpu().numpy())
    np.save(os.path.join(out_dir, f"st_{rank}.npy"), st[: b - a].cpu().numpy())
    t = torch.tensor([float(rank + 1)])
    dist.barrier()
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    np.save(os.path.join(out_dir, f"tmax_{rank}.npy"), t.numpy())
    s.close()
    dist.destroy_process_group()


def test_rank_path_blocks_through_the_library_equal_one_process(tmp_path):
    from paper_2207_09776_b300 import build
    build.build()
    tmp.spawn(_worker, args=(WORLD, _free_port(), str(tmp_path)), nprocs=WORLD, join=True)
    import paper_2207_09776_b300 as msk
    msk.load_library()
    s = msk.Solver(_workload())
    full32 = s.magnus(3, 8, precision=msk.MSK_F32).cpu().numpy()
    full64 = s.magnus(3, 8, precision=msk.MSK_F64).cpu().numpy()
    s.close()
    got32 = np.concatenate([np.load(tmp_path / f"f32_{r}.npy") for r in range(WORLD)])
    got64 = np.concatenate([np.load(tmp_path / f"f64_{r}.npy") for r in range(WORLD)])
    np.testing.assert_array_equal(got32, full32)
    np.testing.assert_array_equal(got64, full64)
    assert all(int(np.load(tmp_path / f"st_{r}.npy").max()) == 0 for r in range(WORLD))
    assert all(float(np.load(tmp_path / f"tmax_{r}.npy")[0]) == float(WORLD) for r in range(WORLD))
