"""Multi-rank host logic on CPU with two gloo ranks: the bench's
max-over-ranks timing reduction and the assembly of a sharded Fock matrix from
per-rank partial J and K (the paper's ddi_gsumf step)."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out_dir):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from paper_1708_00033_gb300.hf import assemble_shards
    m = bench.reduce_max(10.0 + 5.0 * rank, dist, torch.device("cpu"))
    rng = np.random.default_rng(100 + rank)
    N = 12
    Jp, Kp = rng.standard_normal((N, N)), rng.standard_normal((N, N))
    H = np.eye(N)

    def allsum(a):
        t = torch.from_numpy(np.array(a, copy=True))
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
        return t.numpy()

    F, J, K = assemble_shards(H, Jp, Kp, allsum)
    np.savez(os.path.join(out_dir, f"rank{rank}.npz"), m=m, F=F, J=J, K=K, Jp=Jp, Kp=Kp)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks(tmp_path):
    import torch.multiprocessing as mp
    world = 2
    mp.spawn(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    r = [np.load(tmp_path / f"rank{k}.npz") for k in range(world)]
    assert float(r[0]["m"]) == 15.0 and float(r[1]["m"]) == 15.0
    J = r[0]["Jp"] + r[1]["Jp"]
    K = r[0]["Kp"] + r[1]["Kp"]
    for k in range(world):
        assert np.allclose(r[k]["J"], J, atol=1e-14) and np.allclose(r[k]["K"], K, atol=1e-14)
        assert np.allclose(r[k]["F"], np.eye(12) + J - 0.5 * K, atol=1e-14)
