"""Multi-rank host logic on CPU with two gloo ranks: the bench's
max-over-ranks timing reduction and the sharded Fock build's rank logic
(each rank's shard, one sum of J and one of K over the ranks - the paper's
ddi_gsumf step - and the assembly).  The library calls are replaced by
stand-ins here (no GPU); the GPU tests check the same calls on the device."""
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


N = 12


def _partial_stand_in(system, P, shard, n_shards):
    """Deterministic per-shard matrices standing in for hf_fock_build_partial."""
    rng = np.random.default_rng(100 + shard + 10 * n_shards)
    return rng.standard_normal((N, N)), rng.standard_normal((N, N))


def _assemble_stand_in(system, J, K, P=None, energy=False):
    F = np.eye(N) + J - 0.5 * K
    return F, (float(np.sum(P * (np.eye(N) + F))) / 2 if energy else None)


def _worker(rank, world, port, out_dir):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from paper_1708_00033_gb300 import hf
    m = bench.reduce_max(10.0 + 5.0 * rank, dist, torch.device("cpu"))

    def allsum(a):
        t = torch.from_numpy(np.array(a, copy=True))
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
        return t.numpy()

    P = np.full((N, N), 0.1)
    F, J, K, E = hf.sharded_fock_build(None, P, rank, world, allsum, energy=True, build_partial=_partial_stand_in,
                                       assemble=_assemble_stand_in)
    np.savez(os.path.join(out_dir, f"rank{rank}.npz"), m=m, F=F, J=J, K=K, E=E)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks(tmp_path):
    import torch.multiprocessing as mp
    world = 2
    mp.spawn(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    r = [np.load(tmp_path / f"rank{k}.npz") for k in range(world)]
    assert float(r[0]["m"]) == 15.0 and float(r[1]["m"]) == 15.0
    parts = [_partial_stand_in(None, None, k, world) for k in range(world)]
    J = parts[0][0] + parts[1][0]
    K = parts[0][1] + parts[1][1]
    for k in range(world):
        assert np.allclose(r[k]["J"], J, atol=1e-14) and np.allclose(r[k]["K"], K, atol=1e-14)
        assert np.allclose(r[k]["F"], np.eye(N) + J - 0.5 * K, atol=1e-14)
        assert abs(float(r[k]["E"]) - float(r[0]["E"])) == 0.0
