"""Sample sharding across ranks (CPU, gloo, world size 2): each rank holds a disjoint
shard of one ensemble's realisations; the merged per-dof statistics equal the two-pass
statistics of the whole ensemble computed in one place (the FP64 oracle). The second test
steps each rank's shard with the oracle, from fields the rank draws itself as its slice of
the seeded ensemble, as the multi-GPU benchmark does."""
import os
import socket

import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, u_all, bounds, out_path):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2101_09059_gb300.ensemble import sharded_stats
    lo, hi = bounds[rank], bounds[rank + 1]
    shard = u_all[lo:hi]
    mean = shard.mean(axis=0)
    var = shard.var(axis=0, ddof=1) if shard.shape[0] > 1 else np.zeros_like(mean)
    m, v = sharded_stats(shard.shape[0], mean, var)
    np.save(out_path + f".{rank}.npy", np.stack([m, v]))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("bounds", [[0, 13, 33], [0, 1, 33]])
def test_two_rank_merge_equals_whole_ensemble(tmp_path, bounds):
    rng = np.random.default_rng(4)
    u = 1e-3 + 1e-5 * rng.standard_normal((33, 50, 3))
    path = str(tmp_path / "out")
    mp.start_processes(_worker, args=(2, _free_port(), u, bounds, path), nprocs=2, join=True,
                       start_method="spawn")
    ref_m, ref_v = oracle.stats(u)
    for r in range(2):
        m, v = np.load(path + f".{r}.npy")
        assert np.allclose(m, ref_m, rtol=1e-13, atol=0)
        assert np.allclose(v, ref_v, rtol=1e-10, atol=0)


def test_merge_handles_empty_and_single_shards():
    from paper_2101_09059_gb300.ensemble import merge_stats
    rng = np.random.default_rng(1)
    u = rng.standard_normal((7, 4))
    parts = [(0, np.zeros(4), np.zeros(4)), (1, u[0], np.zeros(4)), (6, u[1:].mean(0), u[1:].var(0, ddof=1))]
    m, v = merge_stats(parts)
    assert np.allclose(m, u.mean(0), rtol=1e-14) and np.allclose(v, u.var(0, ddof=1), rtol=1e-12)


def _stepping_worker(rank, world, port, bounds, n, out_path):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import synth
    from paper_2101_09059_gb300.ensemble import sharded_stats
    lo, hi = bounds[rank], bounds[rank + 1]
    case = synth.make_case("tube_small", S=hi - lo, seed=7, n_steps=n, sample0=lo)
    # one ensemble, one time step: the CFL step of the stiffest realisation of any shard
    dt = torch.tensor([case["dt"]], dtype=torch.float64)
    dist.all_reduce(dt, op=dist.ReduceOp.MIN)
    case["dt"] = float(dt.item())
    u = oracle.Model(case).run(n)[0]                 # [S_shard][N][3]
    mean, var = oracle.stats(u)
    m, v = sharded_stats(u.shape[0], mean, var)
    np.save(out_path + f".{rank}.npy", np.stack([m, v]))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_stepped_shards_merge_to_the_whole_ensemble(tmp_path):
    import synth
    n, bounds = 60, [0, 3, 7]
    path = str(tmp_path / "step")
    mp.start_processes(_stepping_worker, args=(2, _free_port(), bounds, n, path), nprocs=2, join=True,
                       start_method="spawn")
    whole = synth.make_case("tube_small", S=7, seed=7, n_steps=n)
    ref_m, ref_v = oracle.stats(oracle.Model(whole).run(n)[0])
    for r in range(2):
        m, v = np.load(path + f".{r}.npy")
        assert np.abs(m - ref_m).max() <= 1e-12 * np.abs(ref_m).max()
        assert np.abs(v - ref_v).max() <= 1e-10 * np.abs(ref_v).max()
