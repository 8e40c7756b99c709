"""Multi-process host logic on CPU (gloo, world size 2).

bench.py under torchrun runs one independent replica per rank and rank 0
reports the maximum time over ranks: the barrier, the max-over-ranks
reduction and the reference arm's rank-0-only output are tested here.  A
sharded run (paper_2008_09441_gb300.shard) splits one run's particles over
the ranks and sums the regular-grid density over them once per step: the
partition and that sum are tested here too, without a GPU.
"""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _max_worker(rank, world, port, out_dir):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    bench.barrier(dist)
    m = bench.max_over_ranks(dist, float(10 * rank + 1))
    with open(os.path.join(out_dir, f"r{rank}.txt"), "w") as f:
        f.write(repr(m))
    dist.destroy_process_group()


def test_max_over_ranks_gloo(tmp_path):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    world = 2
    mp.start_processes(_max_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, start_method="spawn")
    for r in range(world):
        assert float(open(tmp_path / f"r{r}.txt").read()) == 11.0


def test_reference_arm_two_ranks():
    pytest.importorskip("torch")
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()), "bench.py", "--impl", "reference",
           "--gpus", "2", "--steps", "1", "--warmup", "3", "--ref-particles", "2048", "--ref-budget-s", "30"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout  # rank 0 alone prints
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["cpu_baseline"]["kind"] == "oracle"
    # the line keeps the contract's keys; the oracle ran on one BLAS thread
    assert d["unit"] == "particle-steps/s" and d["higher_is_better"] is True and d["metric"]
    assert d["cpu_baseline"]["cores"] == 1 and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["value"] == d["value"] and d["e2e"]["unit"] == d["unit"]


# ------------------------------------------------------------ particle sharding (host side)


def _fixed_point_deposit(u, q, n, scale):
    """CIC deposit of every particle onto the level-n regular grid in integer
    fixed point: each corner contribution rounded once to 1/scale, sums in
    int64 (the accumulation the deposit window uses, so that sums do not
    depend on their order)."""
    import numpy as np
    N = 1 << n
    d = u.shape[1]
    grid = np.zeros((N,) * d, dtype=np.int64)
    s = u * N
    c = np.floor(s).astype(np.int64)
    f = s - c
    for corner in range(1 << d):
        w = q.copy()
        idx = []
        for m in range(d):
            b = (corner >> m) & 1
            w = w * (f[:, m] if b else 1.0 - f[:, m])
            idx.append((c[:, m] + b) % N)
        np.add.at(grid, tuple(idx), np.rint(w * scale).astype(np.int64))
    return grid


def _shard_worker(rank, world, port, out_dir):
    import numpy as np
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    from paper_2008_09441_gb300 import shard, workloads
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    wl = workloads.landau2d(n_particles=20011, n=6, seed=77)
    lo, hi = shard.partition(len(wl.q), world, rank)
    scale = float(1 << 40)
    part = _fixed_point_deposit(wl.u[lo:hi], wl.q[lo:hi], wl.n, scale)
    t = torch.from_numpy(part.copy())
    shard.sum_over_ranks(t)  # the exchange step of a sharded run
    ranges = torch.tensor([lo, hi], dtype=torch.int64)
    gathered = [torch.zeros(2, dtype=torch.int64) for _ in range(world)]
    dist.all_gather(gathered, ranges)
    np.save(os.path.join(out_dir, f"arena{rank}.npy"), t.numpy())
    np.save(os.path.join(out_dir, f"ranges{rank}.npy"), torch.stack(gathered).numpy())
    dist.destroy_process_group()


def test_sharded_density_exchange_gloo(tmp_path):
    """World size 2 (gloo): the ranks' index ranges tile the particles, and
    the sum over the ranks of their fixed-point regular-grid deposits is the
    single-rank deposit of all particles, bit for bit."""
    torch = pytest.importorskip("torch")
    import numpy as np
    import torch.multiprocessing as mp
    sys.path.insert(0, ROOT)
    from paper_2008_09441_gb300 import workloads
    world = 2
    mp.start_processes(_shard_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, start_method="spawn")
    wl = workloads.landau2d(n_particles=20011, n=6, seed=77)
    whole = _fixed_point_deposit(wl.u, wl.q, wl.n, float(1 << 40))
    for r in range(world):
        arena = np.load(tmp_path / f"arena{r}.npy")
        assert np.array_equal(arena, whole)
        rg = np.load(tmp_path / f"ranges{r}.npy")
        assert rg[0, 0] == 0 and rg[-1, 1] == len(wl.q)
        assert all(rg[i, 1] == rg[i + 1, 0] for i in range(world - 1))


def test_partition_tiles_the_particles():
    sys.path.insert(0, ROOT)
    from paper_2008_09441_gb300 import shard
    for n in (0, 1, 7, 1000, 4194304):
        for world in (1, 2, 3, 8):
            ranges = [shard.partition(n, world, r) for r in range(world)]
            assert ranges[0][0] == 0 and ranges[-1][1] == n
            assert all(ranges[i][1] == ranges[i + 1][0] for i in range(world - 1))
            sizes = [b - a for a, b in ranges]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        shard.partition(10, 2, 2)
