"""The N > 1 path on the host: two ranks (gloo, CPU) split the trajectories, gather their
per-trajectory moments and form the ensemble; the result equals the one-process ensemble
of the same trajectories, and the oracle's ensemble formulas."""
import os
import socket
import tempfile

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import synth  # noqa: E402
from oracle.observables import ensemble as oracle_ensemble  # noqa: E402


def _moments_of(global_ids, n_meas, n):
    """Synthetic per-trajectory moments keyed by the global trajectory id (as the library's
    counter-based draws are): |m| < 1, q a valid second-moment table."""
    out = np.zeros((n_meas, len(global_ids), 9))
    for k, gid in enumerate(global_ids):
        g = synth.rng(1000 + int(gid))
        m = g.uniform(-0.8, 0.8, (n_meas, 3))
        q = g.uniform(-0.2, 0.2, (n_meas, 6))
        q[:, :3] = np.abs(q[:, :3]) + 1.0 / n
        out[:, k, :3], out[:, k, 3:] = m, q
    return out


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, ntraj, n_meas, n, outdir):
    import torch.distributed as dist
    from paper_2506_23928_gb300 import sharding
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        traj0, count = sharding.shard(ntraj, rank, world)
        local = _moments_of(range(traj0, traj0 + count), n_meas, n)
        full = sharding.gather_moments(local, ntraj)
        rows = [sharding.ensemble(full[i], n) for i in range(n_meas)]
        slowest = sharding.max_over_ranks(1.5 + rank)
        np.savez(os.path.join(outdir, f"rank{rank}.npz"), full=full, M=np.array([r[0] for r in rows]),
                 C=np.array([r[1] for r in rows]), xi2=np.array([r[2] for r in rows]),
                 dM=np.array([r[3] for r in rows]), slowest=slowest, traj0=traj0, count=count)
    finally:
        dist.destroy_process_group()


@pytest.fixture(scope="module")
def lib():
    from paper_2506_23928_gb300 import build
    build.build()


@pytest.mark.parametrize("ntraj", [10, 7])
def test_two_ranks_gather_and_ensemble(lib, ntraj):
    import torch.multiprocessing as mp
    world, n_meas, n = 2, 3, 12
    with tempfile.TemporaryDirectory() as d:
        mp.start_processes(_worker, args=(world, _free_port(), ntraj, n_meas, n, d), nprocs=world, join=True,
                           start_method="spawn")
        res = [dict(np.load(os.path.join(d, f"rank{r}.npz"))) for r in range(world)]
    want = _moments_of(range(ntraj), n_meas, n)
    # shards cover the trajectories once, in order
    assert [int(r["traj0"]) for r in res] == [0, (ntraj + 1) // 2]
    assert sum(int(r["count"]) for r in res) == ntraj
    from paper_2506_23928_gb300 import sharding
    for r in res:
        assert np.array_equal(r["full"], want)
        assert float(r["slowest"]) == 2.5
        for i in range(n_meas):
            M, C, xi2, dM = sharding.ensemble(want[i], n)
            assert np.array_equal(r["M"][i], M) and np.array_equal(r["C"][i], C)
            assert r["xi2"][i] == xi2 and np.array_equal(r["dM"][i], dM)
            # and the oracle's ensemble formulas on the same moments
            m = want[i, :, :3]
            q = np.zeros((ntraj, 3, 3))
            for (a, b), col in zip([(0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2)], range(3, 9)):
                q[:, a, b] = q[:, b, a] = want[i, :, col]
            M0, C0, dM0 = oracle_ensemble(m, q)
            assert np.allclose(M, M0, rtol=0, atol=1e-14) and np.allclose(C, C0, rtol=0, atol=1e-14)


def test_shard_sizes():
    from paper_2506_23928_gb300.sharding import shard
    for total in (0, 1, 5, 256, 1001):
        for world in (1, 2, 3, 8):
            spans = [shard(total, r, world) for r in range(world)]
            assert spans[0][0] == 0
            for (a0, c0), (a1, _) in zip(spans, spans[1:]):
                assert a0 + c0 == a1
            assert sum(c for _, c in spans) == total
            assert max(c for _, c in spans) - min(c for _, c in spans) <= 1
    with pytest.raises(ValueError):
        shard(4, 2, 2)
