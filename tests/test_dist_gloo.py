"""Multi-rank host logic (paper_2403_04252_gb300.dist) on CPU: two gloo ranks shard an impact-parameter
scan, reduce their timings to the maximum and gather per-path observables to rank 0, which must hold
the single-process scan (its cross sections are then formed by the library, tests/test_gpu_observables.py)."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

def _dist_module():
    # the package __init__ needs the built library; the helper module does not
    import importlib.util
    here = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    spec = importlib.util.spec_from_file_location("wpccc_dist", os.path.join(here, "paper_2403_04252_gb300", "dist.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


def _fake_observables(b):
    # smooth stand-in for per-path probabilities (capture-like and excitation-like)
    return np.stack([np.exp(-b) * (1 + b), 0.3 * np.exp(-0.5 * (b - 2.0) ** 2)], axis=1)


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    D = _dist_module()
    b = D.shard_impact_parameters(0.2, 12.0, 16, rank, world)
    t = D.max_over_ranks(1.0 + rank)            # the slowest rank's time
    bb, PP = D.gather_paths(b, _fake_observables(b))
    if rank == 0:
        out.put((t, bb, PP))
    dist.barrier()
    dist.destroy_process_group()


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def test_two_rank_shard_reduce_gather():
    world = 2
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    t, bb, PP = out.get(timeout=120)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    b_all = np.linspace(0.2, 12.0, 16 * world)
    assert t == float(world)                          # max over ranks
    assert np.array_equal(bb, b_all)                  # the union of the shards is the full scan
    assert np.allclose(PP, _fake_observables(b_all), rtol=0, atol=0)


def test_shards_are_disjoint_and_balanced():
    D = _dist_module()
    for world in (1, 2, 3, 8):
        parts = [D.shard_impact_parameters(0.2, 12.0, 32, r, world) for r in range(world)]
        assert all(p.size == 32 for p in parts)
        allb = np.sort(np.concatenate(parts))
        assert np.array_equal(allb, np.linspace(0.2, 12.0, 32 * world))
    with pytest.raises(ValueError):
        D.shard_impact_parameters(0.2, 12.0, 32, 2, 2)


def test_single_process_fallbacks():
    D = _dist_module()
    assert D.max_over_ranks(3.5) == 3.5
    b = np.array([3.0, 1.0, 2.0])
    bb, PP = D.gather_paths(b, np.array([[3.0], [1.0], [2.0]]))
    assert np.array_equal(bb, [1.0, 2.0, 3.0]) and np.array_equal(PP[:, 0], [1.0, 2.0, 3.0])
