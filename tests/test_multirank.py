"""Multi-process paths under torch.distributed, on CPU with the gloo backend and two ranks:
the replica aggregation of bench.py (the job's time is the slowest rank's, its solves the sum over
ranks, on every rank), and frequency sharding of E_c (paper_2504_01816_gb300/shard.py): each rank
evaluates its range of the quadrature frequencies -- here with the oracle standing in for the
library, which needs a GPU -- and one all-reduce gives every rank the E_c of all frequencies."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
mp = pytest.importorskip("torch.multiprocessing")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, queue):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        ms, solves = bench.aggregate_over_ranks(100.0 + 50.0 * rank, 8192 + rank, torch.device("cpu"))
        queue.put((rank, ms, solves))
    finally:
        dist.destroy_process_group()


def test_replica_aggregation_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    queue = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, queue)) for r in range(2)]
    for p in procs:
        p.start()
    results = sorted(queue.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert results == [(0, 150.0, 16385), (1, 150.0, 16385)]


def _shard_worker(rank, world, port, queue):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import numpy as np
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import importlib.util
        import oracle
        import synth
        # the shard module holds host logic only; load it without the package (which needs the library)
        spec = importlib.util.spec_from_file_location("shard", os.path.join(os.path.dirname(os.path.dirname(
            os.path.abspath(__file__))), "paper_2504_01816_gb300", "shard.py"))
        shard = importlib.util.module_from_spec(spec)
        spec.loader.exec_module(shard)
        s = synth.small_system((9, 8, 7), h=0.5, n_s=2, n_wells=2, seed=51)
        V0 = synth.trial_vectors(51, 4, s.n_d)
        o = oracle.Oracle.from_system(s)
        n_omega = 5

        def evaluate(first, count):
            r = oracle.rpa_ec(o, V0, n_omega, tol=1e-10, eps_c=0.0, fixed_iters=2, independent_frequencies=True,
                              omega_subset=range(first, first + count))
            return r.e_c_per_omega, r.lambdas

        e_c, ecm, lam = shard.ec_sharded(evaluate, n_omega, world, rank)
        queue.put((rank, e_c, ecm.tolist(), lam.tolist(), shard.frequency_partition(n_omega, world, rank)))
    finally:
        dist.destroy_process_group()


def test_frequency_sharding_over_two_gloo_ranks():
    import numpy as np
    import oracle
    import synth
    ctx = mp.get_context("spawn")
    queue = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_shard_worker, args=(r, 2, port, queue)) for r in range(2)]
    for p in procs:
        p.start()
    results = sorted(queue.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    # the two ranks split 5 frequencies 3 + 2 and agree on the combined result
    assert [r[4] for r in results] == [(0, 3), (3, 2)]
    assert results[0][1] == results[1][1] and results[0][2] == results[1][2] and results[0][3] == results[1][3]
    # ... which is the single-process E_c over all frequencies (independent frequencies)
    s = synth.small_system((9, 8, 7), h=0.5, n_s=2, n_wells=2, seed=51)
    ref = oracle.rpa_ec(oracle.Oracle.from_system(s), synth.trial_vectors(51, 4, s.n_d), 5, tol=1e-10, eps_c=0.0,
                        fixed_iters=2, independent_frequencies=True)
    assert abs(results[0][1] - ref.e_c) < 1e-13
    assert np.max(np.abs(np.array(results[0][2]) - ref.e_c_per_omega)) < 1e-14
    assert np.max(np.abs(np.array(results[0][3]) - ref.lambdas)) < 1e-14


def test_frequency_partition_covers_every_frequency_once():
    import importlib.util
    spec = importlib.util.spec_from_file_location("shard", os.path.join(os.path.dirname(os.path.dirname(
        os.path.abspath(__file__))), "paper_2504_01816_gb300", "shard.py"))
    shard = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(shard)
    for n_omega in (1, 5, 8, 12):
        for world in (1, 2, 3, 8, 13):
            seen = []
            for rank in range(world):
                first, count = shard.frequency_partition(n_omega, world, rank)
                seen.extend(range(first, first + count))
            assert seen == list(range(n_omega)), (n_omega, world)
