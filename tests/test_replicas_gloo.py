"""Multi-process path of the benchmark on CPU: a trajectory does not shard, so
`bench.py --gpus N` runs N independent replicas and reports the whole-job
rate over the slowest rank. Two gloo ranks on 127.0.0.1 check the timing
aggregation (maximum over ranks, steps of every rank counted) and that the
replicas start from distinct seeded states."""
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, ms_of_rank, steps, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    import vibmodels as vm
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        ws_env, rank_env, _ = bench._dist()
        ms, value = bench._aggregate_replicas(ms_of_rank[rank], steps, ws_env, "cpu")
        m = vm.model_internal_conversion()
        ts = vm.random_right_canonical_mps(bench.STATE_SEED + rank_env, vm.local_dims(m), 8)
        np.save(os.path.join(out_dir, f"r{rank}.npy"), np.array([ms, value, rank_env, ws_env]))
        np.save(os.path.join(out_dir, f"t{rank}.npy"), ts[3])
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_replicas_report_the_slowest_rank_and_all_steps(tmp_path):
    import torch.multiprocessing as mp
    ms_of_rank = [812.5, 1250.0]
    steps = 5
    mp.start_processes(_rank_main, args=(2, _free_port(), ms_of_rank, steps, str(tmp_path)), nprocs=2,
                       join=True, start_method="spawn")
    r = [np.load(tmp_path / f"r{k}.npy") for k in range(2)]
    for k, (ms, value, rank, ws) in enumerate(r):
        assert (rank, ws) == (k, 2)
        assert ms == max(ms_of_rank)
        assert value == pytest.approx(2 * steps / (max(ms_of_rank) / 1e3), rel=1e-15)
    # every rank propagates its own replica from its own seeded state
    t0, t1 = (np.load(tmp_path / f"t{k}.npy") for k in range(2))
    assert t0.shape == t1.shape and not np.allclose(t0, t1)


def test_single_process_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    ms, value = bench._aggregate_replicas(500.0, 4, 1)
    assert ms == 500.0 and value == pytest.approx(8.0)
