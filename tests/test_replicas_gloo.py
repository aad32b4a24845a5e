"""The multi-process path of bench.py (independent replicas, weak scaling) with world_size 2
over gloo on the CPU: each rank runs its own replica (its own catalog and chain seed), the
timed region's duration is the maximum over ranks, and the whole-job value counts every
rank's units. The replicas here are oracle chains on small catalogs, so that the test needs
no GPU; the reduction and aggregation code is the same that the CUDA benchmark calls."""
import json
import os
import socket
import sys
import time

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import numpy as np
    import torch.distributed as dist

    import bench
    import oracle
    from paper_2105_08026_gb300 import synth

    dist.init_process_group("gloo", rank=rank, world_size=world)
    ws, r, local = bench.dist_env()
    assert (ws, r, local) == (world, rank, rank)
    data_seed, chain_seed = bench.replica_seeds(rank)
    data = synth.nn1_data(400, seed=data_seed)
    theta0, scale, consts = synth.nn1_settings(data)
    ch = oracle.Chain(oracle.NN1, data.y, data.sigma, consts, theta0, scale, chain_seed, data.y.copy())
    dist.barrier()
    t0 = time.perf_counter()
    rows, _ = ch.run(0, 300 + 200 * rank)  # ranks of unequal speed
    ms = (time.perf_counter() - t0) * 1e3
    dist.barrier()
    t_max = bench.max_over_ranks(ms, device="cpu")
    value = bench.replica_value(ws, 400 * 300, t_max)
    with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
        json.dump({"ms": ms, "t_max": t_max, "value": value, "first_row": rows[0].tolist(),
                   "y0": float(data.y[0])}, f)
    dist.destroy_process_group()


@pytest.mark.slow
def test_two_replicas_over_gloo(tmp_path):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    mp.start_processes(_rank_main, args=(2, _free_port(), str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    r = [json.load(open(tmp_path / f"rank{q}.json")) for q in range(2)]
    # both ranks agree on the maximum, and it is the slower rank's time
    assert r[0]["t_max"] == r[1]["t_max"] == max(r[0]["ms"], r[1]["ms"])
    assert r[0]["value"] == r[1]["value"] == pytest.approx(2 * 400 * 300 / (r[0]["t_max"] * 1e-3))
    # replicas are independent: different catalogs and chains
    assert r[0]["y0"] != r[1]["y0"]
    assert r[0]["first_row"] != r[1]["first_row"]


def test_single_process_reduction_is_identity():
    sys.path.insert(0, ROOT)
    pytest.importorskip("torch")
    import bench
    assert bench.max_over_ranks(12.5, device="cpu") == 12.5
    assert bench.replica_value(1, 3e5 * 1000, 81.6) == pytest.approx(3e5 * 1000 / 0.0816)
    assert bench.replica_seeds(0) != bench.replica_seeds(1)
