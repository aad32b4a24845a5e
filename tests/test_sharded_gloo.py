"""The exchange step a split of one population over several devices needs (each rank steps its
own members, then one all-reduce of its exchange words, then every rank takes the same theta
decision), checked on the CPU with world_size 2 over gloo. The member steps come from the oracle
(their draws are keyed by the member's population index and the sweep, so a split leaves each
member's step unchanged); each rank encodes its d_i = log f(chi_i;theta') - log f(chi_i;theta)
into the same 16 words the device's shard pass writes (tests/shard_words.py: 32-bit limbs of an
exact fixed-point sum, flag counts, member count), the ranks add the words with an int64
all-reduce, and every rank decodes the total. The sum is exact, so the split chain equals the
one-rank chain bit for bit: theta rows, latents and RAM factors. The one-rank driver is also
checked against the oracle's own chain (its Neumaier sum differs only in rounding).
"""
import json
import math
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SWEEPS = 150


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _driver(data, theta0, scale, consts, seed, rank, world, allreduce):
    """NN1 chain with its members split over `world` ranks (theta step as the oracle's: RAM on
    theta with each step's update applied one sweep late, log alpha = D + N (c(theta') - c(theta))
    + ln pi(theta') - ln pi(theta), c = -ln tau); D from the all-reduced exchange words."""
    import oracle
    import shard_words
    y, sig = data.y, data.sigma
    n = y.size
    i0, i1 = n * rank // world, n * (rank + 1) // world
    chi = y.copy()
    S = np.ones(n)
    theta = np.array(theta0, dtype=np.float64)
    Sth = np.diag(np.asarray(scale, dtype=np.float64))
    params = np.array([0.4, 2.0 / 3.0, 0.4, 1.0])
    lo, hi = consts[0], consts[1]
    prior = lambda t: 0.0 if lo <= t[1] <= hi else -math.inf
    rows = []
    pend = None  # the previous step's RAM update: (U, alpha, eta)
    for s in range(SWEEPS):
        k = s + 1
        eta = (k + 1.0) ** (-2.0 / 3.0)
        U, ut = oracle.draw(seed, 1, 0, k, 2)
        thp = theta + Sth @ U
        lp_new = prior(thp)
        d_loc, _ = oracle.member_pass(oracle.NN1, y, sig, consts, params, seed, k, i0, i1, theta, thp, chi, S)
        D, _, f, members, shards = shard_words.decode(allreduce(shard_words.encode(d_loc)))
        assert members == n and shards == world and f[1] == 0
        if lp_new == -math.inf or f[0] > 0:
            logalpha = -math.inf
        elif f[2] > 0:
            logalpha = math.inf
        else:
            logalpha = D + n * (-thp[1] + theta[1]) + lp_new - prior(theta)
        alpha = 1.0 if logalpha >= 0.0 else math.exp(logalpha)
        if math.log(ut) < logalpha:
            theta = thp
        if pend is not None:
            Sth = oracle.ram_update(Sth, pend[0], pend[1], 0.4, pend[2])
        pend = (U, alpha, eta)
        rows.append(theta.copy())
    return np.array(rows), chi[i0:i1], S[i0:i1]


def _rank_main(rank, world, port, out_dir):
    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch
    import torch.distributed as dist
    from paper_2105_08026_gb300 import synth

    dist.init_process_group("gloo", rank=rank, world_size=world)
    data = synth.nn1_data(301, seed=77)  # ragged split: 150 + 151 members
    theta0, scale, consts = synth.nn1_settings(data)

    def allreduce(words):  # the exchange words of all ranks, added as 64-bit integers
        t = torch.from_numpy(words.copy())
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
        return t.numpy()

    rows, chi, S = _driver(data, theta0, scale, consts, 5, rank, world, allreduce)
    np.savez(os.path.join(out_dir, f"rank{rank}.npz"), rows=rows, chi=chi, S=S)
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.slow
def test_split_members_equal_one_rank_bit_for_bit(tmp_path):
    import torch.multiprocessing as mp
    from paper_2105_08026_gb300 import synth

    import oracle
    port = _free_port()
    mp.start_processes(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    r0, r1 = np.load(tmp_path / "rank0.npz"), np.load(tmp_path / "rank1.npz")
    assert np.array_equal(r0["rows"], r1["rows"])  # every rank took the same theta decisions
    data = synth.nn1_data(301, seed=77)
    theta0, scale, consts = synth.nn1_settings(data)
    rows1, chi1, S1 = _driver(data, theta0, scale, consts, 5, 0, 1, lambda v: v)
    assert np.array_equal(r0["rows"], rows1)
    assert np.array_equal(np.concatenate([r0["chi"], r1["chi"]]), chi1)
    assert np.array_equal(np.concatenate([r0["S"], r1["S"]]), S1)
    # the one-rank driver is the oracle's chain (Neumaier instead of an exact sum)
    ch = oracle.Chain(oracle.NN1, data.y, data.sigma, consts, theta0, scale, 5, data.y.copy())
    orows, _ = ch.run(0, SWEEPS)
    assert np.allclose(rows1, orows, rtol=1e-12, atol=1e-12)
