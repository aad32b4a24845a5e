"""The all-cores timing runner of the oracle's LF chain (the CPU baseline's all-cores leg).

Members split over threads step exactly as in one thread (draws keyed by member and sweep, the
theta step serial with an order-free correctly rounded sum), so any thread count gives the same
chain bit for bit; and the runner is the oracle's own chain up to the rounding of the sum over
members (math.fsum here, Neumaier's method in the chain)."""
import numpy as np

import oracle
from oracle import allcores
from paper_2105_08026_gb300 import synth


def test_thread_count_does_not_change_the_chain_and_it_is_the_oracles():
    data = synth.lf_data(700, seed=31)
    theta0, scale, consts = synth.lf_settings(data, nL=48, nr=40)
    chi0 = synth.lf_chi_init(data, theta0)
    r1, c1, s1, _ = allcores.lf_run(data.fhat, data.r, consts, theta0, scale, 4, chi0, 60, threads=1)
    r4, c4, s4, _ = allcores.lf_run(data.fhat, data.r, consts, theta0, scale, 4, chi0, 60, threads=4)
    assert np.array_equal(r1, r4) and np.array_equal(c1, c4) and np.array_equal(s1, s4)
    ch = oracle.Chain(oracle.LF, data.fhat, data.r, consts, theta0, scale, 4, chi0)
    orows, _ = ch.run(0, 60)
    assert np.allclose(r4, orows, rtol=1e-12, atol=1e-12)
    assert np.allclose(c4, ch.chi, rtol=1e-12, atol=1e-12)
    assert np.allclose(s4, ch.S, rtol=1e-12, atol=1e-12)
    assert len(np.unique(r4[:, 0])) > 5  # the theta chain moved
