"""Pins of the oracle's per-member running moments of the latents (no GPU needed).

The oracle keeps, for every latent component, Welford's running mean and sum of squared
deviations over the kept sweeps (the sweeps whose theta row is recorded: after the burn-in,
every thin-th). Its definition is the sample mean and the sample variance (divisor m - 1) of
the latent values at those sweeps, so the pin is that definition computed another way: a
twin chain (same seed, same start) is stepped one sweep at a time, its latents copied after
each kept sweep, and numpy's two-pass mean and var(ddof=1) of those copies are compared with
the recurrence. A dropped term, a wrong divisor, an off-by-one in the kept-sweep rule or a
component mix-up (d = 3) each fail one of these.
"""
import numpy as np
import pytest

import oracle
from paper_2105_08026_gb300 import synth


def _kept(n_burn, n_iter, thin):
    return [s for s in range(n_burn + n_iter) if s >= n_burn and (s - n_burn + 1) % thin == 0]


def _snapshots(make, runs):
    """Latents after every kept sweep of the given (n_burn, n_iter, thin) runs, from a twin
    chain stepped one sweep at a time."""
    twin = make(False)
    out = []
    for n_burn, n_iter, thin in runs:
        kept = set(_kept(n_burn, n_iter, thin))
        for s in range(n_burn + n_iter):
            twin.run(0, 1)
            if s in kept:
                out.append(twin.chi.reshape(twin.n, twin.d).copy())
    return np.array(out)


def _check(make, runs, rel=1e-12):
    ch = make(True)
    for r in runs:
        ch.run(*r)
    mean, var, m = ch.moments()
    snaps = _snapshots(make, runs)
    assert m == snaps.shape[0]
    ref_mean = snaps.mean(axis=0)
    ref_var = snaps.var(axis=0, ddof=1) if m > 1 else np.zeros_like(ref_mean)
    scale = np.maximum(1.0, np.abs(ref_mean))
    assert np.all(np.abs(mean - ref_mean) <= rel * scale)
    # the variance of values of size |x| carries rounding of ~ eps |x| sd (both ways of computing it)
    sd = np.sqrt(ref_var)
    assert np.all(np.abs(var - ref_var) <= 1e-12 * (ref_var + scale * sd) + 1e-300)
    return ch, snaps


def _nn1(keep):
    data = synth.nn1_data(60, seed=41)
    theta0, scale, consts = synth.nn1_settings(data)
    return oracle.Chain(oracle.NN1, data.y, data.sigma, consts, theta0, scale, 17, data.y.copy(),
                        keep_chi_moments=keep)


def _lf(keep):
    data = synth.lf_data(80, seed=43)
    theta0, scale, consts = synth.lf_settings(data, nL=16, nr=16)
    return oracle.Chain(oracle.LF, data.fhat, data.r, consts, theta0, scale, 19, synth.lf_chi_init(data, theta0),
                        keep_chi_moments=keep)


def _mvn3(keep):
    data = synth.mvn3_data(40, seed=45)
    theta0, scale, consts = synth.mvn3_settings(data)
    return oracle.Chain(oracle.MVN3, data.y.reshape(-1), data.s.reshape(-1), consts, theta0, scale, 23,
                        data.y.reshape(-1).copy(), keep_chi_moments=keep)


@pytest.mark.parametrize("make", [_nn1, _lf, _mvn3], ids=["nn1", "lf", "mvn3"])
def test_moments_equal_two_pass_mean_and_variance(make):
    _check(make, [(7, 20, 3)])


def test_moments_continue_across_runs():
    """Moments accumulate over every kept sweep since the chain started, across calls."""
    _check(_nn1, [(3, 10, 2), (0, 9, 3), (5, 4, 1)])


def test_burn_in_and_thinning_select_the_kept_sweeps():
    ch, snaps = _check(_nn1, [(10, 12, 4)])
    assert snaps.shape[0] == 3  # sweeps 13, 17, 21 (0-based) of 22


def test_one_kept_sweep_gives_the_value_and_zero_variance():
    ch = _nn1(True)
    ch.run(4, 1)
    mean, var, m = ch.moments()
    assert m == 1
    assert np.array_equal(mean.reshape(-1), ch.chi)
    assert np.all(var == 0.0)


def test_no_kept_sweep_leaves_moments_empty():
    ch = _nn1(True)
    ch.run(6, 0)
    mean, var, m = ch.moments()
    assert m == 0 and np.all(mean == 0.0) and np.all(var == 0.0)


def test_moments_do_not_change_the_chain():
    a, b = _lf(True), _lf(False)
    ra, _ = a.run(5, 12, 2)
    rb, _ = b.run(5, 12, 2)
    assert np.array_equal(ra, rb) and np.array_equal(a.chi, b.chi) and np.array_equal(a.S, b.S)
