"""GPU parity of the paper's normal-normal benchmark model NN3 (Sec. 3: d = 3, C_pop and the
measurement scales known, theta = mu) against the oracle.

FP64: the lockstep bar of the other models (identical member and theta decisions except near
ties |Delta - ln u| < 1e-9; per-member log targets, latents, RAM factors and theta within
1e-12 relative) on the benchmark's population (mu_pop, C_pop = D R D, sigma_j as printed), at
N = 1000 for 1000 sweeps, at ragged sizes up to the benchmark's N = 1e4, and at N = 3e4.

Both forms: the chain's mu draws against the closed-form posterior N(ybar, (C_pop + Sigma)/N)
(means within 4 Monte Carlo standard errors, variances within 4 standard errors of a variance
estimate with the chain's ESS). FP32: per-member log target within 1e-5 relative of the oracle
at the same binary32 latents.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import stats
from paper_2105_08026_gb300 import cudahm, synth

from test_gpu_parity import _check_lockstep, _lockstep

pytestmark = pytest.mark.gpu


def test_nn3_lockstep_n1000():
    data = synth.nn3_data(1000, seed=1004)
    theta0, scale, consts = synth.nn3_settings(data)
    out = _lockstep(oracle.NN3, data.y, data.s, consts, theta0, scale, 4, data.y.copy(), 1000)
    _check_lockstep(*out)


@pytest.mark.parametrize("n,sweeps", [(1, 300), (257, 300), (10_000, 100), (30_000, 4)])
def test_nn3_lockstep_sizes(n, sweeps):
    data = synth.nn3_data(n, seed=90 + n)
    theta0, scale, consts = synth.nn3_settings(data)
    chi0 = data.y + 0.1 * np.random.default_rng(n).standard_normal(data.y.shape)
    out = _lockstep(oracle.NN3, data.y, data.s, consts, theta0, scale, 6, chi0, sweeps)
    _check_lockstep(*out)


def test_nn3_fp32_logdens():
    data = synth.nn3_data(30_000, seed=1004)
    theta0, scale, consts = synth.nn3_settings(data)
    s = cudahm.Sampler(cudahm.NN3, 30_000, theta_init=theta0, theta_prop_scale=scale, model_consts=consts,
                       precision=cudahm.FP32, seed=3)
    s.set_data(data.y, data.s)
    s.run(0, 40)
    chi, _ = s.chi()
    assert np.array_equal(chi, chi.astype(np.float32).astype(np.float64))
    th, _ = s.theta()
    lp32 = s.logdens(th)
    lp64 = oracle.member_logdens(oracle.NN3, data.y, data.s, consts, chi, th)
    err = np.abs(lp32 - lp64) / np.maximum(1.0, np.abs(lp64))
    assert err.max() <= 1e-5, err.max()


@pytest.mark.parametrize("precision", [cudahm.FP64, cudahm.FP32])
def test_nn3_posterior_closed_form(precision):
    n = 100
    data = synth.nn3_data(n, seed=78)
    theta0, scale, consts = synth.nn3_settings(data)
    s = cudahm.Sampler(cudahm.NN3, n, theta_init=theta0, theta_prop_scale=scale, model_consts=consts,
                       precision=precision, seed=12)
    s.set_data(data.y, data.s)
    rows = s.run(10_000, 80_000)
    V = (data.C_pop + np.diag(np.array(synth.NN3_SIGMA) ** 2)) / n
    m = data.y.mean(axis=0)
    ess = cudahm.cudahm_ess(rows)
    for j in range(3):
        x = rows[:, j]
        assert abs(ess[j] - stats.ess_geyer(x)) <= 1e-9 * ess[j]
        se = x.std() / math.sqrt(ess[j])
        assert abs(x.mean() - m[j]) < 4 * se, (j, x.mean(), m[j], se)
        assert abs(x.var() - V[j, j]) < 4 * V[j, j] * math.sqrt(2.0 / ess[j]), (j, x.var(), V[j, j], ess[j])
