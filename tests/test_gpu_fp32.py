"""FP32 bulk form: accuracy of its binary32 member arithmetic and agreement of its posteriors.

Bar (binary32 member terms, binary64 accumulation, accept and RAM factors):
- per-member log density within 1e-5 relative (|a - b| <= 1e-5 max(1, |b|)) of the FP64
  oracle evaluated at the same latents (the binary32 values, exactly as doubles) and theta;
- |sum of per-member log densities - oracle's sum| <= 1e-3 at N = 6e5 (NN1) and N = 1e6 (LF);
- theta posterior means within 4 Monte Carlo standard errors of the exact posterior (NN1,
  closed form) or of the FP64 chain (LF), variances within 4 of their standard errors.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import stats
from paper_2105_08026_gb300 import cudahm, synth

from test_oracle_chain import _nn1_exact_posterior

pytestmark = pytest.mark.gpu


def _rel_ok(a, b, rel):
    fin = np.isfinite(b)
    assert np.array_equal(np.isfinite(a), fin)
    err = np.abs(a[fin] - b[fin]) / np.maximum(1.0, np.abs(b[fin]))
    return float(err.max(initial=0.0))


def test_fp32_lf_logdens_against_oracle():
    data = synth.lf_data(300_000, seed=1002)
    theta0, scale, consts = synth.lf_settings(data)
    s = cudahm.Sampler(cudahm.LF, data.fhat.size, theta_init=theta0, theta_prop_scale=scale, model_consts=consts,
                       precision=cudahm.FP32, seed=8)
    s.set_data(data.fhat, data.r)
    s.run(0, 40)
    chi, _ = s.chi()
    assert np.array_equal(chi, chi.astype(np.float32).astype(np.float64))  # binary32 latents
    th, _ = s.theta()
    err = _rel_ok(s.logdens(th), oracle.member_logdens(oracle.LF, data.fhat, data.r, consts, chi, th), 1e-5)
    assert err <= 1e-5, err


def test_fp32_nn1_logdens_and_sum_n600000():
    data = synth.nn1_data(600_000, seed=1003)
    theta0, scale, consts = synth.nn1_settings(data)
    s = cudahm.Sampler(cudahm.NN1, data.y.size, theta_init=theta0, theta_prop_scale=scale, model_consts=consts,
                       precision=cudahm.FP32, seed=9)
    s.set_data(data.y, data.sigma)
    s.run(0, 30)
    chi, _ = s.chi()
    th, _ = s.theta()
    lp32 = s.logdens(th)
    lp64 = oracle.member_logdens(oracle.NN1, data.y, data.sigma, consts, chi, th)
    err = _rel_ok(lp32, lp64, 1e-5)
    assert err <= 1e-5, err
    assert abs(math.fsum(lp32) - math.fsum(lp64)) <= 1e-3


def test_fp32_lf_logdens_and_sum_n1000000():
    """The luminosity model at N = 1e6 (its log targets span the widest range of the three
    models): per-member error within 1e-5 and the sum within 1e-3 of the oracle's."""
    data = synth.lf_data(1_000_000, seed=1008)
    theta0, scale, consts = synth.lf_settings(data)
    s = cudahm.Sampler(cudahm.LF, data.fhat.size, theta_init=theta0, theta_prop_scale=scale, model_consts=consts,
                       precision=cudahm.FP32, seed=10)
    s.set_data(data.fhat, data.r)
    s.run(0, 30)
    chi, _ = s.chi()
    assert np.array_equal(chi, chi.astype(np.float32).astype(np.float64))
    th, _ = s.theta()
    lp32 = s.logdens(th)
    lp64 = oracle.member_logdens(oracle.LF, data.fhat, data.r, consts, chi, th)
    err = _rel_ok(lp32, lp64, 1e-5)
    assert err <= 1e-5, err
    dsum = math.fsum(lp32) - math.fsum(lp64)
    print("FP32 LF N=1e6: max rel", err, "sum error", dsum)
    assert abs(dsum) <= 1e-3, dsum


def _check_moments(x, E, V):
    se = stats.mcse(x)
    assert abs(x.mean() - E) < 4 * se, (x.mean(), E, se)
    ess = stats.ess_geyer(x)
    assert abs(x.var() - V) < 4 * V * math.sqrt(2.0 / ess), (x.var(), V, ess)


def test_fp32_nn1_posterior_matches_closed_form():
    data = synth.nn1_data(300, seed=4242)
    Emu, Vmu, Es, Vs = _nn1_exact_posterior(data.y, data.sigma)
    theta0, scale, consts = synth.nn1_settings(data)
    s = cudahm.Sampler(cudahm.NN1, 300, theta_init=theta0, theta_prop_scale=scale, model_consts=consts,
                       precision=cudahm.FP32, seed=17)
    s.set_data(data.y, data.sigma)
    rows = s.run(3000, 60000)
    _check_moments(rows[:, 0], Emu, Vmu)
    _check_moments(rows[:, 1], Es, Vs)


def test_fp32_lf_posterior_matches_fp64_chain():
    data = synth.lf_data(3000, seed=314)
    theta0, scale, consts = synth.lf_settings(data, nL=128, nr=128)
    out = {}
    for prec, seed in ((cudahm.FP64, 21), (cudahm.FP32, 22)):
        s = cudahm.Sampler(cudahm.LF, 3000, theta_init=theta0, theta_prop_scale=scale, model_consts=consts,
                           precision=prec, seed=seed)
        s.set_data(data.fhat, data.r)
        out[prec] = s.run(2000, 30000)
    a, b = out[cudahm.FP64], out[cudahm.FP32]
    for j in range(3):
        se = math.hypot(stats.mcse(a[:, j]), stats.mcse(b[:, j]))
        assert abs(a[:, j].mean() - b[:, j].mean()) < 4 * se, (j, a[:, j].mean(), b[:, j].mean(), se)
        ess = min(stats.ess_geyer(a[:, j]), stats.ess_geyer(b[:, j]))
        va, vb = a[:, j].var(), b[:, j].var()
        assert abs(va - vb) < 4 * max(va, vb) * math.sqrt(4.0 / ess), (j, va, vb, ess)
