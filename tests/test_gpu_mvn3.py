"""GPU parity of the d = 3 normal population (Sec. 3 with C_pop unknown) against the oracle.

FP64: the lockstep bar of the other models (identical member and theta decisions except
near ties |Delta - ln u| < 1e-9, per-member log targets, latents, RAM factors and theta
within 1e-12 relative), on the population recipe of the d = 3 workload (mu = (0, 1, -1),
C_pop of condition number 20, s ~ U[0.3, 1]) at N = 1000 for 1000 sweeps, at ragged sizes,
and at the full N = 1e6 for the first sweeps. The device RAM factor is a rank-one Cholesky
modification while the oracle refactors S (I + c U U^T/|U|^2) S^T; both are the same matrix.

FP32 bulk form: per-member log target within 1e-5 relative of the oracle at the same
(binary32) latents, |sum of per-member log targets - oracle's sum| <= 1e-3 at N = 1e6, and
theta posterior means and variances within 4 Monte Carlo standard errors of the oracle's chain.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import stats
from paper_2105_08026_gb300 import cudahm, synth

from test_gpu_parity import _check_lockstep, _lockstep

pytestmark = pytest.mark.gpu


def test_mvn3_lockstep_n1000():
    data = synth.mvn3_data(1000, seed=1003)
    theta0, scale, consts = synth.mvn3_settings(data)
    out = _lockstep(oracle.MVN3, data.y, data.s, consts, theta0, scale, 3, data.y.copy(), 1000)
    _check_lockstep(*out)


@pytest.mark.parametrize("n", [1, 333, 4099])
def test_mvn3_lockstep_ragged_sizes(n):
    data = synth.mvn3_data(n, seed=60 + n)
    theta0, scale, consts = synth.mvn3_settings(data)
    chi0 = data.y + 0.1 * np.random.default_rng(n).standard_normal(data.y.shape)
    out = _lockstep(oracle.MVN3, data.y, data.s, consts, theta0, scale, 5, chi0, 200)
    _check_lockstep(*out)


def test_mvn3_full_size_lockstep_n1000000():
    """The d = 3 workload at its full size, N = 1e6, in the launch shape the benchmark uses."""
    data = synth.mvn3_data(1_000_000, seed=1003)
    theta0, scale, consts = synth.mvn3_settings(data)
    out = _lockstep(oracle.MVN3, data.y, data.s, consts, theta0, scale, 3, data.y.copy(), 3)
    _check_lockstep(*out)


def test_mvn3_run_split_and_checkpoint():
    data = synth.mvn3_data(3000, seed=17)
    theta0, scale, consts = synth.mvn3_settings(data)
    for prec in (cudahm.FP64, cudahm.FP32):
        mk = lambda: cudahm.Sampler(cudahm.MVN3, 3000, theta_init=theta0, theta_prop_scale=scale, seed=8,
                                    precision=prec)
        a, b, c = mk(), mk(), mk()
        for x in (a, b, c):
            x.set_data(data.y, data.s)
        ra = a.run(0, 301)
        rb = np.concatenate([b.run(0, 101), b.run(0, 200)])
        assert np.array_equal(ra, rb)
        assert np.array_equal(a.chi()[0], b.chi()[0]) and np.array_equal(a.chi()[1], b.chi()[1])
        c.run(0, 101)
        blob = c.checkpoint()
        d = mk()
        d.set_data(data.y, data.s)
        d.restore(blob)
        assert np.array_equal(d.run(0, 200), ra[101:])
        assert np.array_equal(d.chi()[1], a.chi()[1])


def test_mvn3_fp32_logdens_and_sum_n1000000():
    data = synth.mvn3_data(1_000_000, seed=1003)
    theta0, scale, consts = synth.mvn3_settings(data)
    s = cudahm.Sampler(cudahm.MVN3, data.y.shape[0], theta_init=theta0, theta_prop_scale=scale,
                       precision=cudahm.FP32, seed=3)
    s.set_data(data.y, data.s)
    s.run(0, 40)
    chi, _ = s.chi()
    assert np.array_equal(chi, chi.astype(np.float32).astype(np.float64))  # binary32 latents
    th, _ = s.theta()
    lp32 = s.logdens(th)
    lp64 = oracle.member_logdens(oracle.MVN3, data.y, data.s, consts, chi, th)
    err = np.abs(lp32 - lp64) / np.maximum(1.0, np.abs(lp64))
    assert err.max() <= 1e-5, err.max()
    assert abs(math.fsum(lp32) - math.fsum(lp64)) <= 1e-3


@pytest.mark.slow
def test_mvn3_fp32_posterior_matches_oracle_chain():
    data = synth.mvn3_data(300, seed=4243)
    theta0, scale, consts = synth.mvn3_settings(data)
    s = cudahm.Sampler(cudahm.MVN3, 300, theta_init=theta0, theta_prop_scale=scale, precision=cudahm.FP32, seed=23)
    s.set_data(data.y, data.s)
    a = s.run(4000, 40000)
    ch = oracle.Chain(oracle.MVN3, data.y, data.s, consts, theta0, scale, 24, data.y.copy())
    b, _ = ch.run(4000, 40000)
    for j in range(9):
        se = math.hypot(stats.mcse(a[:, j]), stats.mcse(b[:, j]))
        assert abs(a[:, j].mean() - b[:, j].mean()) < 4 * se, (j, a[:, j].mean(), b[:, j].mean(), se)
        ess = min(stats.ess_geyer(a[:, j]), stats.ess_geyer(b[:, j]))
        va, vb = a[:, j].var(), b[:, j].var()
        assert abs(va - vb) < 4 * max(va, vb) * math.sqrt(4.0 / ess), (j, va, vb, ess)


@pytest.mark.parametrize("precision", [cudahm.FP64, cudahm.FP32])
def test_mvn3_in_a_mixed_batch_equals_alone(precision):
    specs = []
    d = synth.nn1_data(900, seed=301)
    th, sc, c = synth.nn1_settings(d)
    specs.append(dict(model=cudahm.NN1, n=900, y=d.y, aux=d.sigma, th=th, sc=sc, c=c, seed=51))
    for q, n in enumerate((2000, 70000)):
        m = synth.mvn3_data(n, seed=302 + q)
        th, sc, c = synth.mvn3_settings(m)
        specs.append(dict(model=cudahm.MVN3, n=n, y=m.y, aux=m.s, th=th, sc=sc, c=c, seed=52 + q))
    l = synth.lf_data(1500, seed=305)
    th, sc, c = synth.lf_settings(l, nL=64, nr=128)
    specs.append(dict(model=cudahm.LF, n=1500, y=l.fhat, aux=l.r, th=th, sc=sc, c=c, seed=55))

    def make(sp):
        x = cudahm.Sampler(sp["model"], sp["n"], theta_init=sp["th"], theta_prop_scale=sp["sc"],
                           model_consts=sp["c"], seed=sp["seed"], precision=precision)
        x.set_data(sp["y"], sp["aux"])
        return x

    alone = []
    for sp in specs:
        x = make(sp)
        alone.append((x.run(20, 60, 2), x.chi(), x.theta()))
    batch = [make(sp) for sp in specs]
    rows, _ = cudahm.batch_run(batch, 20, 60, 2)
    for (ra, ca, ta), rb, x in zip(alone, rows, batch):
        assert np.array_equal(ra, rb)
        cb, tb = x.chi(), x.theta()
        assert np.array_equal(ca[0], cb[0]) and np.array_equal(ca[1], cb[1])
        assert np.array_equal(ta[0], tb[0]) and np.array_equal(ta[1], tb[1])
