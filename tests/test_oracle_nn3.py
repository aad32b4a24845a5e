"""Pins of the oracle's normal-normal benchmark model NN3 (Sec. 3: d = 3, C_pop and the
measurement scales known, theta = mu with a flat prior), no GPU needed.

- The member log target equals scipy's densities: log f is the multivariate normal log
  density of chi (mean mu, covariance C_pop) up to its constant normaliser, log l_i the sum
  of three univariate normal log densities up to theirs. This fixes the packing of C_pop in
  the model constants, its Cholesky factorisation and the forward substitution.
- The chain's mu draws match the closed-form posterior. Integrating each latent out,
  y_i | mu ~ N(mu, C_pop + Sigma_i), so with a flat prior mu | y ~ N(m, V) with
  V = (sum_i (C_pop + Sigma_i)^-1)^-1 and m = V sum_i (C_pop + Sigma_i)^-1 y_i; with the
  benchmark's common scales m is the sample mean of y and V = (C_pop + Sigma)/N. Means
  within 4 Monte Carlo standard errors, variances within 4 standard errors of a variance
  estimate with the chain's ESS, whitened cross-covariances within 5/sqrt(ESS).
"""
import math

import numpy as np
import scipy.stats

import oracle
from oracle import stats
from paper_2105_08026_gb300 import synth


def test_nn3_member_log_target_matches_scipy():
    g = np.random.default_rng(15)
    n = 100
    C = synth.nn3_cov()
    consts = synth.nn3_consts(C)
    y = g.normal(size=(n, 3)) * 3.0
    s = np.tile(np.array(synth.NN3_SIGMA), (n, 1))
    chi = y + g.normal(size=(n, 3))
    const = 0.5 * np.linalg.slogdet(2 * math.pi * C)[1]
    for _ in range(4):
        mu = g.normal(size=3) * 2.0
        lp = oracle.member_logdens(oracle.NN3, y, s, consts, chi, mu)
        ref_f = scipy.stats.multivariate_normal(mu, C).logpdf(chi) + const
        ref_l = (scipy.stats.norm(chi, s).logpdf(y) + np.log(s) + 0.5 * math.log(2 * math.pi)).sum(axis=1)
        assert np.allclose(lp, ref_f + ref_l, rtol=1e-12, atol=1e-11)
        for i in range(3):
            assert math.isclose(oracle.logf_obj(oracle.NN3, chi[i], mu, consts), ref_f[i], rel_tol=1e-12,
                                abs_tol=1e-11)


def test_nn3_posterior_closed_form():
    n = 30
    data = synth.nn3_data(n, seed=77)
    th0, sc, consts = synth.nn3_settings(data)
    Sig = np.diag(np.array(synth.NN3_SIGMA) ** 2)
    V = (data.C_pop + Sig) / n
    m = data.y.mean(axis=0)
    ch = oracle.Chain(oracle.NN3, data.y, data.s, consts, th0, sc, 5, data.y.copy())
    rows, _ = ch.run(5000, 60000)
    ess = np.array([stats.ess_geyer(rows[:, j]) for j in range(3)])
    for j in range(3):
        x = rows[:, j]
        assert abs(x.mean() - m[j]) < 4 * stats.mcse(x), (j, x.mean(), m[j])
        assert abs(x.var() - V[j, j]) < 4 * V[j, j] * math.sqrt(2.0 / ess[j]), (j, x.var(), V[j, j], ess[j])
    z = np.linalg.solve(np.linalg.cholesky(V), (rows - m).T).T
    K = np.cov(z, rowvar=False)
    off = K[~np.eye(3, dtype=bool)]
    assert np.all(np.abs(off) < 5.0 / math.sqrt(ess.min())), (K, ess)
    assert abs(ch.member_accepts.value / (65000 * n) - 0.4) < 0.01
