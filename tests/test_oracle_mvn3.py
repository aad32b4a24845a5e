"""Pins of the oracle's d = 3 normal population (Sec. 3 with C_pop unknown), no GPU needed.

- The member log target equals log densities from scipy: log f + c(theta) is the
  multivariate normal log density of chi (mean mu, covariance L L^T) up to -3/2 ln 2 pi, and
  log l_i is the sum of three univariate normal log densities up to their normalisers. This
  fixes the unpacking of theta (log diagonal, row order) and the forward substitution.
- With theta fixed, the member step (three-dimensional RAM) reaches the closed-form
  conditional chi_i | y_i, theta ~ N(m, V), V = (C^-1 + D_i^-1)^-1, m = V (C^-1 mu + D_i^-1 y_i),
  and drives the mean acceptance to alpha_* = 0.4 (started from S_1 = 0.5 I, near the
  conditional's scale: from S_1 = I the three-dimensional adaptation needs ~10^4 sweeps).
- With every theta component but one held at its value, the chain's draws of that component
  match its exact marginal posterior, computed by one-dimensional quadrature of
  prod_i N(y_i; mu, C(theta) + D_i) (the latents integrated analytically, flat prior). This
  covers mu, a log-diagonal entry (and with it c(theta) = -sum ln L_jj) and an off-diagonal entry.
"""
import math

import numpy as np
import pytest
import scipy.stats

import oracle
from oracle import stats
from paper_2105_08026_gb300 import synth


def _L_of(theta):
    t = np.asarray(theta, dtype=np.float64)
    return np.array([[math.exp(t[3]), 0.0, 0.0], [t[4], math.exp(t[5]), 0.0], [t[6], t[7], math.exp(t[8])]])


def test_mvn3_member_log_target_matches_scipy():
    g = np.random.default_rng(5)
    n = 200
    y = g.normal(size=(n, 3))
    s = g.uniform(0.3, 1.0, size=(n, 3))
    chi = y + g.normal(size=(n, 3))
    for _ in range(5):
        theta = g.normal(size=9) * 0.7
        lp = oracle.member_logdens(oracle.MVN3, y, s, None, chi, theta)
        L = _L_of(theta)
        C = L @ L.T
        ref_f = scipy.stats.multivariate_normal(theta[:3], C).logpdf(chi) + (theta[3] + theta[5] + theta[8]) \
            + 1.5 * math.log(2 * math.pi)
        ref_l = (scipy.stats.norm(chi, s).logpdf(y) + np.log(s) + 0.5 * math.log(2 * math.pi)).sum(axis=1)
        assert np.allclose(lp, ref_f + ref_l, rtol=1e-12, atol=1e-12)


@pytest.mark.slow
def test_mvn3_member_conditional_and_ram_acceptance():
    n = 4000
    y = np.array([0.4, -1.0, 2.0])
    s = np.array([0.5, 0.9, 0.3])
    mu = np.array([0.0, 1.0, -1.0])
    theta = synth.mvn3_theta_from(mu, np.array([[2.0, 0.6, -0.3], [0.6, 1.0, 0.2], [-0.3, 0.2, 0.5]]))
    C = _L_of(theta) @ _L_of(theta).T
    ch = oracle.Chain(oracle.MVN3, np.tile(y, (n, 1)), np.tile(s, (n, 1)), None, theta, np.zeros(9), 11,
                      np.tile(y, (n, 1)), adapt_theta=False, chi_init_scale=0.5)
    ch.run(0, 600)
    a0 = ch.member_accepts.value
    ch.run(0, 600)
    acc_rate = (ch.member_accepts.value - a0) / (600 * n)
    Ci, Di = np.linalg.inv(C), np.diag(1.0 / s**2)
    V = np.linalg.inv(Ci + Di)
    m = V @ (Ci @ mu + Di @ y)
    x = ch.chi.reshape(n, 3)
    assert np.all(ch.theta == theta)
    # mean within 4 standard errors, every component
    assert np.all(np.abs(x.mean(axis=0) - m) < 4 * np.sqrt(np.diag(V) / n))
    # whitened draws are independent standard normals
    zw = np.linalg.solve(np.linalg.cholesky(V), (x - m).T).T
    for j in range(3):
        assert scipy.stats.kstest(zw[:, j], "norm").pvalue > 1e-3
    Cov = np.cov(zw, rowvar=False)
    assert np.all(np.abs(Cov - np.eye(3)) < 5 * math.sqrt(2.0 / n))
    assert abs(acc_rate - 0.4) < 0.02


def _marginal_posterior(data, theta, j, grid):
    """Exact posterior of theta_j on a grid (others fixed), prod_i N(y_i; mu, C + D_i)."""
    lp = np.empty(grid.size)
    D = data.s**2
    for q, v in enumerate(grid):
        t = np.array(theta, dtype=np.float64)
        t[j] = v
        L = _L_of(t)
        C = L @ L.T
        M = C[None, :, :] + np.einsum("ij,jk->ijk", D, np.eye(3))
        r = data.y - t[:3]
        sol = np.linalg.solve(M, r[:, :, None])[:, :, 0]
        lp[q] = -0.5 * np.sum(np.linalg.slogdet(M)[1]) - 0.5 * np.sum(r * sol)
    p = np.exp(lp - lp.max())
    p /= np.trapezoid(p, grid)
    E = np.trapezoid(p * grid, grid)
    return E, np.trapezoid(p * (grid - E) ** 2, grid)


@pytest.mark.slow
@pytest.mark.parametrize("j,scale", [(0, 0.3), (3, 0.25), (4, 0.4)])
def test_mvn3_single_component_posterior(j, scale):
    data = synth.mvn3_data(40, seed=808 + j)
    theta = synth.mvn3_theta_from(data.mu, data.C_pop)
    prop = np.zeros(9)
    prop[j] = scale
    ch = oracle.Chain(oracle.MVN3, data.y, data.s, None, theta, prop, 31 + j, data.y.copy(), adapt_theta=False)
    rows, _ = ch.run(2000, 24000)
    x = rows[:, j]
    assert np.all(rows[:, [q for q in range(9) if q != j]] == theta[[q for q in range(9) if q != j]])
    sd0 = math.sqrt(max(x.var(), 1e-6))
    grid = np.linspace(x.mean() - 12 * sd0, x.mean() + 12 * sd0, 1601)
    E, V = _marginal_posterior(data, theta, j, grid)
    se = stats.mcse(x)
    assert abs(x.mean() - E) < 4 * se, (x.mean(), E, se)
    ess = stats.ess_geyer(x)
    assert abs(x.var() - V) < 4 * V * math.sqrt(2.0 / ess), (x.var(), V, ess)
