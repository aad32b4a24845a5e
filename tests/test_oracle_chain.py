"""Statistical pins of the oracle's Markov chain (no GPU needed).

- NN1 member step with theta fixed reaches the closed-form conditional
  N(m, v), v = (1/sigma^2 + 1/tau^2)^-1, m = v (y/sigma^2 + mu/tau^2), and RAM
  drives the mean acceptance to alpha_* = 0.4 (Sec. 2.2).
- NN1 full MWG posterior of (mu, ln tau) agrees with the exact posterior by
  one-dimensional quadrature (mu integrated analytically) within 4 MCSE.
- LF member step with theta fixed passes simulation-based calibration against
  the paper's data-generating process (Sec. 4-5): the rank of the true latent
  among posterior draws is uniform, which fixes the member likelihood, the
  ln L Jacobian and the truncation.
- run(a) followed by run(b) equals run(a+b) exactly (counter-based RNG).
"""
import math

import numpy as np
import pytest
import scipy.integrate
import scipy.stats

import oracle
from oracle import stats
from paper_2105_08026_gb300 import synth


def _fixed_theta_chain(model, y, aux, consts, theta, chi0, seed):
    p = oracle.MODEL_P[model]
    return oracle.Chain(model, y, aux, consts, theta, np.zeros(p), seed, chi0, adapt_theta=False)


def test_nn1_member_conditional_and_ram_acceptance():
    n = 4000
    y, sig, mu, tau = 1.0, 0.8, 0.3, 0.6
    ch = _fixed_theta_chain(oracle.NN1, np.full(n, y), np.full(n, sig), [-10, 10], [mu, math.log(tau)],
                            np.full(n, y), seed=99)
    ch.run(0, 300)
    a0 = ch.member_accepts.value
    ch.run(0, 200)
    acc_rate = (ch.member_accepts.value - a0) / (200 * n)
    v = 1.0 / (1.0 / sig**2 + 1.0 / tau**2)
    m = v * (y / sig**2 + mu / tau**2)
    assert scipy.stats.kstest(ch.chi, scipy.stats.norm(loc=m, scale=math.sqrt(v)).cdf).pvalue > 1e-3
    assert abs(acc_rate - 0.4) < 0.02
    assert np.all(ch.theta == [mu, math.log(tau)])


def _nn1_exact_posterior(y, sig, lo=-10.0, hi=10.0, m=40001):
    s = np.linspace(lo, hi, m)
    tau2 = np.exp(2 * s)[:, None]
    w = 1.0 / (tau2 + sig[None, :] ** 2)
    sw = w.sum(axis=1)
    muhat = (w * y[None, :]).sum(axis=1) / sw
    logp = 0.5 * np.log(2 * math.pi / sw) + 0.5 * np.log(w / (2 * math.pi)).sum(axis=1) \
        - 0.5 * (w * (y[None, :] - muhat[:, None]) ** 2).sum(axis=1)
    p = np.exp(logp - logp.max())
    p /= np.trapezoid(p, s)
    Es = np.trapezoid(p * s, s)
    Vs = np.trapezoid(p * (s - Es) ** 2, s)
    Emu = np.trapezoid(p * muhat, s)
    Vmu = np.trapezoid(p * (1.0 / sw + muhat**2), s) - Emu**2
    return Emu, Vmu, Es, Vs


@pytest.mark.slow
def test_nn1_posterior_matches_quadrature():
    data = synth.nn1_data(300, seed=4242)
    Emu, Vmu, Es, Vs = _nn1_exact_posterior(data.y, data.sigma)
    theta0, scale, consts = synth.nn1_settings(data)
    ch = oracle.Chain(oracle.NN1, data.y, data.sigma, consts, theta0, scale, 7, data.y.copy())
    rows, _ = ch.run(3000, 30000)
    mu_s, s_s = rows[:, 0], rows[:, 1]
    for x, E, V in ((mu_s, Emu, Vmu), (s_s, Es, Vs)):
        se = stats.mcse(x)
        assert abs(x.mean() - E) < 4 * se, (x.mean(), E, se)
        # variance: MCSE of a variance estimate ~ V sqrt(2/ESS)
        ess = stats.ess_geyer(x)
        assert abs(x.var() - V) < 4 * V * math.sqrt(2.0 / ess) + 1e-12


def test_lf_member_step_simulation_based_calibration():
    data = synth.lf_data(2000, seed=77)
    theta = np.array([data.beta, math.log(data.L_star), math.log(data.L_low)])
    consts = oracle.lf_consts(data.sigma_F, data.F_th, data.r_max, 8, 8)  # theta fixed: etabar cancels
    chi0 = synth.lf_chi_init(data, theta)
    ch = _fixed_theta_chain(oracle.LF, data.fhat, data.r, consts, theta, chi0, seed=5)
    ch.run(0, 300)
    draws = []
    for _ in range(16):
        ch.run(0, 20)
        draws.append(ch.chi.copy())
    draws = np.array(draws)
    truth = np.log(data.L_true)
    ranks = (draws < truth[None, :]).sum(axis=0)  # 0..16
    counts = np.bincount(ranks, minlength=17)
    assert scipy.stats.chisquare(counts).pvalue > 1e-3, counts
    assert abs((draws < truth[None, :]).mean() - 0.5) < 0.03


def test_run_split_equals_run_whole():
    data = synth.nn1_data(200, seed=3)
    theta0, scale, consts = synth.nn1_settings(data)
    a = oracle.Chain(oracle.NN1, data.y, data.sigma, consts, theta0, scale, 11, data.y.copy())
    b = oracle.Chain(oracle.NN1, data.y, data.sigma, consts, theta0, scale, 11, data.y.copy())
    ra, _ = a.run(0, 300)
    rb1, _ = b.run(0, 120)
    rb2, _ = b.run(0, 180)
    assert np.array_equal(ra, np.concatenate([rb1, rb2]))
    assert np.array_equal(a.chi, b.chi) and np.array_equal(a.S, b.S) and np.array_equal(a.S_theta, b.S_theta)


@pytest.mark.slow
def test_lf_posterior_recovers_truth():
    """Thinned-likelihood theta step (eq. epdf with the selection integral): with N = 3000 detected
    objects the posterior covers the true (beta, ln L*, ln L_low) within 4 posterior sd."""
    data = synth.lf_data(3000, seed=314)
    theta0, scale, consts = synth.lf_settings(data, nL=64, nr=64)
    ch = oracle.Chain(oracle.LF, data.fhat, data.r, consts, theta0, scale, 21, synth.lf_chi_init(data, theta0))
    rows, _ = ch.run(1000, 3000)
    truth = theta0
    for j in range(3):
        sd = rows[:, j].std()
        assert abs(rows[:, j].mean() - truth[j]) < 4 * sd + 4 * stats.mcse(rows[:, j]), (j, rows[:, j].mean(), sd)


def _lf_member_logp(data, theta, q):
    """log p_i(theta) = log int_{ln L_low} l_i(chi) f(chi;theta) dchi for every member, by Simpson's
    rule on 4001 points over the window where l_i exceeds e^-72 of its peak (down to ln L_low when
    the likelihood stays non-negligible down to zero flux)."""
    beta, lls, llow = theta
    sig = data.sigma_F
    out = np.empty(data.fhat.size)
    for i in range(data.fhat.size):
        top = math.log((data.fhat[i] + 12 * sig) / q[i])
        lo_f = data.fhat[i] - 12 * sig
        a = llow if lo_f <= 0 else max(llow, math.log(lo_f / q[i]))
        if a >= top:
            out[i] = -np.inf
            continue
        x = np.linspace(a, top, 4001)
        lg = -(data.fhat[i] - np.exp(x) * q[i]) ** 2 / (2 * sig * sig) + (beta + 1) * (x - lls) - np.exp(x - lls)
        m = lg.max()
        out[i] = m + math.log(scipy.integrate.simpson(np.exp(lg - m), x=x))
    return out


@pytest.mark.slow
@pytest.mark.parametrize("adapt", [False, True])
@pytest.mark.parametrize("j,scale", [(0, 0.3), (1, 0.6), (2, 0.5)])
def test_lf_single_component_posterior_tiny_n(j, scale, adapt):
    """LF theta step at tiny N (20 detected objects, 64 x 64 rule): with the other two components
    fixed, the chain's marginal of theta_j matches brute-force quadrature of
    pi(theta) prod_i p_i(theta) / etabar(theta)^N (eq. epdf), p_i the 1-D integral of each
    member's likelihood times the population density in ln L, within 4 MCSE in mean and
    variance. This pins the theta step's prior, its truncations, the -N ln etabar term and the
    exact sum over members together with the member steps.

    adapt: the theta step as the chain runs it by default, its RAM adaptation applied one sweep
    late (reading R3). The other two components then get proposal scales of 1e-10 (RAM needs
    every scale positive): the rank-one updates scale the factor along S U, which stays along
    theta_j, so they move by less than 1e-5 over the run (measured: 3e-7), nothing against the
    posterior widths (0.1 to 0.6). A wrong
    adaptation (one that lets the proposal depend on the current state) biases the stationary
    law and fails the comparison."""
    data = synth.lf_data(20, seed=515)
    theta0, _, consts = synth.lf_settings(data, nL=64, nr=64)
    q = 1.0 / (4 * math.pi * data.r**2)
    prop = np.full(3, 1e-10) if adapt else np.zeros(3)
    prop[j] = scale
    ch = oracle.Chain(oracle.LF, data.fhat, data.r, consts, theta0, prop, 41 + j + (10 if adapt else 0),
                      synth.lf_chi_init(data, theta0), adapt_theta=adapt)
    rows, _ = ch.run(2000, 24000)
    x = rows[:, j]
    assert np.allclose(np.delete(rows, j, axis=1), np.delete(theta0, j), rtol=0, atol=1e-5)
    sd0 = max(x.std(), 1e-3)
    lo, hi = x.mean() - 12 * sd0, x.mean() + 12 * sd0
    if j == 0:  # -2 < beta < 0
        lo, hi = max(lo, -2 + 1e-9), min(hi, -1e-9)
    elif j == 1:  # L_low < L*
        lo = max(lo, theta0[2] + 1e-9)
    else:
        hi = min(hi, theta0[1] - 1e-9)
    grid = np.linspace(lo, hi, 401)
    lp = np.empty(grid.size)
    for k, g in enumerate(grid):
        t = theta0.copy()
        t[j] = g
        lp[k] = (-math.log1p(t[0] ** 2) + t[2] + _lf_member_logp(data, t, q).sum()
                 - data.fhat.size * math.log(oracle.lf_etabar(t, consts)))
    p = np.exp(lp - lp.max())
    p /= np.trapezoid(p, grid)
    E = np.trapezoid(p * grid, grid)
    V = np.trapezoid(p * (grid - E) ** 2, grid)
    se = stats.mcse(x)
    assert abs(x.mean() - E) < 4 * se, (x.mean(), E, se)
    # the variance's Monte Carlo error from the squared deviations themselves (their batch means
    # carry the autocorrelation and the posterior's heavy upper tail in ln L*)
    se_v = stats.mcse((x - x.mean()) ** 2)
    assert abs(x.var() - V) < 4 * se_v, (x.var(), V, se_v)

