"""Pins of the oracle's BB1 luminosity-function model (Sec. 5.1-5.2, App. B), no GPU needed.

- The detection threshold reproduces the value the paper prints for its parameters (golden
  fixture tests/golden/bb1_threshold.json, Sec. 5.2 eq. Fth).
- The population term integrates to the normaliser of App. B eq. normLumPDF, u/C(beta,u,l) =
  u Gamma(beta+1) (1 - (1+u/l)^-(beta+1)), or u ln(1+u/l) for beta = -1 (scipy quadrature).
- The member likelihood is the normal density of Fhat_i with mean F and sd sigma(F) (scipy).
- eta(F) is the normal tail P(Fhat > F_th | F) (scipy); H(L) is the detection probability of a
  source of luminosity L placed with density ~ r^2 (simulation); etabar/normaliser is the
  detected fraction of the simulated population (the catalog generator draws by rejection).
- The 1024 x 1024 rule has converged (2048 x 2048).
- With theta fixed, the member step passes simulation-based calibration against the data-
  generating process; with theta free, the posterior covers the truth.
"""
import json
import math
import os

import numpy as np
import pytest
import scipy.integrate
import scipy.special
import scipy.stats

import oracle
from oracle import stats
from paper_2105_08026_gb300 import synth

HERE = os.path.dirname(os.path.abspath(__file__))


def test_threshold_matches_printed_value():
    g = json.load(open(os.path.join(HERE, "golden", "bb1_threshold.json")))
    Fth = oracle.bb1_threshold(g["sigma0"], g["alpha"], g["nu"])
    assert float(f"{Fth:.{g['printed_significant_digits']}g}") == g["F_th_printed"]
    assert abs(synth.bb1_threshold(g["sigma0"], g["alpha"], g["nu"]) - Fth) <= 1e-15 * Fth


def _normaliser(beta, l, u):
    """int_0^inf (1 - e^{-L/l}) (L/u)^beta e^{-L/u} dL = u / C(beta, u, l) (App. B eq. normLumPDF)."""
    if beta == -1.0:
        return u * math.log1p(u / l)
    return u * scipy.special.gamma(beta + 1.0) * (1.0 - (1.0 + u / l) ** (-(beta + 1.0)))


@pytest.mark.parametrize("beta,l,u", [(-1.5, 1e8, 1e10), (-1.0, 3e7, 2e10), (-0.5, 1e8, 1e9), (-1.9, 1e9, 1e11)])
def test_population_term_integrates_to_appendix_normaliser(beta, l, u):
    th = [beta, math.log(l), math.log(u)]

    def f(t):  # exp(log f_obj) in chi = ln L already carries the Jacobian e^chi
        return math.exp(oracle.logf_obj(oracle.BB1, [t], th))
    pts = sorted([math.log(l), math.log(u)])
    lo, hi = math.log(l) - 200.0 / (beta + 2.0), math.log(u) + math.log(60.0) + 3.0
    val = sum(scipy.integrate.quad(f, a, b, epsabs=0, epsrel=1e-12, limit=500)[0]
              for a, b in ((lo, pts[0]), (pts[0], pts[1]), (pts[1], hi)))
    assert val == pytest.approx(_normaliser(beta, l, u), rel=1e-9)


def test_member_likelihood_is_normal_density_of_fhat():
    g = np.random.default_rng(3)
    c = oracle.bb1_consts(2.0, 0.05, 5.0, 1.0, 8, 8)
    th = [-1.5, math.log(1e8), math.log(1e10)]
    for _ in range(50):
        chi = g.uniform(15.0, 25.0)
        r = g.uniform(0.01, 1.0)
        F = math.exp(chi) / (4 * math.pi * r * r)
        sd = math.sqrt(2.0**2 + (0.05 * F) ** 2)
        fhat = F + sd * g.standard_normal()
        lp = oracle.member_logdens(oracle.BB1, [fhat], [r], c, [chi], th)[0]
        ll = lp - oracle.logf_obj(oracle.BB1, [chi], th)
        ref = scipy.stats.norm(F, sd).logpdf(fhat) + 0.5 * math.log(2 * math.pi)
        assert ll == pytest.approx(ref, rel=1e-12, abs=1e-12)


def test_detection_efficiency_is_normal_tail():
    sigma0, alpha, nu = 3.0, 0.02, 5.0
    c = oracle.bb1_consts(sigma0, alpha, nu, 1.0, 8, 8)
    Fth = oracle.bb1_threshold(sigma0, alpha, nu)
    F = np.concatenate([np.linspace(-10.0, 80.0, 901), [Fth, 1e3, 1e5]])
    got = oracle.bb1_detection(F, c)
    ref = scipy.stats.norm.sf(Fth, loc=F, scale=np.sqrt(sigma0**2 + (alpha * F) ** 2))
    assert np.allclose(got, ref, rtol=1e-13, atol=1e-300)


def test_H_equals_detection_probability_by_simulation():
    g = np.random.default_rng(9)
    d = synth.bb1_data(10, seed=5)  # for its sigma0 and F_th
    c = oracle.bb1_consts(d.sigma0, d.alpha, d.nu, d.r_max, 8, 1024)
    m = 2_000_000
    for L in (1e9, 1e10, 5e10, 2e11):
        r = d.r_max * g.random(m) ** (1.0 / 3.0)
        F = L / (4 * math.pi * r * r)
        p = np.mean(F + np.sqrt(d.sigma0**2 + (d.alpha * F) ** 2) * g.standard_normal(m) > d.F_th)
        se = math.sqrt(max(p * (1 - p), 1e-12) / m)
        assert abs(oracle.bb1_H(L, c) - p) < 5 * se + 1e-6


def test_etabar_rule_converged():
    d = synth.bb1_data(10, seed=5)
    th, _, c = synth.bb1_settings(d)
    c2 = c.copy()
    c2[4] = c2[5] = 2048
    a, b = oracle.bb1_etabar(th, c), oracle.bb1_etabar(th, c2)
    assert abs(a - b) / b < 1e-12


@pytest.mark.slow
def test_etabar_is_detected_fraction_times_normaliser():
    d = synth.bb1_data(20000, seed=1004)
    th, _, c = synth.bb1_settings(d)
    frac = oracle.bb1_etabar(th, c) / _normaliser(d.beta, d.l, d.u)
    p = 20000 / d.n_drawn  # binomial estimate of the detected fraction
    assert abs(frac - p) < 4 * math.sqrt(p * (1 - p) / d.n_drawn)


def test_member_step_simulation_based_calibration():
    data = synth.bb1_data(1500, seed=78)
    th = np.array([data.beta, math.log(data.l), math.log(data.u)])
    c = oracle.bb1_consts(data.sigma0, data.alpha, data.nu, data.r_max, 8, 8)  # theta fixed: etabar cancels
    ch = oracle.Chain(oracle.BB1, data.fhat, data.r, c, th, np.zeros(3), 6, synth.bb1_chi_init(data),
                      adapt_theta=False)
    ch.run(0, 300)
    draws = []
    for _ in range(16):
        ch.run(0, 20)
        draws.append(ch.chi.copy())
    draws = np.array(draws)
    truth = np.log(data.L_true)
    ranks = (draws < truth[None, :]).sum(axis=0)
    counts = np.bincount(ranks, minlength=17)
    assert scipy.stats.chisquare(counts).pvalue > 1e-3, counts
    assert abs((draws < truth[None, :]).mean() - 0.5) < 0.035


@pytest.mark.slow
def test_posterior_recovers_truth():
    """Thinned likelihood with the flux-dependent sigma(F) inside the selection integral: with
    N = 2000 detected objects the posterior covers the true (beta, ln l, ln u) within 4 sd."""
    data = synth.bb1_data(2000, seed=315)
    theta0, scale, consts = synth.bb1_settings(data, nL=96, nr=96)
    ch = oracle.Chain(oracle.BB1, data.fhat, data.r, consts, theta0, scale, 22, synth.bb1_chi_init(data))
    rows, _ = ch.run(800, 2400)
    for j in range(3):
        sd = rows[:, j].std()
        assert abs(rows[:, j].mean() - theta0[j]) < 4 * sd + 4 * stats.mcse(rows[:, j]), (j, rows[:, j].mean(), sd)
