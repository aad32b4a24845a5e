"""Pins of the oracle's latent marginalisation by cubature (the theta-only alternative to MCMC
over the latents, Sec. 6), no GPU needed.

- NN1: the member integral int N-shaped l_i(chi) f(chi;theta) dchi has the closed form
  sqrt(2 pi) s exp(-(y - mu)^2/(2 (sigma^2 + tau^2))), s = sigma tau/sqrt(sigma^2 + tau^2);
  the 64-node rule on m +- 10 s reproduces it to rounding for every member and theta.
- LF: the two-panel rule matches adaptive quadrature (scipy's QUADPACK, an independent
  method) on the whole support [ln L_low, ln((Fhat + 40 sigma_F)/q)] for faint, typical and
  bright members and several theta; a theta whose L_low lies above the likelihood window
  gives -inf.
- NN1: the theta-only chain on the marginal posterior reproduces the exact posterior moments
  of (mu, ln tau) (one-dimensional quadrature, mu integrated analytically) within 4 MCSE.
- LF: the marginal chain and the member-by-member MWG chain target the same posterior: their
  theta means agree within 4 combined MCSE.
- BB1 (the paper's model, sigma(F) in the likelihood, no truncation): the rule against
  QUADPACK, and the marginal chain against the MWG chain, as for LF.
"""
import math

import numpy as np
import pytest
from scipy import integrate

import oracle
from oracle import stats
from paper_2105_08026_gb300 import synth

from test_oracle_chain import _nn1_exact_posterior


def test_nn1_member_integral_closed_form():
    g = np.random.default_rng(8)
    y = g.normal(0.0, 3.0, 500)
    sig = g.uniform(0.05, 5.0, 500)
    for _ in range(6):
        th = np.array([g.normal(0.0, 2.0), g.uniform(-3.0, 2.0)])
        lp = oracle.marg_logp(oracle.NN1, y, sig, [-10.0, 10.0], th)
        tau2 = math.exp(2 * th[1])
        s = sig * math.sqrt(tau2) / np.sqrt(sig**2 + tau2)
        ref = np.log(math.sqrt(2 * math.pi) * s) - (y - th[0]) ** 2 / (2 * (sig**2 + tau2))
        assert np.allclose(lp, ref, rtol=1e-14, atol=1e-13)


def _lf_ref(fhat, r, sigF, th):
    q = 1.0 / (4 * math.pi * r * r)
    b, lls, lll = th

    def logint(x):
        return -(fhat - math.exp(x) * q) ** 2 / (2 * sigF * sigF) + (b + 1) * (x - lls) - math.exp(x - lls)

    hi = math.log((fhat + 40 * sigF) / q)
    grid = np.linspace(lll, hi, 20001)
    m = max(max(logint(x) for x in grid), logint(max(math.log(fhat / q), lll)))
    pts = [p for p in (math.log(fhat / q), math.log(max(fhat - 10 * sigF, fhat / 2) / q)) if lll < p < hi]
    v, _ = integrate.quad(lambda x: math.exp(logint(x) - m), lll, hi, points=pts, epsabs=0, epsrel=2e-14, limit=500)
    return m + math.log(v)


def test_lf_member_integral_vs_adaptive_quadrature():
    data = synth.lf_data(20000, seed=1002)
    th0, _, consts = synth.lf_settings(data, nL=8, nr=8)
    sigF = data.sigma_F
    order = np.argsort(data.fhat)
    pick = np.concatenate([order[:8], order[len(order) // 2: len(order) // 2 + 8], order[-8:],
                           np.random.default_rng(1).choice(data.fhat.size, 24, replace=False)])
    for dth in ((0.0, 0.0, 0.0), (0.05, 0.3, 0.5), (-0.1, -0.3, -1.0)):
        th = th0 + np.array(dth)
        lp = oracle.marg_logp(oracle.LF, data.fhat[pick], data.r[pick], consts, th)
        for k, i in enumerate(pick):
            ref = _lf_ref(data.fhat[i], data.r[i], sigF, th)
            if not np.isfinite(ref):
                continue
            # QUADPACK itself drifts ~1e-11 on the narrowest peaks (Fhat/sigma_F ~ 1e4)
            assert abs(lp[k] - ref) < 5e-11, (i, data.fhat[i] / sigF, lp[k], ref)
    # L_low above every likelihood window: no mass left on the support
    th = th0.copy()
    th[2] = 60.0
    assert np.all(oracle.marg_logp(oracle.LF, data.fhat[:10], data.r[:10], consts, th) == -np.inf)


@pytest.mark.slow
def test_nn1_marginal_chain_matches_exact_posterior():
    data = synth.nn1_data(300, seed=4242)
    Emu, Vmu, Es, Vs = _nn1_exact_posterior(data.y, data.sigma)
    theta0, scale, consts = synth.nn1_settings(data)
    ch = oracle.MarginalChain(oracle.NN1, data.y, data.sigma, consts, theta0, scale, 7)
    rows, _ = ch.run(1000, 12000)
    for x, E, V in ((rows[:, 0], Emu, Vmu), (rows[:, 1], Es, Vs)):
        se = stats.mcse(x)
        assert abs(x.mean() - E) < 4 * se, (x.mean(), E, se)
        ess = stats.ess_geyer(x)
        assert abs(x.var() - V) < 4 * V * math.sqrt(2.0 / ess), (x.var(), V, ess)


@pytest.mark.slow
def test_lf_marginal_chain_agrees_with_mwg_chain():
    data = synth.lf_data(200, seed=314)
    theta0, scale, consts = synth.lf_settings(data, nL=64, nr=64)
    mc = oracle.MarginalChain(oracle.LF, data.fhat, data.r, consts, theta0, scale, 21)
    ra, _ = mc.run(1000, 9000)
    ch = oracle.Chain(oracle.LF, data.fhat, data.r, consts, theta0, scale, 22, synth.lf_chi_init(data, theta0))
    rb, _ = ch.run(2000, 30000)
    for j in range(3):
        a, b = ra[:, j], rb[:, j]
        se = math.hypot(stats.mcse(a), stats.mcse(b))
        assert abs(a.mean() - b.mean()) < 4 * se, (j, a.mean(), b.mean(), se)


def _bb1_ref(fhat, r, consts, th):
    s0, al = consts[0], consts[1]
    q = 1.0 / (4 * math.pi * r * r)
    b, lnl, lnu = th

    def logint(x):
        L = math.exp(x)
        F = L * q
        s2 = s0 * s0 + (al * F) ** 2
        z = L / math.exp(lnl)
        lg = math.log(-math.expm1(-z)) if z <= math.log(2.0) else math.log1p(-math.exp(-z))
        return -0.5 * math.log(s2) - (fhat - F) ** 2 / (2 * s2) + lg + b * (x - lnu) - L / math.exp(lnu) + x

    lo = lnl + consts[7]
    hi = math.log((fhat + 60 * math.sqrt(s0 * s0 + (al * fhat) ** 2)) / q)
    grid = np.linspace(lo, hi, 20001)
    m = max(logint(x) for x in grid)
    pk = math.log(fhat / q)
    v, _ = integrate.quad(lambda x: math.exp(logint(x) - m), lo, hi, points=[pk] if lo < pk < hi else None,
                          epsabs=0, epsrel=2e-14, limit=500)
    return m + math.log(v)


def test_bb1_member_integral_vs_adaptive_quadrature():
    """The paper's BB1 model (flux-dependent error sigma(F), no truncation): the rule against
    QUADPACK over [ln l + ln(lower/l), ln((Fhat + 60 sigma(Fhat))/q)], faint and bright members."""
    data = synth.bb1_data(3000, seed=22)
    th0, _, consts = synth.bb1_settings(data, nL=16, nr=16)
    order = np.argsort(data.fhat)
    pick = np.concatenate([order[:6], order[-6:], np.random.default_rng(1).choice(data.fhat.size, 16, replace=False)])
    for dth in ((0.0, 0.0, 0.0), (0.1, 0.3, -0.2), (-0.3, -0.5, 0.4)):
        th = th0 + np.array(dth)
        lp = oracle.marg_logp(oracle.BB1, data.fhat[pick], data.r[pick], consts, th)
        for k, i in enumerate(pick):
            ref = _bb1_ref(data.fhat[i], data.r[i], consts, th)
            assert abs(lp[k] - ref) < 5e-12 * max(1.0, abs(ref)), (i, lp[k], ref)


@pytest.mark.slow
def test_bb1_marginal_chain_agrees_with_mwg_chain():
    data = synth.bb1_data(200, seed=315)
    theta0, scale, consts = synth.bb1_settings(data, nL=64, nr=64)
    mc = oracle.MarginalChain(oracle.BB1, data.fhat, data.r, consts, theta0, scale, 23)
    ra, _ = mc.run(1000, 6000)
    ch = oracle.Chain(oracle.BB1, data.fhat, data.r, consts, theta0, scale, 24, synth.bb1_chi_init(data))
    rb, _ = ch.run(2000, 30000)
    for j in range(3):
        a, b = ra[:, j], rb[:, j]
        se = math.hypot(stats.mcse(a), stats.mcse(b))
        assert abs(a.mean() - b.mean()) < 4 * se, (j, a.mean(), b.mean(), se)
