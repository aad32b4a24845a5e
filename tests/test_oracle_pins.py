"""Pins of the CPU oracle against things other than itself (no GPU needed).

Each test names what fixes the expected value: an independent library
implementation, a closed form, an exact rational computation, an invariant, or
the data-generating process of the paper's model.
"""
import json
import math
import os
import subprocess
import sys
from fractions import Fraction

import numpy as np
import pytest
import scipy.special
import scipy.stats

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))


# ------------------------------------------------------------------ Philox --
def test_philox_matches_triton_implementation():
    """Philox4x32-10 (Salmon et al. SC'11) against Triton's independent implementation,
    run by Triton's CPU interpreter, on random counters and keys."""
    pytest.importorskip("triton")
    g = np.random.default_rng(5)
    ctr = g.integers(0, 2**32, size=(48, 4), dtype=np.uint64).tolist()
    ctr += [[0, 0, 0, 0], [0xFFFFFFFF] * 4, [3, 1, 7, 1999]]
    for key in ([0, 0], [0x9E3779B9, 0x00000001], [int(x) for x in g.integers(0, 2**31, 2)]):
        req = json.dumps({"ctr": ctr, "key": key})
        out = subprocess.run([sys.executable, os.path.join(HERE, "_triton_philox.py")], input=req,
                             capture_output=True, text=True, timeout=600)
        assert out.returncode == 0, out.stderr[-2000:]
        ref = json.loads(out.stdout)
        for c, r in zip(ctr, ref):
            mine = oracle.philox4x32_10(c, key).tolist()
            assert mine == r, (c, key, mine, r)


def test_uniform_recipe_exact():
    """u = (2m+1) 2^-53 with m the top 52 bits of the 64-bit word: checked in exact rationals."""
    g = np.random.default_rng(11)
    cases = [(0, 0), (0xFFFFFFFF, 0xFFFFFFFF), (0x80000000, 0), (0, 0xFFF), (0, 0x1000)]
    cases += [tuple(int(v) for v in g.integers(0, 2**32, 2)) for _ in range(200)]
    for wa, wb in cases:
        x = (wa << 32) | wb
        m = x >> 12
        exact = Fraction(2 * m + 1, 2**53)
        u = oracle.uniform(wa, wb)
        assert Fraction(u) == exact
        assert 0.0 < u < 1.0


def test_normals_and_accept_uniforms_distribution():
    """Box-Muller normals are N(0,1) and accept uniforms are U(0,1): moments and KS tests."""
    zs, us = [], []
    for i in range(4000):
        for k in (1, 2, 3, 977):
            z, u = oracle.draw(42, 0, i, k, 3)
            zs.extend(z)
            us.append(u)
    zs = np.array(zs)
    us = np.array(us)
    assert abs(zs.mean()) < 4.0 / math.sqrt(zs.size)
    assert abs(zs.var() - 1.0) < 4.0 * math.sqrt(2.0 / zs.size)
    assert scipy.stats.kstest(zs, "norm").pvalue > 1e-3
    assert scipy.stats.kstest(us, "uniform").pvalue > 1e-3
    # distinct streams, objects and sweeps give distinct draws
    assert oracle.draw(42, 0, 5, 9, 1)[0][0] != oracle.draw(42, 1, 5, 9, 1)[0][0]
    assert oracle.draw(42, 0, 5, 9, 1)[0][0] != oracle.draw(42, 0, 6, 9, 1)[0][0]
    assert oracle.draw(42, 0, 5, 9, 1)[0][0] != oracle.draw(43, 0, 5, 9, 1)[0][0]


def test_member_draw_layout_and_pairing():
    """Member draws: component a of sweeps k_o (odd) and k_o + 1 are the cosine and the sine of the
    Box-Muller pair of block (a, 0, i, k_o); the accept uniform of sweep k is block (d, 0, i, k)'s first."""
    seed, i = 0x0F1E2D3C4B5A6978, 41
    key = [seed & 0xFFFFFFFF, seed >> 32]
    for d in (1, 3):
        for k_o in (1, 7, 999):
            zo, uo = oracle.draw_member(seed, i, k_o, d)
            ze, ue = oracle.draw_member(seed, i, k_o + 1, d)
            for a in range(d):
                w = oracle.philox4x32_10([a, 0, i, k_o], key)
                ua, ub = oracle.uniform(int(w[0]), int(w[1])), oracle.uniform(int(w[2]), int(w[3]))
                rad = math.sqrt(-2.0 * math.log(ua))
                assert zo[a] == pytest.approx(rad * math.cos(2 * math.pi * ub), rel=1e-15, abs=1e-15)
                assert ze[a] == pytest.approx(rad * math.sin(2 * math.pi * ub), rel=1e-15, abs=1e-15)
            for kk, u in ((k_o, uo), (k_o + 1, ue)):
                w = oracle.philox4x32_10([d, 0, i, kk], key)
                assert u == oracle.uniform(int(w[0]), int(w[1]))
    # paired normals are independent N(0,1): correlation of (cos, sin) parts over many members
    zo = np.array([oracle.draw_member(5, j, 3, 1)[0][0] for j in range(20000)])
    ze = np.array([oracle.draw_member(5, j, 4, 1)[0][0] for j in range(20000)])
    assert abs(np.corrcoef(zo, ze)[0, 1]) < 4 / math.sqrt(zo.size)
    assert scipy.stats.kstest(ze, "norm").pvalue > 1e-3


def test_draw_block_layout():
    """Theta draws: normals 2j, 2j+1 come from block j; the accept uniform is the first uniform of
    block ceil(d/2)."""
    seed, s, i, k = 0x123456789ABCDEF, 0, 17, 4
    key = [seed & 0xFFFFFFFF, seed >> 32]
    w0 = oracle.philox4x32_10([0, s, i, k], key)
    w1 = oracle.philox4x32_10([1, s, i, k], key)
    ua, ub = oracle.uniform(int(w0[0]), int(w0[1])), oracle.uniform(int(w0[2]), int(w0[3]))
    z, u = oracle.draw(seed, s, i, k, 1)
    rad = math.sqrt(-2.0 * math.log(ua))
    assert z[0] == pytest.approx(rad * math.cos(2 * math.pi * ub), rel=1e-15, abs=1e-15)
    assert u == oracle.uniform(int(w1[0]), int(w1[1]))
    z2, _ = oracle.draw(seed, s, i, k, 2)
    assert z2[1] == pytest.approx(rad * math.sin(2 * math.pi * ub), rel=1e-15, abs=1e-15)


# ------------------------------------------------------- sums and algebra ---
def test_neumaier_sum_vs_exact_fsum():
    """Compensated sum against math.fsum (exactly rounded) on ill-conditioned data."""
    g = np.random.default_rng(3)
    for _ in range(20):
        n = int(g.integers(10, 20000))
        v = g.standard_normal(n) * np.exp(g.uniform(-30, 30, n))
        v = np.concatenate([v, -v[: n // 2] * (1 + 1e-12)])
        g.shuffle(v)
        exact = math.fsum(v.tolist())
        got = oracle.neumaier_sum(v)
        assert abs(got - exact) <= 4 * np.spacing(abs(exact)) + 1e-3 * np.abs(v).sum() * 2.0**-104


def test_cholesky_vs_lapack():
    g = np.random.default_rng(4)
    for d in (1, 2, 3, 5, 9):
        A = g.standard_normal((d, d))
        A = A @ A.T + d * np.eye(d)
        np.testing.assert_allclose(oracle.cholesky(A), np.linalg.cholesky(A), rtol=1e-13, atol=1e-13)


def test_ram_update_d1_closed_form():
    """d = 1: S_n = S_{n-1} sqrt(1 + eta (alpha - alpha_*)) (Sec. 2.2 step 3 with U U^T/|U|^2 = 1)."""
    g = np.random.default_rng(6)
    for _ in range(500):
        S = float(np.exp(g.uniform(-5, 5)))
        U = float(g.standard_normal())
        alpha = float(g.uniform())
        eta = float(g.uniform(0, 1))
        out = oracle.ram_update(np.array([[S]]), np.array([U]), alpha, 0.4, eta)[0, 0]
        ref = S * math.sqrt(1.0 + eta * (alpha - 0.4))
        assert abs(out - ref) <= 4 * np.spacing(ref)


@pytest.mark.parametrize("d", [2, 3, 9])
def test_ram_update_matches_lapack_cholesky_of_formula(d):
    """S_n S_n^T = S (I + c U U^T/|U|^2) S^T, factor from LAPACK; positive diagonal."""
    g = np.random.default_rng(7 + d)
    for _ in range(100):
        S = np.tril(g.standard_normal((d, d)))
        S[np.diag_indices(d)] = np.exp(g.uniform(-2, 2, d))
        U = g.standard_normal(d)
        alpha, eta = float(g.uniform()), float(g.uniform(0.0, 1.0))
        c = eta * (alpha - 0.4)
        rhs = S @ (np.eye(d) + c * np.outer(U, U) / (U @ U)) @ S.T
        out = oracle.ram_update(S, U, alpha, 0.4, eta)
        assert np.all(np.diag(out) > 0)
        np.testing.assert_allclose(out @ out.T, rhs, rtol=1e-12, atol=1e-12 * np.abs(rhs).max())
        # two factorisations of the same matrix agree up to its conditioning
        kappa = np.linalg.cond(rhs)
        np.testing.assert_allclose(out, np.linalg.cholesky(0.5 * (rhs + rhs.T)), rtol=1e-14 * kappa,
                                   atol=1e-14 * kappa * np.abs(S).max())


# ------------------------------------------------------------ quadrature ----
@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 16, 64, 100, 151])
def test_gauss_legendre_vs_high_precision(n):
    """Nodes and weights against 40-digit roots of P_n (mpmath), and against numpy's leggauss."""
    mpmath = pytest.importorskip("mpmath")
    x, w = oracle.gauss_legendre(n)
    xn, wn = np.polynomial.legendre.leggauss(n)
    np.testing.assert_allclose(x, xn, atol=2e-15)
    np.testing.assert_allclose(w, wn, rtol=1e-10, atol=1e-16)  # numpy loses ~1e-11 near the ends
    with mpmath.workdps(40):
        for i in range(0, (n + 1) // 2, max(1, n // 16)):
            r = mpmath.mpf(x[i])
            for _ in range(6):  # Newton in 40-digit arithmetic from the oracle's node
                r = r - mpmath.legendre(n, r) / mpmath.diff(lambda t: mpmath.legendre(n, t), r)
            dp = mpmath.diff(lambda t: mpmath.legendre(n, t), r)
            wr = 2 / ((1 - r**2) * dp**2)
            assert abs(float(r) - x[i]) <= 2e-16
            assert abs(float(wr) - w[i]) <= 2e-13 * float(wr)


def test_gauss_legendre_1024_exactness():
    """n-point GL integrates degree <= 2n-1 exactly; also a resolved oscillatory integral."""
    n = 1024
    x, w = oracle.gauss_legendre(n)
    assert abs(w.sum() - 2.0) < 1e-13
    assert np.all(np.diff(x) > 0) and np.all(w > 0)
    for m in (1, 2, 10, 100, 500, 1000, 1023):
        assert abs(np.sum(w * x ** (2 * m)) - 2.0 / (2 * m + 1)) < 1e-13 / math.sqrt(2 * m + 1) + 1e-15
        assert abs(np.sum(w * x ** (2 * m - 1))) < 1e-14
    om = 500.0
    assert abs(np.sum(w * np.cos(om * x)) - 2 * math.sin(om) / om) < 1e-13


# ---------------------------------------------------------- selection -------
def _lf_consts(nL=1024, nr=1024, sigF=2.0, Fth=10.0, rmax=4000.0):
    return oracle.lf_consts(sigF, Fth, rmax, nL, nr)


def test_detection_efficiency_is_normal_cdf():
    """eta(F) = Phi((F - F_th)/sigma_F) against scipy's ndtr (Cephes), across the whole range."""
    sigF, Fth = 2.0, 10.0
    c = _lf_consts(sigF=sigF, Fth=Fth)
    x = np.concatenate([np.linspace(-12, 12, 4001), [-38.0, 0.0, 8.5, 40.0]])
    F = Fth + sigF * x
    got = oracle.lf_detection(F, c)
    ref = scipy.special.ndtr((F - Fth) / sigF)
    assert np.all(np.abs(got - ref) <= 2e-16 + 1e-14 * ref)


def test_H_normalisation_all_detected():
    """When every distance gives a certain detection, H(L) = int h(r) dr = 1 (h ~ 3r^2/r_max^3)."""
    c = _lf_consts()
    L = 1e30  # flux at r_max is astronomically above threshold
    assert abs(oracle.lf_H(L, c) - 1.0) < 1e-14


def test_H_sharp_threshold_closed_form():
    """sigma_F -> 0: eta(F) is a step at F_th, so H(L) = min(1, (L/(4 pi F_th r_max^2))^(3/2)).
    A 1024-node rule resolves the step to O(1/n)."""
    Fth, rmax = 10.0, 4000.0
    c = _lf_consts(sigF=1e-9 * Fth, Fth=Fth, rmax=rmax)
    for frac in (0.01, 0.1, 0.3, 0.7, 0.95):
        L = 4 * math.pi * Fth * rmax**2 * frac ** (2.0 / 3.0)
        ref = frac
        assert abs(oracle.lf_H(L, c) - ref) < 4e-3 * ref + 1e-4


def test_H_equals_detection_probability_by_simulation():
    """H(L) is the probability that a source of luminosity L, placed with density ~ r^2 on
    [0, r_max] and measured with N(0, sigma_F^2) flux noise, is detected (Fhat > F_th)."""
    g = np.random.default_rng(8)
    sigF, Fth, rmax = 2.0, 10.0, 4000.0
    c = _lf_consts(sigF=sigF, Fth=Fth, rmax=rmax)
    m = 2_000_000
    for L in (2e8, 1e9, 2e9, 6e9, 2e10):
        r = rmax * g.random(m) ** (1.0 / 3.0)
        F = L / (4 * math.pi * r * r)
        p = np.mean(F + sigF * g.standard_normal(m) > Fth)
        se = math.sqrt(max(p * (1 - p), 1e-12) / m)
        assert abs(oracle.lf_H(L, c) - p) < 5 * se + 1e-6


def test_etabar_rule_converged():
    """The 1024 x 1024 rule agrees with a 2048 x 2048 rule to 1e-12 relative."""
    th = np.array([-1.2, math.log(1e10), math.log(1e8)])
    a = oracle.lf_etabar(th, _lf_consts(1024, 1024))
    b = oracle.lf_etabar(th, _lf_consts(2048, 2048))
    assert abs(a - b) / b < 1e-12


def test_etabar_is_detection_fraction_times_normaliser():
    """etabar(theta)/Z(theta) is the detected fraction of the population (eq. epdf denominator).
    Z = int_{L_low}^inf (L/L*)^beta e^{-L/L*} dL/L* = Gamma(beta+1, L_low/L*) (upper incomplete gamma,
    continued to beta+1 < 0 by Gamma(a, x) = (Gamma(a+1, x) - x^a e^-x)/a). The synthetic catalog sets
    F_th by Monte Carlo for a 30% detected fraction."""
    from paper_2105_08026_gb300 import synth
    beta, Ls, Ll, rmax = -1.2, 1e10, 1e8, 4000.0
    Fth = synth.solve_threshold(beta, Ls, Ll, rmax, 0.30, 0.2, seed=1002, m=2_000_000)
    c = oracle.lf_consts(0.2 * Fth, Fth, rmax, 1024, 1024)
    th = np.array([beta, math.log(Ls), math.log(Ll)])
    x = Ll / Ls
    a = beta + 1.0
    up = scipy.special.gammaincc(a + 1.0, x) * scipy.special.gamma(a + 1.0)
    Z = (up - x**a * math.exp(-x)) / a
    frac = oracle.lf_etabar(th, c) / Z
    assert abs(frac - 0.30) < 0.004


# -------------------------------------------------------------- models ------
def test_member_logdens_nn1_lf_known_values():
    """Hand-evaluated member log targets at points where the formulas reduce to simple numbers."""
    # NN1 at chi = y = mu: both quadratic terms vanish
    lp = oracle.member_logdens(oracle.NN1, [1.5], [0.7], [-10, 10], [1.5], [1.5, 0.3])
    assert lp[0] == 0.0
    # LF with Fhat = e^chi q (zero residual) and chi = ln L*: (beta+1)*0 - e^0 = -1
    r = 1.0
    q = 1.0 / (4 * math.pi)
    chi = math.log(1e10)
    lp = oracle.member_logdens(oracle.LF, [1e10 * q], [r], _lf_consts(), [chi], [-1.2, chi, math.log(1e8)])
    assert lp[0] == pytest.approx(-1.0, abs=1e-12)
    # LF off support (chi <= ln L_low) is -inf
    lp = oracle.member_logdens(oracle.LF, [1.0], [r], _lf_consts(), [math.log(1e8)], [-1.2, chi, math.log(1e8)])
    assert lp[0] == -math.inf
