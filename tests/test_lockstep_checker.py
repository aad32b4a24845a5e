"""The lockstep comparison rules of the parity tests, checked on the CPU.

An oracle chain is compared with an identical twin through the same function the GPU parity
tests use; disagreements are planted in the twin's trace (the side that stands in for the
device). The rules: a member near tie masks that member only, a theta near tie ends the
comparison at its sweep, D is compared up to the first member divergence, and anything outside
the near-tie band or the tolerances fails.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2105_08026_gb300 import synth

from lockstep import D_REL, NEAR_TIE, _check_lockstep, d_tolerance

T = 40


class _Twin:
    """The device-side interface that the comparison reads, over an oracle chain."""

    def __init__(self, ch):
        self.ch = ch
        self.n = ch.n

    def chi(self):
        return self.ch.chi.copy(), self.ch.S.copy()

    def theta(self):
        return self.ch.theta.copy(), self.ch.S_theta.reshape(self.ch.p, self.ch.p).copy()

    def logdens(self, th):
        return oracle.member_logdens(self.ch.model, self.ch.y, self.ch.aux, self.ch.consts, self.ch.chi, th)


def _pair():
    data = synth.nn1_data(200, seed=5)
    theta0, scale, consts = synth.nn1_settings(data)
    mk = lambda: oracle.Chain(oracle.NN1, data.y, data.sigma, consts, theta0, scale, 3, data.y.copy())
    a, b = mk(), mk()
    ra, ta = a.run(0, T, trace_sweeps=T)
    rb, tb = b.run(0, T, trace_sweeps=T)
    return _Twin(a), b, ra, rb, ta, tb


def test_identical_chains_compare_over_every_sweep():
    out = _check_lockstep(*_pair())
    assert out["member_ties"] == [] and out["theta_tie"] is None
    assert out["members_compared_to"] == T and out["theta_compared_to"] == T and out["D_compared_to"] == T


def test_member_near_tie_masks_that_member_only():
    s, ch, ra, rb, ta, tb = _pair()
    k, i = 17, 33
    lnu = math.log(tb["u"][k, i])
    ta["delta"][k, i] = tb["delta"][k, i] = lnu + 0.3 * NEAR_TIE
    ta["acc"][k, i] ^= 1
    # member i's chain diverges afterwards, and D with it
    ta["acc"][k + 1:, i] ^= 1
    ta["delta"][k + 1:, i] += 0.5
    ta["D"][k:] += 1e-3
    ta["logalpha"][k:] += 1e-3
    s.ch.chi[i] += 0.25
    out = _check_lockstep(s, ch, ra, rb, ta, tb)
    assert out["member_ties"] == [(k, i)]
    assert out["D_compared_to"] == k and out["members_compared_to"] == T


def test_member_decision_outside_the_band_fails():
    s, ch, ra, rb, ta, tb = _pair()
    k, i = 11, 7
    ta["acc"][k, i] ^= 1
    if abs(tb["delta"][k, i] - math.log(tb["u"][k, i])) < NEAR_TIE:
        pytest.skip("the chosen decision happens to be a near tie")
    with pytest.raises(AssertionError, match="member decision differs"):
        _check_lockstep(s, ch, ra, rb, ta, tb)


def test_member_delta_error_fails():
    s, ch, ra, rb, ta, tb = _pair()
    ta["delta"][5, 3] += 1e-9 * max(1.0, abs(tb["delta"][5, 3]))
    with pytest.raises(AssertionError, match="member Delta differs"):
        _check_lockstep(s, ch, ra, rb, ta, tb)


def test_d_error_beyond_tolerance_fails():
    s, ch, ra, rb, ta, tb = _pair()
    k = int(np.nonzero(np.isfinite(tb["D"]))[0][9])
    ta["D"][k] += 2 * d_tolerance(s.n) + 2 * D_REL * abs(tb["D"][k])
    with pytest.raises(AssertionError, match="D differs"):
        _check_lockstep(s, ch, ra, rb, ta, tb)


def test_log_alpha_error_beyond_tolerance_fails():
    s, ch, ra, rb, ta, tb = _pair()
    k = int(np.nonzero(np.isfinite(tb["logalpha"]))[0][5])
    ta["logalpha"][k] += 2 * d_tolerance(s.n)
    with pytest.raises(AssertionError, match="logalpha differs"):
        _check_lockstep(s, ch, ra, rb, ta, tb)


def test_theta_near_tie_ends_the_comparison_there():
    s, ch, ra, rb, ta, tb = _pair()
    k = 21
    lnu = math.log(tb["utheta"][k])
    ta["logalpha"][k] = tb["logalpha"][k] = lnu + 0.5 * NEAR_TIE
    ta["tacc"][k] ^= 1
    # everything after the tie may differ
    ta["theta_prop"][k + 1:] += 0.1
    ta["tacc"][k + 1:] ^= 1
    ta["acc"][k + 2:] ^= 1
    ta["delta"][k + 2:] += 1.0
    ta["D"][k + 1:] += 1.0
    s.ch.chi += 1.0
    s.ch.theta += 1.0
    out = _check_lockstep(s, ch, ra, rb, ta, tb)
    assert out["theta_tie"] == k and out["theta_compared_to"] == k
    assert out["members_compared_to"] == k + 1 and out["D_compared_to"] == k + 1


def test_theta_decision_outside_the_band_fails():
    s, ch, ra, rb, ta, tb = _pair()
    k = 13
    if abs(tb["logalpha"][k] - math.log(tb["utheta"][k])) < NEAR_TIE:
        pytest.skip("the chosen decision happens to be a near tie")
    ta["tacc"][k] ^= 1
    with pytest.raises(AssertionError, match="theta decision differs"):
        _check_lockstep(s, ch, ra, rb, ta, tb)


def test_theta_proposal_error_fails():
    s, ch, ra, rb, ta, tb = _pair()
    ta["theta_prop"][4, 1] *= 1 + 1e-10
    with pytest.raises(AssertionError, match="theta proposals differ"):
        _check_lockstep(s, ch, ra, rb, ta, tb)


def test_final_latent_error_fails():
    s, ch, ra, rb, ta, tb = _pair()
    s.ch.chi[3] *= 1 + 1e-10
    with pytest.raises(AssertionError, match="latents differ"):
        _check_lockstep(s, ch, ra, rb, ta, tb)
