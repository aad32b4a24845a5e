"""GPU parity of the paper's BB1 luminosity-function model (Sec. 5.1-5.2, App. B) against the oracle.

FP64 lockstep bar as for the other models (identical member and theta decisions except near ties,
log targets, latents, RAM factors, theta within 1e-12 relative), the selection integral (with the
flux-dependent sigma(F) inside Phi) within 1e-13 relative of the oracle's rule, and the detection
efficiency table against the oracle's erfc.

D and log alpha get a bound of 1e-9 max(1, N/1e4) instead of 1e-10: the member likelihood is
steep (a 1% flux error, alpha = 0.01, gives curvatures up to ~1/alpha^2 in ln L), so the
ulp-level drift of the two chains' latents (below 1e-14 relative after hundreds of sweeps, checked
by the latents' 1e-12 bound) moves the sums by ~1e-10; from identical states one sweep agrees to
~2e-13. The bound stays inside the near-tie band of 1e-9 per 1e4 members. Sizes: N = 2000 with a 128 x 128 rule for 300 sweeps,
and the paper's case-study size N = 1e5 with the 1024 x 1024 rule for the first sweeps."""
import numpy as np
import pytest

import oracle
from paper_2105_08026_gb300 import cudahm, synth

from test_gpu_parity import _check_lockstep, _lockstep

pytestmark = pytest.mark.gpu


def test_bb1_lockstep_small_rule():
    data = synth.bb1_data(2000, seed=21)
    theta0, scale, consts = synth.bb1_settings(data, nL=128, nr=128)
    out = _lockstep(oracle.BB1, data.fhat, data.r, consts, theta0, scale, 7, synth.bb1_chi_init(data), 300)
    _check_lockstep(*out, d_atol=1e-9)


def test_bb1_full_size_lockstep_n100000():
    """The paper's case study size (N = 1e5 detected galaxies), 1024 x 1024 rule, 4 sweeps."""
    data = synth.bb1_data(100_000, seed=1004)
    theta0, scale, consts = synth.bb1_settings(data)
    out = _lockstep(oracle.BB1, data.fhat, data.r, consts, theta0, scale, 4, synth.bb1_chi_init(data), 4)
    _check_lockstep(*out, d_atol=1e-9)


def test_bb1_lockstep_1000_sweeps_full_rule():
    """The paper's model with the full 1024 x 1024 rule (sigma(F) in every pair), 1000 sweeps in
    lockstep (N = 5000: the oracle's cost is the rule's 2^20 pairs per sweep)."""
    data = synth.bb1_data(5000, seed=1006)
    theta0, scale, consts = synth.bb1_settings(data)
    out = _lockstep(oracle.BB1, data.fhat, data.r, consts, theta0, scale, 8, synth.bb1_chi_init(data), 1000)
    _check_lockstep(*out, d_atol=1e-9)


def test_bb1_etabar_and_detection_match_oracle():
    data = synth.bb1_data(500, seed=22)
    theta0, scale, consts = synth.bb1_settings(data)
    s = cudahm.Sampler(cudahm.BB1, 500, theta_init=theta0, theta_prop_scale=scale, model_consts=consts)
    s.set_data(data.fhat, data.r)
    for dth in ([0, 0, 0], [0.05, 0.1, -0.2], [-0.3, -0.5, 0.4], [0.25, 1.0, 1.5], [-0.45, -5.0, 6.0],
                [0.4, 2.0, 0.5]):
        th = theta0 + np.array(dth)
        g, o = s.etabar(th), oracle.bb1_etabar(th, consts)
        assert abs(g - o) <= 1e-13 * o, (dth, g, o)
    Fth = data.F_th
    F = np.concatenate([np.linspace(-3.0, 40.0, 20001) * Fth, [Fth, 0.0, 1e3 * Fth]])
    got, ref = s.detection(F), oracle.bb1_detection(F, consts)
    assert np.all(np.abs(got - ref) <= 2.5e-16 + 2e-15 * ref), np.max(np.abs(got - ref))


def test_bb1_split_checkpoint_and_batch_equal_alone():
    data = synth.bb1_data(3000, seed=23)
    theta0, scale, consts = synth.bb1_settings(data, nL=96, nr=200)
    mk = lambda: cudahm.Sampler(cudahm.BB1, 3000, theta_init=theta0, theta_prop_scale=scale,
                                model_consts=consts, seed=9)
    a, b, c = mk(), mk(), mk()
    for x in (a, b, c):
        x.set_data(data.fhat, data.r)
    ra = a.run(0, 301)
    assert np.array_equal(ra, np.concatenate([b.run(0, 101), b.run(0, 200)]))
    c.run(0, 101)
    blob = c.checkpoint()
    d = mk()
    d.set_data(data.fhat, data.r)
    d.restore(blob)
    assert np.array_equal(d.run(0, 200), ra[101:])
    # in one batched launch with NN1 and LF populations: the same chain
    n1 = synth.nn1_data(700, seed=24)
    t1, s1, c1 = synth.nn1_settings(n1)
    l1 = synth.lf_data(900, seed=25)
    t2, s2, c2 = synth.lf_settings(l1, nL=64, nr=128)
    e = mk()
    e.set_data(data.fhat, data.r)
    p1 = cudahm.Sampler(cudahm.NN1, 700, theta_init=t1, theta_prop_scale=s1, model_consts=c1, seed=3)
    p1.set_data(n1.y, n1.sigma)
    p2 = cudahm.Sampler(cudahm.LF, 900, theta_init=t2, theta_prop_scale=s2, model_consts=c2, seed=4)
    p2.set_data(l1.fhat, l1.r)
    rows, _ = cudahm.batch_run([p1, e, p2], 0, 301)
    assert np.array_equal(rows[1], ra)
    assert np.array_equal(e.chi()[0], a.chi()[0])
