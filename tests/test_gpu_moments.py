"""GPU parity of the per-member running moments of the latents (keep_chi_moments).

Against the oracle, in lockstep: the device chain and the oracle's chain run the same thinned
runs with moments on; the member and theta decisions must agree (as in the other lockstep
tests), and then the moments must agree to the precision of the latents themselves. Each kept
latent agrees to REL = 1e-12 relative, so
  |mean - mean_o| <= REL max(1, |mean|)
  |var - var_o|   <= 8 REL max(1, |mean|) sd + REL var + 4 (REL max(1, |mean|))^2
(the deviations x - mean carry twice the latents' error; var sums their squares over m - 1).

Properties that hold at any size: run(a) + run(b) equals run(a + b) bit for bit, across the
launch boundaries of long runs (two moment buffers, committed at each launch's end);
checkpoint and restore carry the moments; a batched run gives each population the moments it
gets alone; a run that fails commits nothing; the FP32 form's moments are the mean and the
sample variance of its own latents at the kept sweeps.
"""
import numpy as np
import pytest

import oracle
from paper_2105_08026_gb300 import cudahm, synth

from test_gpu_parity import _check_lockstep

pytestmark = pytest.mark.gpu

REL = 1e-12


def _pair(model, y, aux, consts, theta0, scale, seed, chi0, T):
    n = np.asarray(y).shape[0]
    s = cudahm.Sampler(model, n, theta_init=theta0, theta_prop_scale=scale, model_consts=consts, seed=seed,
                       trace_sweeps=T, keep_chi_moments=True)
    s.set_data(y, aux)
    s.set_chi(chi0)
    ch = oracle.Chain(model, y, aux, consts, theta0, scale, seed, chi0, keep_chi_moments=True)
    return s, ch


def _run_both(s, ch, n_burn, n_iter, thin, d_atol=None):
    T = n_burn + n_iter
    rows = s.run(n_burn, n_iter, thin)
    tr = s.trace(T)
    orows, otr = ch.run(n_burn, n_iter, thin, trace_sweeps=T)
    _check_lockstep(s, ch, rows, orows, tr, otr, d_atol=d_atol)


def _check_moments(s, ch):
    m, v, c = s.chi_moments()
    om, ov, oc = ch.moments()
    assert c == oc and c > 0
    sc = np.maximum(1.0, np.abs(om))
    err = np.abs(m - om)
    assert np.all(err <= REL * sc), f"means differ: worst {np.max(err / (REL * sc)):.3g} x tol"
    tol = 8 * REL * sc * np.sqrt(ov) + REL * ov + 4 * (REL * sc) ** 2
    err = np.abs(v - ov)
    assert np.all(err <= tol), f"variances differ: worst {np.max(err / tol):.3g} x tol"


def test_nn1_moments_lockstep():
    data = synth.nn1_data(1000, seed=1001)
    theta0, scale, consts = synth.nn1_settings(data)
    s, ch = _pair(oracle.NN1, data.y, data.sigma, consts, theta0, scale, 1, data.y.copy(), 210)
    _run_both(s, ch, 10, 200, 5)
    _check_moments(s, ch)
    _run_both(s, ch, 0, 60, 3)  # moments continue over the next run's kept sweeps
    _check_moments(s, ch)


def test_lf_moments_lockstep():
    data = synth.lf_data(3000, seed=11)
    theta0, scale, consts = synth.lf_settings(data, nL=256, nr=256)
    s, ch = _pair(oracle.LF, data.fhat, data.r, consts, theta0, scale, 2, synth.lf_chi_init(data, theta0), 65)
    _run_both(s, ch, 5, 60, 2)
    _check_moments(s, ch)


def test_bb1_moments_lockstep():
    data = synth.bb1_data(2000, seed=21)
    theta0, scale, consts = synth.bb1_settings(data, nL=128, nr=128)
    s, ch = _pair(oracle.BB1, data.fhat, data.r, consts, theta0, scale, 7, synth.bb1_chi_init(data), 80)
    _run_both(s, ch, 20, 60, 1, d_atol=1e-9)
    _check_moments(s, ch)


def test_mvn3_moments_lockstep_streamed():
    """d = 3: member state streams through the batched kernel; moments per component."""
    data = synth.mvn3_data(1500, seed=1003)
    theta0, scale, consts = synth.mvn3_settings(data)
    s, ch = _pair(oracle.MVN3, data.y, data.s, consts, theta0, scale, 3, data.y.copy(), 43)
    _run_both(s, ch, 3, 40, 3)
    _check_moments(s, ch)


def test_lf_full_size_moments_lockstep_n300000():
    """The benchmark workload (N = 3e5, 1024 x 1024 rule) in the benchmark's launch shape."""
    data = synth.lf_data(300_000, seed=1002)
    theta0, scale, consts = synth.lf_settings(data)
    s, ch = _pair(oracle.LF, data.fhat, data.r, consts, theta0, scale, 2, synth.lf_chi_init(data, theta0), 6)
    _run_both(s, ch, 2, 4, 1)
    _check_moments(s, ch)


def _kept(n_burn, n_iter, thin):
    return [q for q in range(n_burn + n_iter) if q >= n_burn and (q - n_burn + 1) % thin == 0]


@pytest.mark.parametrize("model", ["lf", "mvn3"])
def test_fp32_moments_are_mean_and_variance_of_its_latents(model):
    """FP32 bulk form (resident LF kernel; streamed d = 3 kernel): the moments equal numpy's
    mean and var(ddof=1) of the latents of a twin chain read after each kept sweep."""
    if model == "lf":
        data = synth.lf_data(2500, seed=31)
        theta0, scale, consts = synth.lf_settings(data, nL=128, nr=128)
        y, aux, M = data.fhat, data.r, cudahm.LF
    else:
        data = synth.mvn3_data(2500, seed=32)
        theta0, scale, consts = synth.mvn3_settings(data)
        y, aux, M = data.y, data.s, cudahm.MVN3
    mk = lambda keep: cudahm.Sampler(M, 2500, theta_init=theta0, theta_prop_scale=scale, model_consts=consts,
                                     seed=12, precision=cudahm.FP32, keep_chi_moments=keep)
    a, b = mk(True), mk(False)
    a.set_data(y, aux)
    b.set_data(y, aux)
    n_burn, n_iter, thin = 4, 30, 3
    a.run(n_burn, n_iter, thin)
    kept = set(_kept(n_burn, n_iter, thin))
    snaps = []
    for q in range(n_burn + n_iter):
        b.run(0, 1)
        if q in kept:
            snaps.append(b.chi()[0].reshape(2500, -1))
    snaps = np.array(snaps)
    m, v, c = a.chi_moments()
    assert c == snaps.shape[0] == 10
    ref_m, ref_v = snaps.mean(axis=0), snaps.var(axis=0, ddof=1)
    sc = np.maximum(1.0, np.abs(ref_m))
    assert np.all(np.abs(m - ref_m) <= 1e-13 * sc)
    assert np.all(np.abs(v - ref_v) <= 1e-12 * (ref_v + sc * np.sqrt(ref_v)) + 1e-300)


def test_moments_split_runs_and_launch_boundaries_bit_identical():
    """Runs longer than one launch (4096 sweeps), split at other places: identical moments."""
    data = synth.nn1_data(300, seed=33)
    theta0, scale, consts = synth.nn1_settings(data)
    mk = lambda: cudahm.Sampler(cudahm.NN1, 300, theta_init=theta0, theta_prop_scale=scale, model_consts=consts,
                                seed=9, keep_chi_moments=True)
    a, b = mk(), mk()
    a.set_data(data.y, data.sigma)
    b.set_data(data.y, data.sigma)
    a.run(100, 8900, 1)
    b.run(100, 3000, 1)
    b.run(0, 5900, 1)
    ma, va, ca = a.chi_moments()
    mb, vb, cb = b.chi_moments()
    assert ca == cb == 8900
    assert np.array_equal(ma, mb) and np.array_equal(va, vb)
    assert np.array_equal(a.chi()[0], b.chi()[0])


def test_moments_checkpoint_restore():
    data = synth.lf_data(2000, seed=34)
    theta0, scale, consts = synth.lf_settings(data, nL=128, nr=128)
    mk = lambda: cudahm.Sampler(cudahm.LF, 2000, theta_init=theta0, theta_prop_scale=scale, model_consts=consts,
                                seed=10, keep_chi_moments=True)
    a, c, d = mk(), mk(), mk()
    for x in (a, c, d):
        x.set_data(data.fhat, data.r)
    a.run(3, 40, 2)
    a.run(0, 30, 3)
    c.run(3, 40, 2)
    blob = c.checkpoint()
    d.restore(blob)
    assert d.chi_moments()[2] == 20
    d.run(0, 30, 3)
    ma, va, ca = a.chi_moments()
    md, vd, cd = d.chi_moments()
    assert ca == cd == 30
    assert np.array_equal(ma, md) and np.array_equal(va, vd)


def test_batched_run_gives_each_population_its_own_moments():
    nd = synth.nn1_data(500, seed=35)
    ld = synth.lf_data(800, seed=36)
    t1, s1, c1 = synth.nn1_settings(nd)
    t2, s2, c2 = synth.lf_settings(ld, nL=64, nr=64)

    def pair():
        a = cudahm.Sampler(cudahm.NN1, 500, theta_init=t1, theta_prop_scale=s1, model_consts=c1, seed=3,
                           keep_chi_moments=True)
        b = cudahm.Sampler(cudahm.LF, 800, theta_init=t2, theta_prop_scale=s2, model_consts=c2, seed=4,
                           keep_chi_moments=True)
        a.set_data(nd.y, nd.sigma)
        b.set_data(ld.fhat, ld.r)
        return a, b

    a1, b1 = pair()
    a2, b2 = pair()
    cudahm.batch_run([a1, b1], 5, 40, 2)
    a2.run(5, 40, 2)
    b2.run(5, 40, 2)
    for x, y in ((a1, a2), (b1, b2)):
        mx, vx, cx = x.chi_moments()
        my, vy, cy = y.chi_moments()
        assert cx == cy == 20
        assert np.array_equal(mx, my) and np.array_equal(vx, vy)


def test_failed_run_commits_no_moments():
    """A block that never arrives at the grid barrier: the run fails with ETIMEOUT after the
    bound, and the moments it wrote for its first (kept) sweep are not committed."""
    data = synth.nn1_data(4000, seed=15)
    theta0, scale, consts = synth.nn1_settings(data)
    s = cudahm.Sampler(cudahm.NN1, 4000, theta_init=theta0, theta_prop_scale=scale, model_consts=consts,
                       barrier_timeout_ns=200_000_000, debug_skip_barrier_cta=1, keep_chi_moments=True)
    s.set_data(data.y, data.sigma)
    with pytest.raises(cudahm.CudahmError) as ei:
        s.run(0, 10)
    assert ei.value.code == cudahm.ETIMEOUT
    m, v, c = s.chi_moments()
    assert c == 0 and np.all(m == 0.0) and np.all(v == 0.0)


def test_moment_calls_without_the_option():
    data = synth.nn1_data(50, seed=37)
    theta0, scale, consts = synth.nn1_settings(data)
    s = cudahm.Sampler(cudahm.NN1, 50, theta_init=theta0, theta_prop_scale=scale, model_consts=consts)
    s.set_data(data.y, data.sigma)
    s.run(0, 5)
    with pytest.raises(cudahm.CudahmError) as ei:
        s.chi_moments()
    assert ei.value.code == cudahm.ESTATE
    t = cudahm.Sampler(cudahm.NN1, 50, theta_init=theta0, theta_prop_scale=scale, model_consts=consts,
                       keep_chi_moments=True)
    t.set_data(data.y, data.sigma)
    t.run(5, 0)  # burn-in only: nothing kept
    m, v, c = t.chi_moments()
    assert c == 0 and np.all(m == 0.0)
    t.run(0, 1)
    m, v, c = t.chi_moments()
    assert c == 1 and np.array_equal(m.reshape(-1), t.chi()[0]) and np.all(v == 0.0)
