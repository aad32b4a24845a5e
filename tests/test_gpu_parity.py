"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle, in lockstep.

FP64 acceptance bar:
- member and theta accept decisions identical at every (sweep, member), except where
  |Delta - ln u| < 1e-9 (a near tie, which rounding may flip);
- per-member log densities within 1e-12 relative (|a - b| <= 1e-12 max(1, |a|));
- the selection integral etabar(theta) within 1e-13 relative of the oracle's rule;
- theta rows, latents and RAM factors within 1e-12 relative.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2105_08026_gb300 import cudahm, synth

pytestmark = pytest.mark.gpu

REL = 1e-12       # latents, RAM factors, theta rows, per-member log densities
DELTA_REL = 1e-11  # member Delta = lp(Y) - lp(X): ~10 ulp of log targets of size ~1e3
NEAR_TIE = 1e-9


def _close(a, b, rel=REL):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    both_inf = np.isinf(a) & np.isinf(b) & (np.sign(a) == np.sign(b))
    err = np.abs(a - b)
    tol = rel * np.maximum(1.0, np.maximum(np.abs(a), np.abs(b)))
    return np.all(both_inf | (err <= tol)), float(np.max(np.where(both_inf, 0.0, err / tol), initial=0.0))


def _lockstep(model, y, aux, consts, theta0, scale, seed, chi0, sweeps, adapt_theta=True, block_threads=0):
    n = np.asarray(y).shape[0]
    s = cudahm.Sampler(model, n, theta_init=theta0, theta_prop_scale=scale, model_consts=consts, seed=seed,
                       trace_sweeps=sweeps, adapt_theta=adapt_theta, block_threads=block_threads)
    s.set_data(y, aux)
    s.set_chi(chi0)
    rows = s.run(0, sweeps)
    tr = s.trace(sweeps)
    ch = oracle.Chain(model, y, aux, consts, theta0, scale, seed, chi0, adapt_theta=adapt_theta)
    orows, otr = ch.run(0, sweeps, trace_sweeps=sweeps)
    return s, ch, rows, orows, tr, otr


def _check_lockstep(s, ch, rows, orows, tr, otr, d_atol=None):
    # member decisions
    diff = tr["acc"] != otr["acc"]
    if diff.any():
        k, i = np.argwhere(diff)[0]
        gap = abs(otr["delta"][k, i] - math.log(otr["u"][k, i]))
        assert gap < NEAR_TIE, f"member decision differs at sweep {k}, member {i}: |Delta - ln u| = {gap}"
        pytest.skip(f"near tie at sweep {k}, member {i}; chains legitimately diverge afterwards")
    assert np.array_equal(tr["u"], otr["u"]), "accept uniforms differ (RNG layout)"
    ok, worst = _close(tr["delta"], otr["delta"], rel=DELTA_REL)
    assert ok, f"member Delta differs: worst {worst:.3g} x tolerance"
    # theta decisions
    tdiff = tr["tacc"] != otr["tacc"]
    if tdiff.any():
        k = int(np.argwhere(tdiff)[0][0])
        gap = abs(otr["logalpha"][k] - math.log(otr["utheta"][k]))
        assert gap < NEAR_TIE, f"theta decision differs at sweep {k}: |log alpha - ln u| = {gap}"
        pytest.skip(f"theta near tie at sweep {k}")
    assert np.array_equal(tr["utheta"], otr["utheta"])
    ok, worst = _close(tr["theta_prop"], otr["theta_prop"])
    assert ok, f"theta proposals differ: {worst:.3g} x tol"
    # D and log alpha are sums over members of terms that each carry a few ulp of formula
    # rounding: a bound linear in N (1e-10 at N <= 1e4) keeps them 10x inside the near-tie band.
    # Models with a steeper member likelihood pass their own bound (see the caller).
    atol = (1e-10 if d_atol is None else d_atol) * max(1.0, s.n / 1e4)
    for key in ("D", "logalpha"):
        a, b = tr[key], otr[key]
        fin = np.isfinite(a) & np.isfinite(b)
        assert np.array_equal(np.isfinite(a), np.isfinite(b)), key
        assert np.array_equal(a[~fin], b[~fin]), key
        err = np.max(np.abs(a[fin] - b[fin]), initial=0.0)
        assert err <= atol, f"{key} differs by {err:.3g} > {atol:.3g}"
    # the selection integral at each traced proposal, against the oracle's rule at the same proposal
    # (the chains' theta' agree to the 1e-12 above; the integral is compared as arithmetic)
    eb = tr["etabar"]
    if ch.model in (oracle.LF, oracle.BB1):
        rule = oracle.lf_etabar if ch.model == oracle.LF else oracle.bb1_etabar
        ks = np.nonzero(eb > 0)[0]
        assert ks.size > 0
        ref = np.array([rule(tr["theta_prop"][k], ch.consts) for k in ks])
        assert np.all(np.abs(eb[ks] - ref) <= 1e-13 * ref), "selection integral differs"
    ok, worst = _close(rows, orows)
    assert ok, f"theta rows differ: {worst:.3g} x tol"
    chi, S = s.chi()
    ok, worst = _close(chi, ch.chi)
    assert ok, f"latents differ: {worst:.3g} x tol"
    ok, worst = _close(S, ch.S)
    assert ok, f"RAM factors differ: {worst:.3g} x tol"
    th, Sth = s.theta()
    ok, _ = _close(th, ch.theta)
    assert ok
    ok, _ = _close(Sth.reshape(-1), ch.S_theta)
    assert ok
    # per-member log targets of the device against the oracle's formula at the same (device) state
    lp = s.logdens(th)
    olp = oracle.member_logdens(ch.model, ch.y, ch.aux, ch.consts, chi, th)
    ok, worst = _close(lp, olp)
    assert ok, f"per-member log densities differ: {worst:.3g} x tol"


def test_nn1_lockstep_normal_normal_n1000():
    """Normal-normal, N = 1000, d = 1, mu = 2, tau = 0.8, sigma ~ U[0.5, 1.5]; 1000 sweeps."""
    data = synth.nn1_data(1000, seed=1001)
    theta0, scale, consts = synth.nn1_settings(data)
    out = _lockstep(oracle.NN1, data.y, data.sigma, consts, theta0, scale, 1, data.y.copy(), 1000)
    _check_lockstep(*out)


@pytest.mark.parametrize("n", [1, 37, 256, 2001])
def test_nn1_lockstep_ragged_sizes(n):
    data = synth.nn1_data(n, seed=50 + n)
    theta0, scale, consts = synth.nn1_settings(data)
    out = _lockstep(oracle.NN1, data.y, data.sigma, consts, theta0, scale, 3, data.y.copy(), 300)
    _check_lockstep(*out)


def test_nn1_lockstep_across_chunk_boundary():
    """More sweeps than one persistent launch holds (4096): the chain continues across launches."""
    data = synth.nn1_data(64, seed=9)
    theta0, scale, consts = synth.nn1_settings(data)
    out = _lockstep(oracle.NN1, data.y, data.sigma, consts, theta0, scale, 4, data.y.copy(), 4200)
    _check_lockstep(*out)


def test_lf_lockstep_small_rule():
    """Luminosity model, N = 3000 (several blocks and a ragged tail), 256 x 256 rule, 120 sweeps."""
    data = synth.lf_data(3000, seed=11)
    theta0, scale, consts = synth.lf_settings(data, nL=256, nr=256)
    chi0 = synth.lf_chi_init(data, theta0)
    out = _lockstep(oracle.LF, data.fhat, data.r, consts, theta0, scale, 2, chi0, 120)
    _check_lockstep(*out)


def test_lf_etabar_matches_oracle_rule():
    data = synth.lf_data(1000, seed=12)
    theta0, scale, consts = synth.lf_settings(data)  # 1024 x 1024
    s = cudahm.Sampler(cudahm.LF, 1000, theta_init=theta0, theta_prop_scale=scale, model_consts=consts)
    s.set_data(data.fhat, data.r)
    # the last rows reach the ends of the tabulated inner sum: outer nodes down to L ~ 1e-9 L*
    # (H constant to rounding below the table) and up to ~1e4 L* (every pair past x = 8.5)
    for dth in ([0, 0, 0], [0.05, 0.1, -0.2], [-0.3, -0.5, 0.4], [0.25, 1.0, 1.5], [-0.7, 5.0, -20.0],
                [0.6, -6.0, -3.0], [-0.7, 9.0, 4.4]):
        th = theta0 + np.array(dth)
        g = s.etabar(th)
        o = oracle.lf_etabar(th, consts)
        assert abs(g - o) <= 1e-13 * o, (th, g, o, (g - o) / o)


def test_detection_efficiency_table_matches_oracle():
    """The device's normal-CDF table (local Taylor series) against the oracle's erfc-based Phi,
    on a dense grid, at interval centres and edges, and at the ends of the table."""
    consts = oracle.lf_consts(2.0, 10.0, 4000.0, 8, 8)
    s = cudahm.Sampler(cudahm.LF, 1, theta_init=[-1.2, 23.0, 18.4], theta_prop_scale=[0.01] * 3,
                       model_consts=consts)
    c = np.arange(265) / 16.0 - 8.0
    x = np.concatenate([np.linspace(-12.0, 12.0, 200_001), c, c + 1 / 32, c - 1 / 32,
                        [-8.0, -8.0 - 1e-12, 8.5, 8.5 + 1e-12, 0.0, -1e-300, 1e-300]])
    F = 10.0 + 2.0 * x
    got = s.detection(F)
    ref = oracle.lf_detection(F, consts)
    err = np.abs(got - ref)
    assert np.all(err <= 2.5e-16 + 2e-15 * ref), (x[np.argmax(err)], err.max())


def test_lf_full_size_lockstep_n300000():
    """The benchmark workload (N = 3e5 detected objects, 1024 x 1024 rule) in the benchmark's launch
    shape, 6 sweeps in lockstep with the oracle over every member."""
    data = synth.lf_data(300_000, seed=1002)
    theta0, scale, consts = synth.lf_settings(data)
    chi0 = synth.lf_chi_init(data, theta0)
    out = _lockstep(oracle.LF, data.fhat, data.r, consts, theta0, scale, 2, chi0, 6)
    st = out[0].stats()
    assert st.objects_per_thread >= 1 and st.grid_blocks >= 1
    _check_lockstep(*out)


def test_default_start_matches_recipe():
    data = synth.lf_data(500, seed=13)
    theta0, scale, consts = synth.lf_settings(data)
    s = cudahm.Sampler(cudahm.LF, 500, theta_init=theta0, theta_prop_scale=scale, model_consts=consts)
    s.set_data(data.fhat, data.r)
    chi, S = s.chi()
    ok, worst = _close(chi, synth.lf_chi_init(data, theta0), rel=1e-14)
    assert ok, worst
    assert np.all(S == 1.0)


def test_run_split_equals_whole_and_checkpoint_resume():
    data = synth.lf_data(5000, seed=14)
    theta0, scale, consts = synth.lf_settings(data, nL=128, nr=128)
    mk = lambda: cudahm.Sampler(cudahm.LF, 5000, theta_init=theta0, theta_prop_scale=scale,
                                model_consts=consts, seed=77)
    a, b, c = mk(), mk(), mk()
    for x in (a, b, c):
        x.set_data(data.fhat, data.r)
    ra = a.run(0, 400)
    rb = np.concatenate([b.run(0, 150), b.run(0, 250)])
    assert np.array_equal(ra, rb)
    assert np.array_equal(a.chi()[0], b.chi()[0]) and np.array_equal(a.chi()[1], b.chi()[1])
    # checkpoint after 150 sweeps, restore into a fresh handle, continue
    c.run(0, 150)
    blob = c.checkpoint()
    d = mk()
    d.set_data(data.fhat, data.r)
    d.restore(blob)
    rd = d.run(0, 250)
    assert np.array_equal(rd, ra[150:])
    assert np.array_equal(d.chi()[0], a.chi()[0])


def test_barrier_timeout_reports_error_and_context_survives():
    """A block that never arrives at the grid barrier: the other blocks give up after the bound,
    the run returns ETIMEOUT, and the CUDA context stays usable."""
    data = synth.nn1_data(4000, seed=15)
    theta0, scale, consts = synth.nn1_settings(data)
    s = cudahm.Sampler(cudahm.NN1, 4000, theta_init=theta0, theta_prop_scale=scale, model_consts=consts,
                       barrier_timeout_ns=200_000_000, debug_skip_barrier_cta=1)
    s.set_data(data.y, data.sigma)
    chi_before = s.chi()[0]
    with pytest.raises(cudahm.CudahmError) as ei:
        s.run(0, 10)
    assert ei.value.code == cudahm.ETIMEOUT
    assert np.array_equal(s.chi()[0], chi_before)  # state untouched by the failed run
    ok = cudahm.Sampler(cudahm.NN1, 4000, theta_init=theta0, theta_prop_scale=scale, model_consts=consts)
    ok.set_data(data.y, data.sigma)
    assert ok.run(0, 5).shape == (5, 2)


def test_torch_allocator_and_stream():
    torch = pytest.importorskip("torch")
    data = synth.nn1_data(3000, seed=16)
    theta0, scale, consts = synth.nn1_settings(data)
    st = torch.cuda.Stream()
    s = cudahm.Sampler(cudahm.NN1, 3000, theta_init=theta0, theta_prop_scale=scale, model_consts=consts, seed=5,
                       use_torch_allocator=True, stream=st.cuda_stream)
    s.set_data(data.y, data.sigma)
    r1 = s.run(10, 50)
    s2 = cudahm.Sampler(cudahm.NN1, 3000, theta_init=theta0, theta_prop_scale=scale, model_consts=consts, seed=5)
    s2.set_data(data.y, data.sigma)
    assert np.array_equal(r1, s2.run(10, 50))


def test_invalid_calls():
    data = synth.nn1_data(10, seed=17)
    theta0, scale, consts = synth.nn1_settings(data)
    s = cudahm.Sampler(cudahm.NN1, 10, theta_init=theta0, theta_prop_scale=scale, model_consts=consts)
    with pytest.raises(cudahm.CudahmError) as ei:
        s.run(0, 5)
    assert ei.value.code == cudahm.ESTATE
    bad = data.sigma.copy()
    bad[3] = -1.0
    with pytest.raises(cudahm.CudahmError) as ei:
        s.set_data(data.y, bad)
    assert ei.value.code == cudahm.EINVAL
    s.set_data(data.y, data.sigma)
    with pytest.raises(cudahm.CudahmError) as ei:
        s.run(0, 5, thin=0)
    assert ei.value.code == cudahm.EINVAL


def test_restore_rejects_another_layout_version_or_config():
    data = synth.nn1_data(500, seed=18)
    theta0, scale, consts = synth.nn1_settings(data)
    mk = lambda seed: cudahm.Sampler(cudahm.NN1, 500, theta_init=theta0, theta_prop_scale=scale,
                                     model_consts=consts, seed=seed)
    a, b, c = mk(3), mk(3), mk(4)
    for x in (a, b, c):
        x.set_data(data.y, data.sigma)
    a.run(0, 20)
    blob = bytearray(a.checkpoint())
    b.restore(bytes(blob))  # same configuration and layout: accepted
    assert np.array_equal(b.chi()[0], a.chi()[0])
    with pytest.raises(cudahm.CudahmError) as ei:  # another seed: another chain
        c.restore(bytes(blob))
    assert ei.value.code == cudahm.EINVAL
    blob[8:16] = (1).to_bytes(8, "little", signed=True)  # layout version 1
    with pytest.raises(cudahm.CudahmError) as ei:
        b.restore(bytes(blob))
    assert ei.value.code == cudahm.EINVAL
