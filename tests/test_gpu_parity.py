"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle, in lockstep.

FP64 acceptance bar:
- member and theta accept decisions identical at every (sweep, member), except where
  |Delta - ln u| < 1e-9 (a near tie, which rounding may flip); after a member's near tie that
  member is masked and the others are still compared, a theta near tie ends the comparison at
  that sweep (both reported, never skipped);
- D and log alpha_theta within 1e-10 sqrt(N/1e4) absolute (below the near-tie band);
- per-member log densities within 1e-12 relative (|a - b| <= 1e-12 max(1, |a|));
- the selection integral etabar(theta) within 1e-13 relative of the oracle's rule;
- theta rows, latents and RAM factors within 1e-12 relative.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2105_08026_gb300 import cudahm, synth

from lockstep import DELTA_REL, NEAR_TIE, REL, _check_lockstep, _close, _lockstep, d_tolerance  # noqa: F401

pytestmark = pytest.mark.gpu


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


def test_lf_lockstep_1000_sweeps_full_rule_n10000():
    """Luminosity model, N = 1e4, the full 1024 x 1024 rule, 1000 sweeps in lockstep: the RAM
    adaptation's later steps of every member and of theta, every decision compared."""
    data = synth.lf_data(10_000, seed=1005)
    theta0, scale, consts = synth.lf_settings(data)
    chi0 = synth.lf_chi_init(data, theta0)
    out = _lockstep(oracle.LF, data.fhat, data.r, consts, theta0, scale, 2, chi0, 1000)
    _check_lockstep(*out)


def test_lf_lockstep_across_launch_boundary():
    """Luminosity model, 4200 sweeps: the chain continues across the boundary of a persistent
    launch (4096 sweeps), in lockstep (N = 2000, 128 x 128 rule)."""
    data = synth.lf_data(2000, seed=1007)
    theta0, scale, consts = synth.lf_settings(data, nL=128, nr=128)
    chi0 = synth.lf_chi_init(data, theta0)
    out = _lockstep(oracle.LF, data.fhat, data.r, consts, theta0, scale, 6, chi0, 4200)
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
    blob[8:16] = (2).to_bytes(8, "little", signed=True)  # layout version 2
    with pytest.raises(cudahm.CudahmError) as ei:
        b.restore(bytes(blob))
    assert ei.value.code == cudahm.EINVAL


# checkpoint layout (version 3): 10 header words, then ChainState: theta[9], S_theta[81], etabar,
# sweeps, member_acc, theta_acc, rows (8 bytes each), mcur, mom_sel (4 bytes each), mom_n, ...
_HDR = 80
_OFF_SWEEPS = _HDR + 8 * (9 + 81 + 1)
_OFF_MCUR = _HDR + 8 * (9 + 81 + 5)
_OFF_MOMSEL = _OFF_MCUR + 4


def test_restore_rejects_a_corrupted_chain_state():
    """Fields that index device buffers or size launches are checked before anything is copied."""
    data = synth.nn1_data(500, seed=18)
    theta0, scale, consts = synth.nn1_settings(data)
    mk = lambda: cudahm.Sampler(cudahm.NN1, 500, theta_init=theta0, theta_prop_scale=scale,
                                model_consts=consts, seed=3, keep_chi_moments=True)
    a, b = mk(), mk()
    for x in (a, b):
        x.set_data(data.y, data.sigma)
    a.run(0, 20)
    good = bytes(a.checkpoint())
    assert int.from_bytes(good[_OFF_SWEEPS:_OFF_SWEEPS + 8], "little") == 20  # the layout assumed here
    chi_before = b.chi()[0]
    for off, width, val in ((_OFF_MOMSEL, 4, 2), (_OFF_MOMSEL, 4, -1), (_OFF_MCUR, 4, 7),
                            (_OFF_SWEEPS, 8, -5), (_OFF_SWEEPS, 8, 1 << 33)):
        blob = bytearray(good)
        blob[off:off + width] = val.to_bytes(width, "little", signed=True)
        with pytest.raises(cudahm.CudahmError) as ei:
            b.restore(bytes(blob))
        assert ei.value.code == cudahm.EINVAL, (off, val)
    blob = bytearray(good)
    blob[_HDR:_HDR + 8] = np.array([np.nan]).tobytes()  # theta[0]
    with pytest.raises(cudahm.CudahmError):
        b.restore(bytes(blob))
    assert np.array_equal(b.chi()[0], chi_before)  # nothing was copied
    b.restore(good)
    assert np.array_equal(b.chi()[0], a.chi()[0])


def test_restore_rejects_other_model_constants_or_form():
    """A checkpoint continues only the chain it was taken from: another selection rule, another
    precision or another moments setting is rejected."""
    data = synth.lf_data(800, seed=19)
    theta0, scale, consts = synth.lf_settings(data, nL=64, nr=64)
    mk = lambda c, **kw: cudahm.Sampler(cudahm.LF, 800, theta_init=theta0, theta_prop_scale=scale,
                                        model_consts=c, seed=3, **kw)
    a = mk(consts)
    a.set_data(data.fhat, data.r)
    a.run(0, 10)
    blob = a.checkpoint()
    other = consts.copy()
    other[3] = 128  # another outer rule size
    for b in (mk(other), mk(consts, precision=cudahm.FP32), mk(consts, keep_chi_moments=True)):
        b.set_data(data.fhat, data.r)
        with pytest.raises(cudahm.CudahmError) as ei:
            b.restore(blob)
        assert ei.value.code == cudahm.EINVAL
    c = mk(consts)
    c.set_data(data.fhat, data.r)
    c.restore(blob)
    assert np.array_equal(c.run(0, 15), a.run(0, 15))
