"""Batched runs: many populations in one persistent launch.

Every population's chain is the same function of its own inputs whatever else shares the
launch (sums are exact, per-member values are the same expressions), so the bar is
bit-identity with the population run alone, in both precisions, for any launch shape."""
import numpy as np
import pytest

from paper_2105_08026_gb300 import cudahm, synth

pytestmark = pytest.mark.gpu


def _populations(precision, seed0=0):
    specs = [("nn1", 1), ("lf", 700), ("nn1", 2500), ("lf", 5000), ("nn1", 40000), ("lf", 256), ("nn1", 777)]
    out = []
    for q, (kind, n) in enumerate(specs):
        if kind == "nn1":
            d = synth.nn1_data(n, seed=100 + q + seed0)
            th, sc, c = synth.nn1_settings(d)
            out.append(dict(model=cudahm.NN1, n=n, y=d.y, aux=d.sigma, th=th, sc=sc, c=c, seed=31 + q))
        else:
            d = synth.lf_data(n, seed=200 + q + seed0)
            th, sc, c = synth.lf_settings(d, nL=96, nr=200)
            out.append(dict(model=cudahm.LF, n=n, y=d.fhat, aux=d.r, th=th, sc=sc, c=c, seed=41 + q))
    return out


def _make(spec, precision):
    s = cudahm.Sampler(spec["model"], spec["n"], theta_init=spec["th"], theta_prop_scale=spec["sc"],
                       model_consts=spec["c"], seed=spec["seed"], precision=precision)
    s.set_data(spec["y"], spec["aux"])
    return s


def _state(s):
    chi, S = s.chi()
    th, Sth = s.theta()
    return chi, S, th, Sth


@pytest.mark.parametrize("precision", [cudahm.FP64, cudahm.FP32])
def test_batch_equals_each_population_alone(precision):
    specs = _populations(precision)
    alone = []
    for sp in specs:
        s = _make(sp, precision)
        rows = s.run(30, 90, 3)
        alone.append((rows, _state(s)))
    batch = [_make(sp, precision) for sp in specs]
    rows_b, chosen = cudahm.batch_run(batch, 30, 90, 3)
    assert chosen.block_threads in (128, 256)
    for (ra, sa), rb, s in zip(alone, rows_b, batch):
        assert np.array_equal(ra, rb)
        for x, y in zip(sa, _state(s)):
            assert np.array_equal(x, y)


def test_batch_result_does_not_depend_on_launch_shape():
    specs = _populations(cudahm.FP32, seed0=7)
    runs = []
    for block, chunk, grid in ((128, 17, 0), (256, 1000, 0), (128, 33, 200)):
        ss = [_make(sp, cudahm.FP32) for sp in specs]
        tune = cudahm.CudahmTune(block, chunk, 0, grid)
        rows, chosen = cudahm.batch_run(ss, 0, 60, 1, tune)
        assert chosen.block_threads == block and chosen.sweeps_per_launch == chunk
        assert chosen.grid_blocks == grid if grid else chosen.grid_blocks >= len(specs)
        runs.append((rows, [_state(s) for s in ss]))
    for r in runs[1:]:
        for a, b in zip(runs[0][0], r[0]):
            assert np.array_equal(a, b)
        for sa, sb in zip(runs[0][1], r[1]):
            for x, y in zip(sa, sb):
                assert np.array_equal(x, y)


def test_batch_rejects_mixed_precision():
    specs = _populations(cudahm.FP64)[:2]
    a = _make(specs[0], cudahm.FP64)
    b = _make(specs[1], cudahm.FP32)
    with pytest.raises(cudahm.CudahmError) as ei:
        cudahm.batch_run([a, b], 0, 5)
    assert ei.value.code == cudahm.EINVAL


def test_large_population_streams_with_the_same_chain():
    """A population too large for register residency (7e5 members, FP32) runs through the streaming
    kernel; it gives the chain the batched path gives it, and kept rows match a split run."""
    d = synth.nn1_data(700_000, seed=5)
    th, sc, c = synth.nn1_settings(d)
    mk = lambda: cudahm.Sampler(cudahm.NN1, d.y.size, theta_init=th, theta_prop_scale=sc, model_consts=c, seed=3,
                                precision=cudahm.FP32)
    a, b = mk(), mk()
    a.set_data(d.y, d.sigma)
    b.set_data(d.y, d.sigma)
    assert a.stats().objects_per_thread == 0
    ra = a.run(10, 40)
    rb = np.concatenate([b.run(10, 15), b.run(0, 25)])
    assert np.array_equal(ra, rb)
    assert np.array_equal(a.chi()[0], b.chi()[0])
