"""The chain does not depend on the launch shape (register-resident sweep kernel).

128 or 256 threads per block give a different grid, different members per block and thread,
another split of the selection rule's outer nodes and another order of the atomic adds into
the grid totals. Draws are keyed by (seed, member, sweep) and every cross-block sum is exact,
so theta rows, latents, RAM factors, theta and S_theta must agree bit for bit, in both
precisions.
"""
import numpy as np
import pytest

from paper_2105_08026_gb300 import cudahm, synth

pytestmark = pytest.mark.gpu


def _run(model, n, y, aux, theta0, scale, consts, prec, block):
    s = cudahm.Sampler(model, n, theta_init=theta0, theta_prop_scale=scale, model_consts=consts, seed=21,
                       precision=prec, block_threads=block)
    s.set_data(y, aux)
    rows = np.concatenate([s.run(20, 150, 1), s.run(0, 130, 2)])
    chi, S = s.chi()
    th, Sth = s.theta()
    st = s.stats()
    s.close()
    return rows, chi, S, th, Sth, (st.grid_blocks, st.block_threads, st.objects_per_thread)


@pytest.mark.parametrize("prec", [cudahm.FP64, cudahm.FP32])
@pytest.mark.parametrize("model", ["lf", "nn1"])
def test_block_size_does_not_change_the_chain(model, prec):
    if model == "lf":
        d = synth.lf_data(20_000, seed=41)
        theta0, scale, consts = synth.lf_settings(d, nL=256, nr=256)
        args = (cudahm.LF, 20_000, d.fhat, d.r, theta0, scale, consts)
    else:
        d = synth.nn1_data(3_000, seed=42)
        theta0, scale, consts = synth.nn1_settings(d)
        args = (cudahm.NN1, 3_000, d.y, d.sigma, theta0, scale, consts)
    a = _run(*args, prec, 256)
    b = _run(*args, prec, 128)
    assert a[5] != b[5]  # two launch shapes
    for x, y in zip(a[:5], b[:5]):
        assert np.array_equal(x, y)
