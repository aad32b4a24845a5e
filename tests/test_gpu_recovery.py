"""Truth recovery on the benchmark's synthetic populations (the sanity check the paper makes in
Sec. 5.3: the posterior covers the parameters the data were drawn from).

- LF, N = 3e5 (the benchmark workload): the FP64 member-form chain started at the truth, and
  the FP32 marginal chain started away from it, both cover (beta, ln L*, ln L_low) within
  4 posterior standard deviations plus 4 Monte Carlo standard errors.
- BB1 (the paper's model), N = 1e5: the FP64 member-form chain covers (beta, ln l, ln u) the
  same way.
"""
import math

import numpy as np
import pytest

from paper_2105_08026_gb300 import cudahm, synth

pytestmark = pytest.mark.gpu


def _covers(rows, truth):
    for j in range(rows.shape[1]):
        x = rows[:, j]
        sd = x.std()
        mcse = sd / math.sqrt(float(cudahm.cudahm_ess(x)[0]))
        assert abs(x.mean() - truth[j]) < 4 * sd + 4 * mcse, (j, x.mean(), truth[j], sd, mcse)


def test_lf_recovers_truth_member_and_marginal_forms():
    data = synth.lf_data(300_000, seed=1002)
    th0, sc, c = synth.lf_settings(data)
    truth = th0.copy()
    s = cudahm.Sampler(cudahm.LF, data.fhat.size, theta_init=th0, theta_prop_scale=sc, model_consts=c, seed=31)
    s.set_data(data.fhat, data.r)
    s.set_chi(synth.lf_chi_init(data, th0))
    _covers(s.run(1000, 4000), truth)
    start = th0 + np.array([0.08, 0.3, -0.4])
    m = cudahm.Sampler(cudahm.LF, data.fhat.size, theta_init=start, theta_prop_scale=sc, model_consts=c, seed=32,
                       precision=cudahm.FP32, marginal=True)
    m.set_data(data.fhat, data.r)
    _covers(m.run(3000, 12000), truth)


def test_bb1_recovers_truth():
    data = synth.bb1_data(100_000, seed=1004)
    th0, sc, c = synth.bb1_settings(data)
    s = cudahm.Sampler(cudahm.BB1, data.fhat.size, theta_init=th0, theta_prop_scale=sc, model_consts=c, seed=33)
    s.set_data(data.fhat, data.r)
    s.set_chi(synth.bb1_chi_init(data))
    _covers(s.run(2000, 8000), th0)
