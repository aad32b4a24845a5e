"""The library's effective-sample-size estimator (host code, no GPU): the measure of the
paper's normal-normal benchmark (time to an ESS of about 1000 after burn-in, Sec. 3).

- On AR(1) series x_t = rho x_{t-1} + e_t the integrated autocorrelation time is
  (1 + rho)/(1 - rho) in closed form, so ESS/n tends to (1 - rho)/(1 + rho); at n = 2e5 the
  estimator's spread is a few per cent (checked over seeds), the bound 12 %.
- It equals the oracle's independent estimator (FFT autocovariances, same initial monotone
  sequence rule) to rounding on every column of a strided matrix.
- Edge cases: fewer than 4 rows, a constant column, non-finite samples, bad arguments.
"""
import math

import numpy as np
import pytest
from scipy.signal import lfilter

from oracle import stats
from paper_2105_08026_gb300 import build as cbuild
from paper_2105_08026_gb300 import cudahm


@pytest.fixture(scope="module", autouse=True)
def lib():
    if not cbuild.up_to_date():
        try:
            cbuild.build()
        except RuntimeError as e:  # no nvcc on this machine
            pytest.skip(str(e))
    return cudahm.lib()


def _ar1(rho, n, seed):
    return lfilter([1.0], [1.0, -rho], np.random.default_rng(seed).standard_normal(n))


@pytest.mark.parametrize("rho", [0.0, 0.5, 0.9, 0.98])
def test_ess_ar1_closed_form(rho):
    n = 200_000
    x = _ar1(rho, n, 7 + int(100 * rho))
    want = n * (1.0 - rho) / (1.0 + rho)
    got = cudahm.cudahm_ess(x)[0]
    assert abs(got / want - 1.0) < 0.12, (got, want)
    assert abs(stats.ess_geyer(x) / want - 1.0) < 0.12


def test_ess_matches_oracle_estimator_per_column():
    cols = [_ar1(r, 30_000, 40 + q) for q, r in enumerate((0.2, 0.7, 0.95))]
    cols.append(np.random.default_rng(3).standard_normal(30_000))
    X = np.stack(cols, axis=1)
    got = cudahm.cudahm_ess(X)
    for j in range(X.shape[1]):
        ref = stats.ess_geyer(X[:, j])
        assert abs(got[j] - ref) <= 1e-9 * ref, (j, got[j], ref)


def test_ess_edge_cases():
    assert cudahm.cudahm_ess(np.array([1.0, 2.0, 3.0])).tolist() == [3.0]
    assert cudahm.cudahm_ess(np.full(50, 2.5)).tolist() == [50.0]
    with pytest.raises(cudahm.CudahmError) as ei:
        cudahm.cudahm_ess(np.array([1.0, math.nan, 2.0, 3.0, 4.0]))
    assert ei.value.code == cudahm.ENUMERIC
    with pytest.raises(cudahm.CudahmError) as ei:
        cudahm.cudahm_ess(np.zeros((0, 2)))
    assert ei.value.code == cudahm.EINVAL
