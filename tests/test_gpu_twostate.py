"""GPU two-state test model of the member accept rule (the device's own accept routine).

FP64: the device chains use the member step's accept uniform (Philox block (1, 0, chain, sweep))
and accept routine (u < e^Delta with the table exp, compared as bit patterns); the oracle's use
the same uniform and ln u < Delta with the C library log. A decision can differ only where
|Delta - ln u| is at rounding level (probability ~1e-16 a step), so the transition counts must
be identical. Both the FP64 and the FP32 bulk form's rule must satisfy detailed balance, the
exact uphill accepts and the stationary occupation (5 sigma) on 1e8 steps.
"""
import numpy as np
import pytest

import oracle
from paper_2105_08026_gb300 import cudahm

from test_oracle_twostate import check_detailed_balance

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("pi1", [0.7, 0.2, 0.5, 0.999])
def test_fp64_counts_equal_the_oracle(pi1):
    g = cudahm.cudahm_twostate_run(pi1, cudahm.FP64, 4001, 500, seed=11)
    o = oracle.twostate_counts(pi1, 4001, 500, seed=11)
    assert np.array_equal(g, o), (g, o)


@pytest.mark.parametrize("precision", [cudahm.FP64, cudahm.FP32])
@pytest.mark.parametrize("pi1", [0.7, 0.2, 0.999])
def test_detailed_balance_on_1e8_steps(precision, pi1):
    c = cudahm.cudahm_twostate_run(pi1, precision, 1_000_000, 100, seed=12)
    assert c.sum() == 100_000_000
    check_detailed_balance(c, pi1, 100)


def test_invalid_arguments():
    for args in ((0.0, cudahm.FP64, 10, 10), (1.0, cudahm.FP64, 10, 10), (0.5, 7, 10, 10), (0.5, cudahm.FP64, 0, 10),
                 (0.5, cudahm.FP64, 10, 0)):
        with pytest.raises(cudahm.CudahmError) as ei:
            cudahm.cudahm_twostate_run(*args)
        assert ei.value.code == cudahm.EINVAL
