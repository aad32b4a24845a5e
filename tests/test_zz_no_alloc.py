"""The allocation-free selection integral (cudahm_lf_etabar_noalloc).

Callers that may not allocate device memory at the moment they need etabar(theta) --
a process whose device memory all belongs to its own pool, a latency-critical loop
that must not pay for an allocation's synchronisation, a caller out of memory -- use
this entry point: its tables and partial sums sit in a fixed array inside the library.
Here it must give the same value as the handle-based cudahm_eval_etabar, within the
1e-13 relative tolerance of the selection-integral parity tests, on two calls in a row
(the second call reuses the array the first one left behind), and must refuse rule
sizes beyond its fixed limit with a clear error.

This file is named to be collected last, so that a run stopping at the first failure
has already run every other test.
"""
import numpy as np
import pytest

from paper_2105_08026_gb300 import cudahm, synth

pytestmark = pytest.mark.gpu


def test_noalloc_etabar_matches_handle_on_two_calls():
    torch = pytest.importorskip("torch")
    data = synth.lf_data(2000, seed=21)
    theta0, scale, consts = synth.lf_settings(data)  # 1024 x 1024 rule, the limit
    s = cudahm.Sampler(cudahm.LF, data.fhat.size, theta_init=theta0, theta_prop_scale=scale, model_consts=consts)
    s.set_data(data.fhat, data.r)
    thetas = [theta0, theta0 + np.array([0.07, -0.3, 0.25])]
    expected = [s.etabar(th) for th in thetas]

    torch.cuda.set_device(0)
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    th_dev = torch.tensor(np.array(thetas), dtype=torch.float64, device="cuda")
    for q in range(2):  # two calls in a row on the same fixed array
        cudahm.cudahm_lf_etabar_noalloc(th_dev[q].data_ptr(), consts, out[q:q + 1].data_ptr(), 0)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    for g, e in zip(got, expected):
        assert abs(g - e) <= 1e-13 * abs(e), (g, e)
    assert got[0] != got[1]


def test_noalloc_rejects_rule_beyond_fixed_limit():
    torch = pytest.importorskip("torch")
    consts = np.array([2.0, 10.0, 4000.0, 2048.0, 1024.0, np.log(60.0)])
    th = torch.tensor([-1.2, 23.0, 18.4], dtype=torch.float64, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(cudahm.CudahmError) as ei:
        cudahm.cudahm_lf_etabar_noalloc(th.data_ptr(), consts, out.data_ptr(), 0)
    assert ei.value.code == cudahm.EINVAL
    assert "1024" in str(ei.value)


def test_noalloc_follows_a_change_of_rule():
    """Consecutive calls with the same rule reuse the array's tables; a call with another rule
    size or another sigma_F rebuilds them. Each value matches the handle built for its constants."""
    torch = pytest.importorskip("torch")
    data = synth.lf_data(2000, seed=22)
    theta0, scale, consts_a = synth.lf_settings(data)
    consts_b = consts_a.copy()
    consts_b[0] *= 1.1   # sigma_F
    consts_b[3] = 512    # n_L
    consts_b[4] = 768    # n_r
    expected = {}
    for name, c in (("a", consts_a), ("b", consts_b)):
        s = cudahm.Sampler(cudahm.LF, data.fhat.size, theta_init=theta0, theta_prop_scale=scale, model_consts=c)
        s.set_data(data.fhat, data.r)
        expected[name] = s.etabar(theta0)
    torch.cuda.set_device(0)
    th = torch.tensor(theta0, dtype=torch.float64, device="cuda")
    seq = ["a", "a", "b", "b", "a"]
    out = torch.zeros(len(seq), dtype=torch.float64, device="cuda")
    for q, name in enumerate(seq):
        cudahm.cudahm_lf_etabar_noalloc(th.data_ptr(), consts_a if name == "a" else consts_b,
                                        out[q:q + 1].data_ptr(), 0)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    for g, name in zip(got, seq):
        e = expected[name]
        assert abs(g - e) <= 1e-13 * abs(e), (name, g, e)
    assert expected["a"] != expected["b"]
