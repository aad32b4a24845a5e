"""One population split into shards (one handle per contiguous member range) on one GPU, every
sweep's exchange words added between the shards' passes and decisions (an all-reduce emulated on
the device by a sum over the shards' word buffers, on the same stream), equals one handle
holding the whole population: theta rows, latents and RAM factors bit for bit. The decoded
words (tests/shard_words.py, the CPU codec the gloo test uses) equal the unsplit chain's traced
theta' sums, which ties the device's exchange format to the CPU ranks' one."""
import numpy as np
import pytest

from paper_2105_08026_gb300 import cudahm, synth

import shard_words

pytestmark = pytest.mark.gpu


def _problem(model, n, seed, nL=128, nr=128):
    if model == cudahm.NN1:
        d = synth.nn1_data(n, seed=seed)
        th, sc, c = synth.nn1_settings(d)
        return d.y, d.sigma, th, sc, c
    if model == cudahm.LF:
        d = synth.lf_data(n, seed=seed)
        th, sc, c = synth.lf_settings(d, nL=nL, nr=nr)
        return d.fhat, d.r, th, sc, c
    if model == cudahm.BB1:
        d = synth.bb1_data(n, seed=seed)
        th, sc, c = synth.bb1_settings(d, nL=nL, nr=nr)
        return d.fhat, d.r, th, sc, c
    if model == cudahm.MVN3:
        d = synth.mvn3_data(n, seed=seed)
        th, sc, c = synth.mvn3_settings(d)
        return d.y, d.s, th, sc, c
    d = synth.nn3_data(n, seed=seed)
    th, sc, c = synth.nn3_settings(d)
    return d.y, d.s, th, sc, c


def _chi0(model, n, seed):
    """BB1 starts from the chi the BB1 tests use; the other models from the library's default."""
    return synth.bb1_chi_init(synth.bb1_data(n, seed=seed)) if model == cudahm.BB1 else None


def _split_run(model, y, aux, th, sc, c, prec, seed, cuts, burn, iters, thin, keep_words=False, drop=None,
               chi0=None):
    """The population split at `cuts`; returns (rows, chi, S, per-sweep summed words)."""
    import torch
    st = torch.cuda.Stream()
    n = y.shape[0]
    parts = len(cuts) - 1
    shards = []
    for r in range(parts):
        a, b = cuts[r], cuts[r + 1]
        s = cudahm.Sampler(model, b - a, theta_init=th, theta_prop_scale=sc, model_consts=c, seed=seed,
                           precision=prec, stream=st.cuda_stream)
        s.set_data(y[a:b], aux[a:b])
        if chi0 is not None:
            s.set_chi(chi0[a:b])
        s.shard(a, n, r, parts)
        shards.append(s)
    words = [torch.zeros(cudahm.SHARD_WORDS, dtype=torch.int64, device="cuda") for _ in shards]
    total = torch.zeros(cudahm.SHARD_WORDS, dtype=torch.int64, device="cuda")
    seen = []
    with torch.cuda.stream(st):
        for s in shards:
            cudahm.cudahm_shard_begin(s.h, burn, iters, thin)
        for k in range(burn + iters):
            for s, w in zip(shards, words):
                cudahm.cudahm_shard_pass(s.h, w.data_ptr())
            use = [w for r, w in enumerate(words) if r != drop]
            torch.sum(torch.stack(use), dim=0, out=total)
            if keep_words:
                seen.append(total.cpu().numpy().copy())
            for s in shards:
                cudahm.cudahm_shard_decide(s.h, total.data_ptr())
    nrows = [cudahm.cudahm_shard_end(s.h) for s in shards]
    assert len(set(nrows)) == 1
    rows = [cudahm.cudahm_get_samples(s.h, s.p, nrows[0]) for s in shards]
    for r in rows[1:]:
        assert np.array_equal(r, rows[0])  # every shard took the same decisions
    chis, Ss = zip(*[s.chi() for s in shards])
    for s in shards:
        s.close()
    return rows[0], np.concatenate(chis), np.concatenate(Ss), seen


def _whole(model, y, aux, th, sc, c, prec, seed, burn, iters, thin, trace=0, chi0=None):
    s = cudahm.Sampler(model, y.shape[0], theta_init=th, theta_prop_scale=sc, model_consts=c, seed=seed,
                       precision=prec, trace_sweeps=trace)
    s.set_data(y, aux)
    if chi0 is not None:
        s.set_chi(chi0)
    rows = s.run(burn, iters, thin)
    chi, S = s.chi()
    tr = s.trace(trace) if trace else None
    s.close()
    return rows, chi, S, tr


CASES = [
    # model, precision, N, cuts (ragged; offsets not multiples of 4), sweeps
    (cudahm.NN1, cudahm.FP64, 3001, [0, 1000, 1001, 3001], 300),
    (cudahm.NN1, cudahm.FP32, 4099, [0, 1237, 4099], 300),
    (cudahm.LF, cudahm.FP64, 2000, [0, 501, 1003, 1502, 2000], 200),
    (cudahm.LF, cudahm.FP32, 5000, [0, 1237, 3001, 5000], 300),
    (cudahm.BB1, cudahm.FP64, 1500, [0, 750, 1500], 150),
    (cudahm.MVN3, cudahm.FP64, 1200, [0, 401, 1200], 150),
    (cudahm.NN3, cudahm.FP32, 1200, [0, 599, 1200], 150),
]


@pytest.mark.parametrize("model,prec,n,cuts,sweeps", CASES)
def test_split_population_equals_whole_bit_for_bit(model, prec, n, cuts, sweeps):
    y, aux, th, sc, c = _problem(model, n, seed=2100 + n)
    chi0 = _chi0(model, n, 2100 + n)
    burn, thin = sweeps // 3, 2
    iters = sweeps - burn
    rows, chi, S, _ = _split_run(model, y, aux, th, sc, c, prec, 41, cuts, burn, iters, thin, chi0=chi0)
    wrows, wchi, wS, _ = _whole(model, y, aux, th, sc, c, prec, 41, burn, iters, thin, chi0=chi0)
    assert rows.shape == (iters // thin, cudahm.MODEL_P[model])
    assert np.array_equal(rows, wrows)
    assert np.array_equal(chi, wchi)
    assert np.array_equal(S, wS)


def test_rule_split_over_more_shards_than_outer_nodes():
    """LF with n_L = 2 outer nodes over 3 shards: one shard adds no rule term."""
    y, aux, th, sc, c = _problem(cudahm.LF, 600, seed=2201, nL=2, nr=64)
    rows, chi, S, _ = _split_run(cudahm.LF, y, aux, th, sc, c, cudahm.FP64, 5, [0, 200, 400, 600], 20, 80, 1)
    wrows, wchi, wS, _ = _whole(cudahm.LF, y, aux, th, sc, c, cudahm.FP64, 5, 20, 80, 1)
    assert np.array_equal(rows, wrows) and np.array_equal(chi, wchi) and np.array_equal(S, wS)


def test_one_shard_at_full_size_equals_the_resident_kernel():
    """The shard path (streaming kernel + decision kernel) with one shard at N = 3e5, LF, the
    1024 x 1024 rule, FP32 and FP64: the register-resident kernel's chain."""
    for prec in (cudahm.FP64, cudahm.FP32):
        y, aux, th, sc, c = _problem(cudahm.LF, 300_000, seed=2202, nL=1024, nr=1024)
        rows, chi, S, _ = _split_run(cudahm.LF, y, aux, th, sc, c, prec, 9, [0, 300_000], 0, 30, 1)
        wrows, wchi, wS, _ = _whole(cudahm.LF, y, aux, th, sc, c, prec, 9, 0, 30, 1)
        assert np.array_equal(rows, wrows) and np.array_equal(chi, wchi) and np.array_equal(S, wS)


def test_decoded_words_equal_the_traced_theta_sums():
    """The CPU codec decodes the summed device words to the unsplit chain's traced D (the exact
    theta' sum as binary64), sweep by sweep; member counts and shard counts add up."""
    y, aux, th, sc, c = _problem(cudahm.NN1, 2500, seed=2203)
    T = 60
    _, _, _, seen = _split_run(cudahm.NN1, y, aux, th, sc, c, cudahm.FP64, 13, [0, 999, 2500], 0, T, 1,
                               keep_words=True)
    _, _, _, tr = _whole(cudahm.NN1, y, aux, th, sc, c, cudahm.FP64, 13, 0, T, 1, trace=T)
    D_trace = tr["D"]
    for k, w in enumerate(seen):
        D, E, f, members, shards = shard_words.decode(w)
        assert members == 2500 and shards == 2 and f[1] == 0
        if f[0] == 0 and f[2] == 0 and np.isfinite(D_trace[k]):
            assert D == D_trace[k], (k, D, D_trace[k])


def test_words_missing_a_shard_stop_the_run():
    y, aux, th, sc, c = _problem(cudahm.NN1, 900, seed=2204)
    with pytest.raises(cudahm.CudahmError) as ei:
        _split_run(cudahm.NN1, y, aux, th, sc, c, cudahm.FP64, 3, [0, 300, 900], 0, 10, 1, drop=1)
    assert ei.value.code == cudahm.ESTATE


def test_shard_calls_out_of_order_are_rejected():
    y, aux, th, sc, c = _problem(cudahm.NN1, 100, seed=2205)
    s = cudahm.Sampler(cudahm.NN1, 100, theta_init=th, theta_prop_scale=sc, model_consts=c, seed=1)
    s.set_data(y, aux)
    with pytest.raises(cudahm.CudahmError):
        cudahm.cudahm_shard_begin(s.h, 0, 5, 1)  # before shard_config
    with pytest.raises(cudahm.CudahmError):
        s.shard(50, 120, 0, 2)  # members beyond the population
    s.shard(0, 100, 0, 1)
    cudahm.cudahm_shard_begin(s.h, 0, 5, 1)
    with pytest.raises(cudahm.CudahmError):
        s.run(0, 5)  # a plain run during a sharded run
    import torch
    w = torch.zeros(cudahm.SHARD_WORDS, dtype=torch.int64, device="cuda")
    with pytest.raises(cudahm.CudahmError):
        cudahm.cudahm_shard_decide(s.h, w.data_ptr())  # decide before a pass
    cudahm.cudahm_shard_pass(s.h, w.data_ptr())
    with pytest.raises(cudahm.CudahmError):
        cudahm.cudahm_shard_pass(s.h, w.data_ptr())  # a second pass before the decision
    cudahm.cudahm_shard_decide(s.h, w.data_ptr())
    assert cudahm.cudahm_shard_end(s.h) == 1  # one sweep of five made and kept (no burn-in, thin 1)
    s.close()
