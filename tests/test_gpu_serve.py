"""Serving with continuous batching: requests admitted while others run share launches, and
each result must equal running the request alone (bit for bit: batched chains do not depend
on what else is in the launch)."""
import time

import numpy as np
import pytest

from paper_2105_08026_gb300 import cudahm, synth

pytestmark = pytest.mark.gpu


def _requests():
    out = []
    for q, (kind, n, sweeps) in enumerate([("nn1", 3000, 400), ("lf", 1500, 300), ("nn1", 50, 700),
                                           ("lf", 9000, 250), ("nn1", 120000, 200), ("lf", 600, 500)]):
        if kind == "nn1":
            d = synth.nn1_data(n, seed=300 + q)
            th, sc, c = synth.nn1_settings(d)
            model, y, aux = cudahm.NN1, d.y, d.sigma
        else:
            d = synth.lf_data(n, seed=400 + q)
            th, sc, c = synth.lf_settings(d, nL=128, nr=256)
            model, y, aux = cudahm.LF, d.fhat, d.r
        cfg = cudahm.make_config(model, n, theta_init=th, theta_prop_scale=sc, model_consts=c, seed=70 + q,
                                 precision=cudahm.FP32)
        out.append(dict(cfg=cfg, y=y, aux=aux, burn=sweeps // 4, iters=sweeps, thin=2,
                        alone=dict(model=model, n=n, th=th, sc=sc, c=c, seed=70 + q)))
    return out


def _alone(r):
    a = r["alone"]
    s = cudahm.Sampler(a["model"], a["n"], theta_init=a["th"], theta_prop_scale=a["sc"], model_consts=a["c"],
                       seed=a["seed"], precision=cudahm.FP32)
    s.set_data(r["y"], r["aux"])
    return s.run(r["burn"], r["iters"], r["thin"])


def test_served_results_equal_running_alone():
    """Staggered arrivals: later requests are admitted while earlier ones are on the GPU (the
    server reports several requests on the device at once), and every result is still the chain
    the request gives alone."""
    reqs = _requests()
    reqs[0]["iters"] = 4000  # a long first request that the later ones join
    sv = cudahm.Server(8 << 30, precision=cudahm.FP32, max_active=64, sweeps_per_step=37)
    tickets = []
    peak = 0
    for r in reqs:
        tickets.append(sv.submit(r["cfg"], r["y"], r["aux"], r["burn"], r["iters"], r["thin"]))
        t_end = time.perf_counter() + 0.01
        while time.perf_counter() < t_end:
            peak = max(peak, sv.stats()["active"])
            time.sleep(0.0005)
    while not all(sv.poll(t) for t in tickets):
        peak = max(peak, sv.stats()["active"])
        time.sleep(0.0005)
    assert peak >= 2, f"requests never shared the device (peak active {peak})"
    for r, t in zip(reqs, tickets):
        rows, lat = sv.result(t)
        assert lat > 0
        assert np.array_equal(rows, _alone(r))
    st = sv.stats()
    assert st["completed"] == len(reqs) and st["queued"] == 0 and st["active"] == 0
    sv.close()


def test_budget_admits_one_at_a_time_and_rejects_oversize():
    reqs = _requests()[:3]
    sv = cudahm.Server(200 << 20, precision=cudahm.FP32, max_active=1, sweeps_per_step=50)
    tickets = [sv.submit(r["cfg"], r["y"], r["aux"], r["burn"], r["iters"], r["thin"]) for r in reqs]
    peak = 0
    while not all(sv.poll(t) for t in tickets):
        peak = max(peak, sv.stats()["active"])
        time.sleep(0.002)
    assert peak <= 1
    for r, t in zip(reqs, tickets):
        rows, _ = sv.result(t)
        assert np.array_equal(rows, _alone(r))
    n_big = 6_000_000  # about 0.4 GB of device state: more than the whole 200 MiB budget
    cfg = cudahm.make_config(cudahm.NN1, n_big, theta_init=[0.0, 0.0], theta_prop_scale=[0.05, 0.05],
                             model_consts=[-10.0, 10.0], precision=cudahm.FP32)
    with pytest.raises(cudahm.CudahmError) as ei:
        sv.submit(cfg, np.zeros(n_big), np.ones(n_big), 0, 10)
    assert ei.value.code == cudahm.ENOMEM
    sv.close()
