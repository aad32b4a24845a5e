"""All-cores timing driver of the oracle's luminosity-function chain (CPU baseline only).

TEST INFRASTRUCTURE, like the rest of this package: only the test suite and the CPU-baseline
legs of ``bench.py`` use it. It runs the oracle's own arithmetic on every host core: the member
half of each sweep (eq. psi_sampling, Sec. 2.1; the RAM step of Sec. 2.2) split into contiguous
member ranges, one per thread, each range stepped by the oracle's ``orc_member_pass`` (ctypes
releases the interpreter lock during the call); the theta step (eq. theta_sampling with the
thinned likelihood of Sec. 4.2 and the delayed theta RAM update of reading R3) serially in the
calling thread, in the oracle's order. Member draws are keyed by member and sweep, so the split
changes no member's step; the sum over members is math.fsum (correctly rounded) where the
oracle's chain sums with Neumaier's method, so theta agrees with the oracle's chain to rounding
(tests/test_oracle_allcores.py).
"""
from __future__ import annotations

import math
import time
from concurrent.futures import ThreadPoolExecutor

import numpy as np

from . import LF, _f64, _p, draw, lib, member_pass, ram_update


def _lf_logprior(th) -> float:
    """Truncated Cauchy in beta on (-2, 0), log-flat L*, flat L_low (Jacobian L_low), L_low < L*."""
    if not (-2.0 < th[0] < 0.0) or not (th[2] < th[1]):
        return -math.inf
    return -math.log(1.0 + th[0] * th[0]) + th[2]


def _propose(theta, S_theta, U):
    """theta + S_theta U with the lower factor, summed in the oracle's order."""
    p = theta.size
    out = np.empty(p)
    for a in range(p):
        t = theta[a]
        for b in range(a + 1):
            t += S_theta[a, b] * U[b]
        out[a] = t
    return out


def lf_run(fhat, r, consts, theta0, scale, seed, chi0, sweeps, threads, adapt_theta=True):
    """`sweeps` sweeps of the LF chain from (chi0, S = 1, theta0, S_theta = diag(scale)) on
    `threads` threads. Returns (theta rows, chi, S, seconds of the sweep loop)."""
    fhat, r, consts = _f64(fhat), _f64(r), _f64(consts)
    n = fhat.size
    chi = _f64(chi0).copy()
    S = np.ones(n)
    theta = _f64(theta0).copy()
    S_th = np.diag(_f64(scale))
    params = np.array([0.4, 2.0 / 3.0, 0.4, 1.0 if adapt_theta else 0.0])
    L = lib()
    rule = L.orc_lf_rule_new(_p(consts))
    eb = lambda th: L.orc_lf_rule_etabar(rule, _p(_f64(th)), _p(consts))
    bounds = [(n * t // threads, n * (t + 1) // threads) for t in range(threads)]
    rows = np.empty((sweeps, 3))
    pend = None
    try:
        eb_cur = eb(theta)
        lp_cur = _lf_logprior(theta)
        t0 = time.perf_counter()
        with ThreadPoolExecutor(max_workers=threads) as ex:
            for s in range(sweeps):
                k = s + 1
                eta = (k + 1.0) ** (-2.0 / 3.0)
                U, ut = draw(seed, 1, 0, k, 3)
                thp = _propose(theta, S_th, U)
                futs = [ex.submit(member_pass, LF, fhat, r, consts, params, seed, k, i0, i1, theta, thp, chi, S)
                        for (i0, i1) in bounds if i1 > i0]
                d = np.concatenate([f.result()[0] for f in futs])
                lp_new = _lf_logprior(thp)
                eb_new = 0.0
                if lp_new == -math.inf or np.isneginf(d).any():
                    logalpha = -math.inf
                else:
                    eb_new = eb(thp)
                    logalpha = math.fsum(d.tolist()) + lp_new - lp_cur - n * (math.log(eb_new) - math.log(eb_cur))
                alpha = 1.0 if logalpha >= 0.0 else math.exp(logalpha)
                if math.log(ut) < logalpha:
                    theta, eb_cur, lp_cur = thp, eb_new, lp_new
                if adapt_theta:
                    if pend is not None:
                        S_th = ram_update(S_th, pend[0], pend[1], 0.4, pend[2])
                    pend = (U, alpha, eta)
                rows[s] = theta
        dt = time.perf_counter() - t0
    finally:
        L.orc_lf_rule_free(rule)
    return rows, chi, S, dt
