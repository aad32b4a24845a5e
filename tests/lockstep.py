"""Lockstep comparison of a sampler chain with the CPU oracle's chain (test helper).

Used by the GPU parity tests (device chain through the C ABI against the oracle) and by a CPU
test of the comparison rules themselves (oracle against oracle, with disagreements planted in
one trace).
"""
import math

import numpy as np

import oracle
from paper_2105_08026_gb300 import cudahm

REL = 1e-12       # latents, RAM factors, theta rows, per-member log densities
# Member Delta = lp(Y) - lp(X), relative to max(1, |Delta|). From identical states the two sides
# agree to ~2e-13 (a few ulp of log targets of size ~1e2). Over a long run the chains' latents
# drift apart by a few ulp (each side rounds its own exp/log), and a bright member's likelihood
# curvature (Fhat/sigma_F)^2 ~ 1e5 turns that into Delta differences that grow about linearly
# with the sweep index k: ~2e-11 after 1000 sweeps (luminosity workload, N = 1e4) and 1.35e-10
# after 4200 (N = 2000), every decision identical (measured). The bound at sweep k,
# DELTA_REL + DELTA_DRIFT k, stays below the 1e-9 near-tie band up to k = 2e4.
DELTA_REL = 1e-11
DELTA_DRIFT = 5e-14
NEAR_TIE = 1e-9


def _close(a, b, rel=REL):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    both_inf = np.isinf(a) & np.isinf(b) & (np.sign(a) == np.sign(b))
    err = np.abs(a - b)
    tol = rel * np.maximum(1.0, np.maximum(np.abs(a), np.abs(b)))
    return np.all(both_inf | (err <= tol)), float(np.max(np.where(both_inf, 0.0, err / tol), initial=0.0))


def _lockstep(model, y, aux, consts, theta0, scale, seed, chi0, sweeps, adapt_theta=True, block_threads=0):
    n = np.asarray(y).shape[0]
    s = cudahm.Sampler(model, n, theta_init=theta0, theta_prop_scale=scale, model_consts=consts, seed=seed,
                       trace_sweeps=sweeps, adapt_theta=adapt_theta, block_threads=block_threads)
    s.set_data(y, aux)
    s.set_chi(chi0)
    rows = s.run(0, sweeps)
    tr = s.trace(sweeps)
    ch = oracle.Chain(model, y, aux, consts, theta0, scale, seed, chi0, adapt_theta=adapt_theta)
    orows, otr = ch.run(0, sweeps, trace_sweeps=sweeps)
    return s, ch, rows, orows, tr, otr


def _rows_close(a, b, rel=REL):
    """Per row: every element within rel (both infinite with one sign also counts)."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    both_inf = np.isinf(a) & np.isinf(b) & (np.sign(a) == np.sign(b))
    tol = rel * np.maximum(1.0, np.maximum(np.abs(a), np.abs(b)))
    return np.all(both_inf | (np.abs(a - b) <= tol), axis=-1)


def d_tolerance(n, d_atol=None):
    """Absolute bound on the traced log alpha_theta (and the base of the bound on D).

    Each of the N terms log f(chi_i;theta') - log f(chi_i;theta) carries a few ulp of formula
    rounding (table exp/log on the device, libm in the oracle); the device sum is exact and the
    oracle's compensated sum is within one ulp of exact. Rounding errors without a common sign
    grow like sqrt(N): 1e-10 sqrt(N/1e4) keeps the bound below the 1e-9 near-tie band up to
    N = 1e6. Models with a steeper member likelihood pass their own base."""
    return (1e-10 if d_atol is None else d_atol) * max(1.0, math.sqrt(n / 1e4))


# D alone also carries the part of the two sides' exp rounding that has a common sign: every
# term's exp(chi - ln L*) moves by the same relative few 1e-16, so D moves in proportion to the
# proposal's step, like |D| itself (measured on the luminosity workload at N = 1e4: 2e-10 at
# |D| = 284, 3e-11 median at |D| ~ 1e2). That part cancels in log alpha_theta (the selection
# integral term -N ln etabar carries the same bias; measured log alpha error <= 1.3e-11), which
# is what decides, so log alpha keeps the tighter bound above.
D_REL = 2e-12


def _check_lockstep(s, ch, rows, orows, tr, otr, d_atol=None):
    """Compare the device chain with the oracle's over every traced sweep.

    Near ties (|Delta - ln u| < 1e-9, which rounding may decide either way):
    - a member whose decision differs in that band is masked from the next sweep on (its chain
      legitimately diverges), and every other member is still compared;
    - D and log alpha_theta sum over every member, so they are compared up to the sweep of the
      first member divergence;
    - the theta chain is compared while its decisions and accepted proposals agree; a theta
      decision that differs before any member diverged must be a near tie, and it ends the
      comparison there (members are compared through that sweep, whose theta was still common).
    Returns a summary: the sweeps each part was compared over, the near ties, the largest D error.
    """
    T, n = tr["acc"].shape
    assert np.array_equal(tr["u"], otr["u"]), "accept uniforms differ (RNG layout)"
    assert np.array_equal(tr["utheta"], otr["utheta"]), "theta accept uniforms differ (RNG layout)"
    # first member near-tie divergence (provisional; refined below with the theta path)
    diff = tr["acc"] != otr["acc"]
    k_m = int(np.argwhere(diff)[0][0]) if diff.any() else T
    # the theta path: step k is common while the decisions agree and an accepted proposal agrees
    tsame = tr["tacc"] == otr["tacc"]
    pclose = _rows_close(tr["theta_prop"], otr["theta_prop"])
    step_ok = tsame & (pclose | (tr["tacc"] == 0))
    bad = np.nonzero(~step_ok)[0]
    k_t = int(bad[0]) if bad.size else T
    theta_tie = None
    if k_t < min(T, k_m):
        # before any member diverged the theta steps must agree (from the sweep of a member
        # divergence on, D carries that member's other latent)
        assert pclose[k_t], f"theta proposals differ at sweep {k_t} before any divergence"
        gap = abs(otr["logalpha"][k_t] - math.log(otr["utheta"][k_t]))
        assert gap < NEAR_TIE, f"theta decision differs at sweep {k_t}: |log alpha - ln u| = {gap}"
        theta_tie = k_t
    # members: sweep k uses theta after sweep k - 1, common for k <= k_t
    k_mem = min(T, k_t + 1)
    masked_from = np.full(n, T, dtype=np.int64)
    ties = []
    for k, i in np.argwhere(diff[:k_mem]):  # row-major: ordered by sweep
        if k >= masked_from[i]:
            continue
        gap = abs(otr["delta"][k, i] - math.log(otr["u"][k, i]))
        assert gap < NEAR_TIE, f"member decision differs at sweep {k}, member {i}: |Delta - ln u| = {gap}"
        masked_from[i] = k + 1
        ties.append((int(k), int(i)))
    k_m = ties[0][0] if ties else T
    valid = np.arange(k_mem)[:, None] < masked_from[None, :]
    rel_k = np.broadcast_to((DELTA_REL + DELTA_DRIFT * np.arange(k_mem))[:, None], valid.shape)
    ok, worst = _close(tr["delta"][:k_mem][valid], otr["delta"][:k_mem][valid], rel=rel_k[valid])
    assert ok, f"member Delta differs: worst {worst:.3g} x tolerance"
    # proposals: sweep k's depends on theta after k - 1 and S_theta through step k - 2 (delayed RAM)
    k_p = min(T, k_t + 1, k_m + 2)
    ok, worst = _close(tr["theta_prop"][:k_p], otr["theta_prop"][:k_p])
    assert ok, f"theta proposals differ: {worst:.3g} x tol"
    # D and log alpha: every member's latent enters; compared before the first member divergence
    k_d = min(T, k_m, k_t + 1)
    atol = d_tolerance(s.n, d_atol)
    errs = {}
    for key in ("D", "logalpha"):
        a, b = tr[key][:k_d], otr[key][:k_d]
        fin = np.isfinite(a) & np.isfinite(b)
        assert np.array_equal(np.isfinite(a), np.isfinite(b)), key
        assert np.array_equal(a[~fin], b[~fin]), key
        err = np.abs(a[fin] - b[fin])
        tol = atol + (D_REL * np.abs(b[fin]) if key == "D" else 0.0)
        errs[key] = float(np.max(err, initial=0.0))
        assert np.all(err <= tol), f"{key} differs by {np.max(err - tol):.3g} beyond its bound at sweep " \
                                   f"{int(np.nonzero(fin)[0][np.argmax(err - tol)])}"
    d_err = errs["D"]
    # the selection integral at each traced proposal, against the oracle's rule at the same proposal
    # (the integral is compared as arithmetic, at the device's own theta')
    eb = tr["etabar"]
    if ch.model in (oracle.LF, oracle.BB1):
        rule = oracle.lf_etabar if ch.model == oracle.LF else oracle.bb1_etabar
        ks = np.nonzero(eb > 0)[0]
        assert ks.size > 0
        ref = np.array([rule(tr["theta_prop"][k], ch.consts) for k in ks])
        assert np.all(np.abs(eb[ks] - ref) <= 1e-13 * ref), "selection integral differs"
    if k_t == T:  # the kept theta rows are points of the common theta path
        ok, worst = _close(rows, orows)
        assert ok, f"theta rows differ: {worst:.3g} x tol"
    chi, S = s.chi()
    if k_mem == T:  # final latents and RAM factors of the members compared to the end
        keep = masked_from == T  # per member (latents and factors reshaped member-major)
        ok, worst = _close(np.asarray(chi).reshape(n, -1)[keep], np.asarray(ch.chi).reshape(n, -1)[keep])
        assert ok, f"latents differ: {worst:.3g} x tol"
        ok, worst = _close(np.asarray(S).reshape(n, -1)[keep], np.asarray(ch.S).reshape(n, -1)[keep])
        assert ok, f"RAM factors differ: {worst:.3g} x tol"
    th, Sth = s.theta()
    if k_t == T and k_m == T:  # S_theta depends on every log alpha
        ok, _ = _close(th, ch.theta)
        assert ok
        ok, _ = _close(Sth.reshape(-1), ch.S_theta)
        assert ok
    # per-member log targets of the device against the oracle's formula at the same (device) state
    lp = s.logdens(th)
    olp = oracle.member_logdens(ch.model, ch.y, ch.aux, ch.consts, chi, th)
    ok, worst = _close(lp, olp)
    assert ok, f"per-member log densities differ: {worst:.3g} x tol"
    summary = {"sweeps": T, "n": n, "member_ties": ties, "theta_tie": theta_tie, "members_compared_to": k_mem,
               "theta_compared_to": k_t, "D_compared_to": k_d, "D_err": d_err, "logalpha_err": errs["logalpha"],
               "logalpha_tol": atol}
    print("lockstep", summary)
    return summary


