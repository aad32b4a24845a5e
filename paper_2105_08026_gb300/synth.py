"""Seeded synthetic populations shaped like the paper's demonstrations.

This module only generates inputs (simulated catalogs and run settings). It
holds none of the sampler's arithmetic: no member log-densities, no selection
integral, no RAM or MH step. Both the CUDA path and the CPU oracle consume what
it produces; it imports neither.

Workloads (all numpy ``Generator(PCG64(seed))``):

- ``nn1_data``: normal-normal population, d = 1 (Sec. 3 reduced to one
  characteristic): chi_i ~ N(mu, tau^2), sigma_i ~ U[lo, hi], y_i ~ N(chi_i, sigma_i^2).
- ``lf_data``: thinned luminosity-function catalog (Sec. 4-5): L from a
  Schechter-form density (L/L*)^beta exp(-L/L*) truncated to L > L_low, distance
  r with density ~ r^2 on [0, r_max], flux F = L/(4 pi r^2) (Sec. 4.1), measured
  flux Fhat = F + N(0, sigma_F^2) with sigma_F = sigma_frac * F_th, kept iff
  Fhat > F_th (Sec. 5.2); F_th is chosen by Monte Carlo so that a fraction
  ``detect_frac`` of the population is detected.
- ``mvn3_data``: d = 3 normal population with condition-number-20 covariance and
  heteroscedastic diagonal measurement errors (Sec. 3 with unknown C_pop).
- ``bb1_data``: the paper's own simulation (Sec. 5.1-5.2): BB1 luminosity function, r ~ r^2 on
  [0, r_max], flux-dependent measurement error sigma(F), detection at nu = 5 times the error.
- ``nn3_data``: the paper's normal-normal benchmark (Sec. 3): chi_i ~ N(mu_pop, D R D) with the
  printed mu_pop, D and R, y_ij ~ N(chi_ij, sigma_j^2) with the printed sigma_j for every i.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


# ----------------------------------------------------------------- NN1 -----
@dataclass
class NN1Data:
    y: np.ndarray
    sigma: np.ndarray
    chi_true: np.ndarray
    mu: float
    tau: float


def nn1_data(n: int, mu: float = 2.0, tau: float = 0.8, sig_lo: float = 0.5, sig_hi: float = 1.5,
             seed: int = 1001) -> NN1Data:
    g = _rng(seed)
    chi = mu + tau * g.standard_normal(n)
    sigma = g.uniform(sig_lo, sig_hi, n)
    y = chi + sigma * g.standard_normal(n)
    return NN1Data(y=y, sigma=sigma, chi_true=chi, mu=mu, tau=tau)


# ----------------------------------------------------------------- LF ------
@dataclass
class LFData:
    fhat: np.ndarray
    r: np.ndarray
    L_true: np.ndarray
    F_th: float
    sigma_F: float
    r_max: float
    beta: float
    L_star: float
    L_low: float
    n_drawn: int


def _schechter_draw(g: np.random.Generator, m: int, beta: float, L_star: float, L_low: float) -> np.ndarray:
    """m draws of L with density ~ (L/L*)^beta exp(-L/L*) on L > L_low (rejection sampling)."""
    out = np.empty(0)
    while out.size < m:
        k = max(2 * (m - out.size), 1024)
        if beta < -1.0:
            # Pareto proposal ~ L^beta on [L_low, inf), accepted with exp(-(L - L_low)/L*)
            v = 1.0 - g.random(k)  # (0, 1]
            with np.errstate(over="ignore"):  # overflow -> inf, rejected below
                L = L_low * v ** (1.0 / (beta + 1.0))
            keep = g.random(k) < np.exp(-(L - L_low) / L_star)
        else:
            # gamma(beta+1, L*) proposal restricted to L > L_low
            L = g.gamma(beta + 1.0, L_star, k)
            keep = L > L_low
        out = np.concatenate([out, L[keep]])
    return out[:m]


def _population(g, m, beta, L_star, L_low, r_max):
    L = _schechter_draw(g, m, beta, L_star, L_low)
    r = r_max * g.random(m) ** (1.0 / 3.0)
    r = np.maximum(r, 1e-300)
    return L, r


def solve_threshold(beta: float, L_star: float, L_low: float, r_max: float, detect_frac: float,
                    sigma_frac: float, seed: int, m: int = 400_000) -> float:
    """F_th with P(Fhat > F_th) = detect_frac over the population, by bisection on a fixed
    Monte Carlo sample (sigma_F = sigma_frac * F_th inside the criterion)."""
    g = _rng(seed + 7_000_003)
    L, r = _population(g, m, beta, L_star, L_low, r_max)
    F = L / (4.0 * math.pi * r * r)
    z = g.standard_normal(m)
    lo, hi = np.log(np.quantile(F, 1e-3)), np.log(np.quantile(F, 1.0 - 1e-4))

    def frac(lf):
        fth = math.exp(lf)
        return float(np.mean(F + sigma_frac * fth * z > fth))

    for _ in range(80):
        mid = 0.5 * (lo + hi)
        if frac(mid) > detect_frac:
            lo = mid
        else:
            hi = mid
    return math.exp(0.5 * (lo + hi))


def lf_data(n: int, beta: float = -1.2, L_star: float = 1e10, L_low: float = 1e8, r_max: float = 4000.0,
            detect_frac: float = 0.30, sigma_frac: float = 0.2, seed: int = 1002, mc: int = 400_000) -> LFData:
    F_th = solve_threshold(beta, L_star, L_low, r_max, detect_frac, sigma_frac, seed, m=mc)
    sigma_F = sigma_frac * F_th
    g = _rng(seed)
    fh, rr, LL = [], [], []
    got, drawn = 0, 0
    while got < n:
        m = int((n - got) / max(detect_frac, 1e-3) * 1.2) + 1024
        L, r = _population(g, m, beta, L_star, L_low, r_max)
        F = L / (4.0 * math.pi * r * r)
        fhat = F + sigma_F * g.standard_normal(m)
        keep = fhat > F_th
        idx = np.nonzero(keep)[0]
        need = n - got
        if idx.size > need:
            drawn += int(idx[need - 1]) + 1
            idx = idx[:need]
        else:
            drawn += m
        fh.append(fhat[idx]); rr.append(r[idx]); LL.append(L[idx])
        got += idx.size
    return LFData(fhat=np.concatenate(fh), r=np.concatenate(rr), L_true=np.concatenate(LL), F_th=F_th,
                  sigma_F=sigma_F, r_max=r_max, beta=beta, L_star=L_star, L_low=L_low, n_drawn=drawn)


# ----------------------------------------------------------------- BB1 -----
@dataclass
class BB1Data:
    fhat: np.ndarray
    r: np.ndarray
    L_true: np.ndarray
    sigma0: float
    alpha: float
    nu: float
    F_th: float
    r_max: float
    beta: float
    l: float
    u: float
    n_drawn: int


def _bb1_draw(g: np.random.Generator, m: int, beta: float, l: float, u: float) -> np.ndarray:
    """m draws of L with density ~ (1 - e^{-L/l}) (L/u)^beta e^{-L/u} (the BB1 form), -2 < beta < -1,
    by rejection from the envelope min(1, L/l) L^beta: a power law L^(beta+1) on (0, l) and a Pareto
    L^beta on [l, inf), accepted with probability (1 - e^{-L/l})/min(1, L/l) * e^{-L/u} (>= 0.63 e^{-L/u})."""
    assert -2.0 < beta < -1.0
    mA = l ** (beta + 1.0) / (beta + 2.0)    # int_0^l L^(beta+1)/l dL
    mB = l ** (beta + 1.0) / (-beta - 1.0)   # int_l^inf L^beta dL
    out = np.empty(0)
    while out.size < m:
        k = max(2 * (m - out.size), 4096)
        first = g.random(k) < mA / (mA + mB)
        v = 1.0 - g.random(k)  # (0, 1]
        with np.errstate(over="ignore", divide="ignore"):
            L = np.where(first, l * v ** (1.0 / (beta + 2.0)), l * v ** (1.0 / (beta + 1.0)))
            x = L / l
            ratio = np.where(x < 1.0, -np.expm1(-x) / x, -np.expm1(-x)) * np.exp(-L / u)
        keep = np.isfinite(L) & (L > 0.0) & (g.random(k) < ratio)
        out = np.concatenate([out, L[keep]])
    return out[:m]


def bb1_threshold(sigma0: float, alpha: float, nu: float) -> float:
    """F_th = nu sigma0/sqrt(1 - alpha^2): the flux whose estimate is nu times its error (Sec. 5.2)."""
    return nu * sigma0 / math.sqrt(1.0 - alpha * alpha)


def bb1_data(n: int, beta: float = -1.5, l: float = 1e8, u: float = 1e10, r_max: float = 1.0, alpha: float = 1e-2,
             nu: float = 5.0, seed: int = 1004) -> BB1Data:
    """Detected catalog of the paper's BB1 simulation (Sec. 5.1-5.2): L from the BB1 form, r with density
    ~ r^2 on [0, r_max], F = L/(4 pi r^2), Fhat = F + sigma(F) N(0, 1) with sigma(F)^2 = sigma0^2 + (alpha F)^2,
    kept iff Fhat > F_th = nu sigma0/sqrt(1 - alpha^2). sigma0 is set, as the paper chooses it, so that a
    source with L = 20 u at r = r_max sits at the threshold: F_th = 20 u/(4 pi r_max^2). Units: L in solar
    luminosities, r in Gpc, fluxes in L_sun/Gpc^2."""
    F_th = 20.0 * u / (4.0 * math.pi * r_max * r_max)
    sigma0 = F_th * math.sqrt(1.0 - alpha * alpha) / nu
    g = _rng(seed)
    fh, rr, LL = [], [], []
    got, drawn = 0, 0
    while got < n:
        m = 2_000_000
        L = _bb1_draw(g, m, beta, l, u)
        r = np.maximum(r_max * g.random(m) ** (1.0 / 3.0), 1e-300)
        F = L / (4.0 * math.pi * r * r)
        sig = np.sqrt(sigma0 * sigma0 + (alpha * F) ** 2)
        fhat = F + sig * g.standard_normal(m)
        idx = np.nonzero(fhat > F_th)[0]
        need = n - got
        if idx.size > need:
            drawn += int(idx[need - 1]) + 1
            idx = idx[:need]
        else:
            drawn += m
        fh.append(fhat[idx]); rr.append(r[idx]); LL.append(L[idx])
        got += idx.size
    return BB1Data(fhat=np.concatenate(fh), r=np.concatenate(rr), L_true=np.concatenate(LL), sigma0=sigma0,
                   alpha=alpha, nu=nu, F_th=F_th, r_max=r_max, beta=beta, l=l, u=u, n_drawn=drawn)


def bb1_settings(data: BB1Data, nL: int = 1024, nr: int = 1024, ln_upper: float = math.log(60.0),
                 ln_lower: float = -40.0):
    """theta_init (truth: beta, ln l, ln u), theta_prop_scale, consts of the BB1 model."""
    theta0 = np.array([data.beta, math.log(data.l), math.log(data.u)])
    scale = np.array([0.01, 0.01, 0.01])
    consts = np.array([data.sigma0, data.alpha, data.nu, data.r_max, float(nL), float(nr), ln_upper, ln_lower])
    return theta0, scale, consts


def bb1_chi_init(data: BB1Data) -> np.ndarray:
    """Default start: chi_i = ln(4 pi r_i^2 max(Fhat_i, F_th))."""
    return np.log(4.0 * math.pi * data.r * data.r * np.maximum(data.fhat, data.F_th))


# ----------------------------------------------------------------- MVN3 ----
@dataclass
class MVN3Data:
    y: np.ndarray       # (n, 3)
    s: np.ndarray       # (n, 3)
    chi_true: np.ndarray
    mu: np.ndarray
    C_pop: np.ndarray


def mvn3_data(n: int, mu=(0.0, 1.0, -1.0), cond: float = 20.0, s_lo: float = 0.3, s_hi: float = 1.0,
              seed: int = 1003) -> MVN3Data:
    g = _rng(seed)
    Q, _ = np.linalg.qr(g.standard_normal((3, 3)))
    ev = np.array([1.0, math.sqrt(cond), cond])
    C = (Q * ev) @ Q.T
    C = 0.5 * (C + C.T)
    Lc = np.linalg.cholesky(C)
    mu = np.asarray(mu, dtype=np.float64)
    chi = mu + g.standard_normal((n, 3)) @ Lc.T
    s = g.uniform(s_lo, s_hi, (n, 3))
    y = chi + s * g.standard_normal((n, 3))
    return MVN3Data(y=y, s=s, chi_true=chi, mu=mu, C_pop=C)


def mvn3_theta_from(mu, C) -> np.ndarray:
    """theta layout of the d = 3 model: mu[3], then the Cholesky factor of C packed
    row-major (L11, L21, L22, L31, L32, L33) with the diagonal stored as logs."""
    L = np.linalg.cholesky(np.asarray(C, dtype=np.float64))
    return np.array([mu[0], mu[1], mu[2], math.log(L[0, 0]), L[1, 0], math.log(L[1, 1]), L[2, 0], L[2, 1],
                     math.log(L[2, 2])])


# Sec. 3 normal-normal benchmark: population means, marginal standard deviations D, correlation
# matrix R, measurement scales sigma_j (the values printed in that section).
NN3_MU = (1.2, -0.4, 3.4)
NN3_D = (2.3, 0.45, 13.4)
NN3_R = ((1.0, 0.3, -0.5), (0.3, 1.0, 0.54), (-0.5, 0.54, 1.0))
NN3_SIGMA = (1.2, 0.4, 0.24)


def nn3_cov() -> np.ndarray:
    """C_pop = D R D of the Sec. 3 benchmark."""
    D = np.diag(NN3_D)
    return D @ np.array(NN3_R) @ D


def nn3_data(n: int, seed: int = 1004) -> MVN3Data:
    """n members of the Sec. 3 benchmark population, measured with the common scales sigma_j."""
    g = _rng(seed)
    C = nn3_cov()
    Lc = np.linalg.cholesky(C)
    mu = np.array(NN3_MU)
    chi = mu + g.standard_normal((n, 3)) @ Lc.T
    s = np.tile(np.array(NN3_SIGMA), (n, 1))
    y = chi + s * g.standard_normal((n, 3))
    return MVN3Data(y=y, s=s, chi_true=chi, mu=mu, C_pop=C)


def nn3_consts(C) -> np.ndarray:
    """Model constants of NN3: C_pop's lower triangle packed row-major (C11, C21, C22, C31, C32, C33)."""
    C = np.asarray(C, dtype=np.float64)
    return np.array([C[0, 0], C[1, 0], C[1, 1], C[2, 0], C[2, 1], C[2, 2]])


# ----------------------------------------------------------- run settings --
def nn3_settings(data: MVN3Data, scale: float = 0.05):
    """theta_init (the sample mean of y), theta_prop_scale, consts (C_pop known) for NN3."""
    return data.y.mean(axis=0).copy(), np.full(3, scale), nn3_consts(data.C_pop)


def nn1_settings(data: NN1Data):
    """theta_init, theta_prop_scale, consts for the NN1 model (flat mu, flat ln tau on [-10, 10])."""
    theta0 = np.array([float(np.mean(data.y)), math.log(max(float(np.std(data.y)), 1e-3))])
    scale = np.array([0.05, 0.05])
    consts = np.array([-10.0, 10.0])
    return theta0, scale, consts


def lf_settings(data: LFData, nL: int = 1024, nr: int = 1024, ln_upper: float = math.log(60.0)):
    """theta_init (truth), theta_prop_scale, consts for the luminosity model."""
    theta0 = np.array([data.beta, math.log(data.L_star), math.log(data.L_low)])
    scale = np.array([0.01, 0.01, 0.01])
    consts = np.array([data.sigma_F, data.F_th, data.r_max, float(nL), float(nr), ln_upper])
    return theta0, scale, consts


def mvn3_settings(data: MVN3Data, scale: float = 0.005):
    """theta_init, theta_prop_scale, consts for the d = 3 model: start from the sample mean
    of y and the Cholesky factor of the sample covariance of y (which is C_pop plus the mean
    measurement covariance, positive definite); the chain moves from there."""
    ybar = data.y.mean(axis=0)
    C = np.cov(data.y, rowvar=False) if data.y.shape[0] > 3 else np.eye(3)
    theta0 = mvn3_theta_from(ybar, C)
    return theta0, np.full(9, scale), np.zeros(1)


def lf_chi_init(data: LFData, theta) -> np.ndarray:
    """Default start: chi_i = ln(4 pi r_i^2 max(Fhat_i, F_th)), raised to ln L_low + 1e-6."""
    chi = np.log(4.0 * math.pi * data.r * data.r * np.maximum(data.fhat, data.F_th))
    return np.maximum(chi, theta[2] + 1e-6)


# ------------------------------------------------------ batched workloads --
@dataclass
class PopSpec:
    kind: str            # "nn1" or "lf"
    n: int
    seed: int
    params: dict


def batch_specs(k: int = 256, seed: int = 2000, n_lo: float = 1e3, n_hi: float = 1e6) -> list:
    """k populations, half normal-normal and half luminosity-function, each parameter of the
    single-population workloads scaled by U[0.8, 1.2], N log-uniform on [n_lo, n_hi]."""
    g = _rng(seed)
    out = []
    for q in range(k):
        n = int(round(math.exp(g.uniform(math.log(n_lo), math.log(n_hi)))))
        f = g.uniform(0.8, 1.2, 5)
        if q % 2 == 0:
            out.append(PopSpec("nn1", n, seed + q, dict(mu=2.0 * f[0], tau=0.8 * f[1])))
        else:
            out.append(PopSpec("lf", n, seed + q, dict(beta=-1.2 * f[0], L_star=1e10 * f[1], L_low=1e8 * f[2],
                                                       r_max=4000.0 * f[3], detect_frac=0.30 * f[4])))
    return out


def pop_data(spec: PopSpec, nL: int = 1024, nr: int = 1024):
    """(y, aux, theta_init, theta_prop_scale, consts) of one population of batch_specs."""
    if spec.kind == "nn1":
        d = nn1_data(spec.n, mu=spec.params["mu"], tau=spec.params["tau"], seed=spec.seed)
        th, sc, c = nn1_settings(d)
        return d.y, d.sigma, th, sc, c
    p = spec.params
    d = lf_data(spec.n, beta=p["beta"], L_star=p["L_star"], L_low=p["L_low"], r_max=p["r_max"],
                detect_frac=p["detect_frac"], seed=spec.seed, mc=100_000)
    th, sc, c = lf_settings(d, nL=nL, nr=nr)
    return d.fhat, d.r, th, sc, c
