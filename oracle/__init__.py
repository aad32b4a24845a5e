"""CPU FP64 oracle for the CUDAHM sampler (arXiv:2105.08026).

TEST INFRASTRUCTURE ONLY: the plain single-threaded reference that the CUDA
path is checked against. Only the test suite, ``__graft_entry__.smoke()`` and
the CPU-baseline / reference legs of ``bench.py`` may import this package. It
shares no code with the CUDA library (``paper_2105_08026_gb300``) and never
imports it; the CUDA library never imports this package.

The arithmetic lives in ``cudahm_oracle.c`` (built with ``-O2
-ffp-contract=off``, no fast-math); this module is ctypes marshalling plus the
pure-numpy Monte Carlo statistics in :mod:`oracle.stats`.

Parity status of each function is listed in the module docstring of
``cudahm_oracle.c`` and pinned by ``tests/test_oracle_*.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cudahm_oracle.c")
_LIB = os.path.join(_HERE, "libcudahm_oracle.so")
_lock = threading.Lock()
_lib = None

NN1, MVN3, LF, BB1, NN3 = 0, 1, 2, 3, 4
MODEL_D = {NN1: 1, MVN3: 3, LF: 1, BB1: 1, NN3: 3}
MODEL_P = {NN1: 2, MVN3: 9, LF: 3, BB1: 3, NN3: 3}

_dp = ctypes.POINTER(ctypes.c_double)
_u8p = ctypes.POINTER(ctypes.c_uint8)
_i64p = ctypes.POINTER(ctypes.c_int64)
_u32p = ctypes.POINTER(ctypes.c_uint32)


def build(force: bool = False) -> str:
    """Compile the oracle shared library with gcc (plain C99, strict FP64)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-std=c99", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
                               "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            L.orc_philox4x32_10.argtypes = [_u32p, _u32p, _u32p]
            L.orc_uniform.argtypes = [ctypes.c_uint32, ctypes.c_uint32]
            L.orc_uniform.restype = ctypes.c_double
            L.orc_draw.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32,
                                   ctypes.c_int, _dp, _dp]
            L.orc_draw_member.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_int, _dp, _dp]
            L.orc_neumaier_sum.argtypes = [_dp, ctypes.c_int64]
            L.orc_neumaier_sum.restype = ctypes.c_double
            L.orc_cholesky.argtypes = [ctypes.c_int, _dp, _dp]
            L.orc_ram_update.argtypes = [ctypes.c_int, _dp, _dp, ctypes.c_double, ctypes.c_double,
                                         ctypes.c_double]
            L.orc_gauss_legendre.argtypes = [ctypes.c_int, _dp, _dp]
            L.orc_lf_etabar.argtypes = [_dp, _dp]
            L.orc_lf_etabar.restype = ctypes.c_double
            L.orc_lf_detection.argtypes = [ctypes.c_double, _dp]
            L.orc_lf_detection.restype = ctypes.c_double
            L.orc_lf_H.argtypes = [ctypes.c_double, _dp]
            L.orc_lf_H.restype = ctypes.c_double
            L.orc_bb1_threshold.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_double]
            L.orc_bb1_threshold.restype = ctypes.c_double
            L.orc_bb1_detection.argtypes = [ctypes.c_double, _dp]
            L.orc_bb1_detection.restype = ctypes.c_double
            L.orc_bb1_H.argtypes = [ctypes.c_double, _dp]
            L.orc_bb1_H.restype = ctypes.c_double
            L.orc_bb1_etabar.argtypes = [_dp, _dp]
            L.orc_bb1_etabar.restype = ctypes.c_double
            L.orc_logf_obj.argtypes = [ctypes.c_int, ctypes.c_int, _dp, _dp, _dp]
            L.orc_logf_obj.restype = ctypes.c_double
            L.orc_member_logdens.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int64, _dp, _dp, _dp, _dp, _dp,
                                             _dp]
            L.orc_run.argtypes = ([ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int64, _dp, _dp, _dp, _dp,
                                   ctypes.c_uint64, _dp, _dp, _dp, _dp, _i64p, _dp,
                                   ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, _dp, _i64p, _i64p, _i64p,
                                   ctypes.c_int64, _dp, _dp, _u8p, _dp, _dp, _dp, _dp, _u8p, _dp, _dp, _dp, _dp,
                                   _i64p])
            L.orc_run.restype = ctypes.c_int
            L.orc_twostate_run.argtypes = [ctypes.c_double, ctypes.c_int64, ctypes.c_int64, ctypes.c_uint64, _i64p]
            L.orc_twostate_run.restype = None
            L.orc_marg_logp.argtypes = [ctypes.c_int, ctypes.c_int64, _dp, _dp, _dp, _dp, _dp]
            L.orc_marg_run.argtypes = ([ctypes.c_int, ctypes.c_int, ctypes.c_int64, _dp, _dp, _dp, _dp,
                                        ctypes.c_uint64, _dp, _dp, _dp, _i64p, _dp, ctypes.c_int64, ctypes.c_int64,
                                        ctypes.c_int64, _dp, _i64p, _i64p, ctypes.c_int64, _dp, _dp, _dp, _dp,
                                        _u8p, _dp])
            L.orc_marg_run.restype = ctypes.c_int
            L.orc_member_pass.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int64, _dp, _dp, _dp, _dp,
                                          ctypes.c_uint64, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, _dp, _dp,
                                          _dp, _dp, _dp, _i64p]
            L.orc_member_pass.restype = ctypes.c_int
            L.orc_lf_rule_new.argtypes = [_dp]
            L.orc_lf_rule_new.restype = ctypes.c_void_p
            L.orc_lf_rule_etabar.argtypes = [ctypes.c_void_p, _dp, _dp]
            L.orc_lf_rule_etabar.restype = ctypes.c_double
            L.orc_lf_rule_free.argtypes = [ctypes.c_void_p]
            _lib = L
    return _lib


def _p(a, t=_dp):
    if a is None:
        return None
    return a.ctypes.data_as(t)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


# ---------------------------------------------------------------- RNG ------
def philox4x32_10(ctr, key):
    """Philox4x32-10 block for one 4-word counter and 2-word key (Salmon et al. SC'11)."""
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32_10(_p(c, _u32p), _p(k, _u32p), _p(out, _u32p))
    return out


def uniform(wa: int, wb: int) -> float:
    return lib().orc_uniform(wa, wb)


def draw_member(seed: int, index: int, sweep: int, d: int):
    """d standard normals and the accept uniform of member `index` at sweep `sweep`."""
    z = np.zeros(max(d, 1), dtype=np.float64)
    u = ctypes.c_double(0.0)
    lib().orc_draw_member(seed, index, sweep, d, _p(z), ctypes.byref(u))
    return z[:d], u.value


def draw(seed: int, stream: int, index: int, sweep: int, d: int):
    """d standard normals and the accept uniform of one theta step (block j: normals 2j, 2j+1)."""
    z = np.zeros(max(d, 1), dtype=np.float64)
    u = ctypes.c_double(0.0)
    lib().orc_draw(seed, stream, index, sweep, d, _p(z), ctypes.byref(u))
    return z[:d], u.value


# ---------------------------------------------------------------- numerics -
def neumaier_sum(v) -> float:
    v = _f64(v)
    return lib().orc_neumaier_sum(_p(v), v.size)


def cholesky(A):
    A = _f64(A)
    d = A.shape[0]
    L = np.zeros_like(A)
    rc = lib().orc_cholesky(d, _p(A), _p(L))
    if rc != 0:
        raise np.linalg.LinAlgError("not positive definite")
    return L


def ram_update(S, U, alpha, alpha_star, eta):
    """RAM factor update (Sec. 2.2 step 3); returns the new lower factor."""
    S = _f64(S).copy()
    U = _f64(U)
    d = U.size
    rc = lib().orc_ram_update(d, _p(S), _p(U), alpha, alpha_star, eta)
    if rc != 0:
        raise np.linalg.LinAlgError("RAM update lost positive definiteness")
    return S


def gauss_legendre(n: int):
    x = np.zeros(n)
    w = np.zeros(n)
    lib().orc_gauss_legendre(n, _p(x), _p(w))
    return x, w


def lf_consts(sigma_F, F_th, r_max, nL=1024, nr=1024, ln_upper=float(np.log(60.0))):
    """Constants vector of the luminosity model: sigma_F, F_th, r_max, n_L, n_r, ln(upper/L*)."""
    return np.array([sigma_F, F_th, r_max, nL, nr, ln_upper], dtype=np.float64)


def lf_etabar(theta, consts) -> float:
    th = _f64(theta)
    c = _f64(consts)
    return lib().orc_lf_etabar(_p(th), _p(c))


def lf_detection(F, consts) -> np.ndarray:
    """eta(F) = Phi((F - F_th)/sigma_F) for an array of fluxes."""
    c = _f64(consts)
    return np.array([lib().orc_lf_detection(float(f), _p(c)) for f in np.atleast_1d(F)])


def lf_H(L, consts) -> float:
    c = _f64(consts)
    return lib().orc_lf_H(float(L), _p(c))


def bb1_consts(sigma0, alpha, nu, r_max, nL=1024, nr=1024, ln_upper=float(np.log(60.0)), ln_lower=-40.0):
    """Constants of the BB1 model: sigma0, alpha, nu, r_max, n_L, n_r, ln(upper/u), ln(lower/l)."""
    return np.array([sigma0, alpha, nu, r_max, nL, nr, ln_upper, ln_lower], dtype=np.float64)


def bb1_threshold(sigma0, alpha, nu) -> float:
    """F_th = nu sigma0/sqrt(1 - alpha^2) (Sec. 5.2, eq. Fth)."""
    return lib().orc_bb1_threshold(sigma0, alpha, nu)


def bb1_detection(F, consts) -> np.ndarray:
    """eta(F) = Phi((F - F_th)/sigma(F)), sigma(F)^2 = sigma0^2 + (alpha F)^2."""
    c = _f64(consts)
    return np.array([lib().orc_bb1_detection(float(f), _p(c)) for f in np.atleast_1d(F)])


def bb1_H(L, consts) -> float:
    c = _f64(consts)
    return lib().orc_bb1_H(float(L), _p(c))


def bb1_etabar(theta, consts) -> float:
    th = _f64(theta)
    c = _f64(consts)
    return lib().orc_bb1_etabar(_p(th), _p(c))


def logf_obj(model, chi, theta, consts=None) -> float:
    """log f_obj(chi;theta) of one member (the population term of its target); consts are
    needed by models that read them (NN3: the packed lower triangle of C_pop)."""
    c = _f64(np.atleast_1d(chi))
    th = _f64(theta)
    k = _f64(consts if consts is not None else np.zeros(8))
    return lib().orc_logf_obj(model, MODEL_D[model], _p(c), _p(th), _p(k))


def member_logdens(model, y, aux, consts, chi, theta):
    d = MODEL_D[model]
    y, aux, chi, theta = _f64(y), _f64(aux), _f64(chi), _f64(theta)
    consts = _f64(consts if consts is not None else np.zeros(1))
    n = chi.size // d
    out = np.zeros(n)
    lib().orc_member_logdens(model, d, n, _p(y), _p(aux), _p(consts), _p(chi), _p(theta), _p(out))
    return out


def member_pass(model, y, aux, consts, params, seed, k, i0, i1, theta, theta_prop, chi, S):
    """The member half of sweep k over members [i0, i1): updates chi and S (numpy arrays, in
    place) and returns d_i = log f(chi_i;theta') - log f(chi_i;theta) of the updated members and
    the number of accepts. params = (target_accept, adapt_exponent, ...)."""
    d = MODEL_D[model]
    y, aux, theta, theta_prop, params = _f64(y), _f64(aux), _f64(theta), _f64(theta_prop), _f64(params)
    consts = _f64(consts if consts is not None else np.zeros(1))
    out = np.zeros(max(i1 - i0, 1))
    acc = ctypes.c_int64(0)
    lib().orc_member_pass(model, d, y.size // d, _p(y), _p(aux), _p(consts), _p(params), int(seed), int(k), int(i0),
                          int(i1), _p(theta), _p(theta_prop), _p(chi), _p(S), _p(out), ctypes.byref(acc))
    return out[: i1 - i0], acc.value


def marg_logp(model, y, aux, consts, theta):
    """Per-member log p_i(theta) = log int l_i(chi) f(chi;theta) dchi by the cubature rule of
    the marginal form (NN1: aux = sigma_i; LF: aux = r_i)."""
    y, aux, theta = _f64(y), _f64(aux), _f64(theta)
    consts = _f64(consts if consts is not None else np.zeros(1))
    out = np.zeros(y.size)
    lib().orc_marg_logp(model, y.size, _p(y), _p(aux), _p(consts), _p(theta), _p(out))
    return out


class MarginalChain:
    """theta-only chain on the marginal posterior (latents integrated out by the cubature rule)."""

    def __init__(self, model, y, aux, consts, theta_init, theta_prop_scale, seed, adapt_exponent=2.0 / 3.0,
                 theta_target_accept=0.4, adapt_theta=True, keep_chi_moments=False):
        self.model = model
        self.p = MODEL_P[model]
        self.y = _f64(y)
        self.aux = _f64(aux)
        self.n = self.y.size
        self.consts = _f64(consts if consts is not None else np.zeros(1))
        self.seed = int(seed)
        self.params = np.array([0.4, adapt_exponent, theta_target_accept, 1.0 if adapt_theta else 0.0])
        self.theta = _f64(theta_init).copy()
        self.S_theta = np.diag(_f64(theta_prop_scale)).reshape(-1).copy()
        self.lp = marg_logp(model, self.y, self.aux, self.consts, self.theta)
        self.sweep = ctypes.c_int64(0)
        self.etabar = ctypes.c_double(0.0)
        self.theta_accepts = ctypes.c_int64(0)

    def run(self, n_burn, n_iter, thin=1, trace_sweeps=0):
        p = self.p
        total = n_burn + n_iter
        cap = (n_iter // thin) if thin > 0 else 0
        rows = np.zeros((max(cap, 1), p))
        rows_out = ctypes.c_int64(0)
        T = int(min(trace_sweeps, total))
        tr = None
        args_tr = [None] * 6
        if T > 0:
            tr = dict(theta_prop=np.zeros((T, p)), D=np.zeros(T), logalpha=np.zeros(T), utheta=np.zeros(T),
                      tacc=np.zeros(T, np.uint8), etabar=np.zeros(T))
            args_tr = [_p(tr["theta_prop"]), _p(tr["D"]), _p(tr["logalpha"]), _p(tr["utheta"]),
                       _p(tr["tacc"], _u8p), _p(tr["etabar"])]
        rc = lib().orc_marg_run(self.model, p, self.n, _p(self.y), _p(self.aux), _p(self.consts), _p(self.params),
                                self.seed, _p(self.theta), _p(self.S_theta), _p(self.lp), ctypes.byref(self.sweep),
                                ctypes.byref(self.etabar), n_burn, n_iter, thin, _p(rows), ctypes.byref(rows_out),
                                ctypes.byref(self.theta_accepts), T, *args_tr)
        if rc != 0:
            raise RuntimeError(f"oracle marginal run failed: {rc}")
        return rows[: rows_out.value].copy(), tr


def twostate_counts(pi1, n, sweeps, seed):
    """Transition counts [[0->0, 0->1], [1->0, 1->1]] of n two-state chains run with the member
    step's accept rule (Sec. 2.2), target (1 - pi1, pi1), flip proposal, for `sweeps` steps."""
    c = np.zeros(4, dtype=np.int64)
    lib().orc_twostate_run(float(pi1), int(n), int(sweeps), int(seed), c.ctypes.data_as(_i64p))
    return c.reshape(2, 2)


# ---------------------------------------------------------------- chain ----
class Chain:
    """State of one MWG chain run by the oracle (Sec. 2.1-2.2)."""

    def __init__(self, model, y, aux, consts, theta_init, theta_prop_scale, seed, chi0,
                 chi_init_scale=1.0, target_accept=0.4, adapt_exponent=2.0 / 3.0,
                 theta_target_accept=0.4, adapt_theta=True, keep_chi_moments=False):
        self.model = model
        self.d = MODEL_D[model]
        self.p = MODEL_P[model]
        self.y = _f64(y)
        self.aux = _f64(aux)
        self.n = self.y.size // self.d
        self.consts = _f64(consts if consts is not None else np.zeros(1))
        self.seed = int(seed)
        self.params = np.array([target_accept, adapt_exponent, theta_target_accept, 1.0 if adapt_theta else 0.0])
        self.chi = _f64(chi0).copy().reshape(-1)
        assert self.chi.size == self.n * self.d
        self.S = np.zeros((self.n, self.d, self.d))
        for a in range(self.d):
            self.S[:, a, a] = chi_init_scale
        self.S = self.S.reshape(-1).copy()
        self.theta = _f64(theta_init).copy()
        self.S_theta = np.diag(_f64(theta_prop_scale)).reshape(-1).copy()
        self.sweep = ctypes.c_int64(0)
        self.etabar = ctypes.c_double(0.0)
        self.member_accepts = ctypes.c_int64(0)
        self.theta_accepts = ctypes.c_int64(0)
        # running moments of the latents over the kept sweeps (Welford), when asked
        self.mom_mean = np.zeros(self.n * self.d) if keep_chi_moments else None
        self.mom_m2 = np.zeros(self.n * self.d) if keep_chi_moments else None
        self.mom_n = ctypes.c_int64(0)
        # theta RAM update pending from the last sweep (applied one sweep late): U, alpha, eta
        self.theta_pend = np.zeros(self.p + 2)

    def moments(self):
        """(mean, var, count): per-member mean and sample variance (M2/(count - 1), 0 for one
        sample) of every latent component over the kept sweeps so far, shaped (n, d)."""
        m = self.mom_n.value
        var = self.mom_m2 / (m - 1) if m > 1 else np.zeros_like(self.mom_m2)
        return self.mom_mean.reshape(self.n, self.d).copy(), var.reshape(self.n, self.d), m

    def run(self, n_burn, n_iter, thin=1, trace_sweeps=0):
        n, p = self.n, self.p
        total = n_burn + n_iter
        cap = (n_iter // thin) if thin > 0 else 0
        rows = np.zeros((max(cap, 1), p))
        rows_out = ctypes.c_int64(0)
        T = int(min(trace_sweeps, total))
        tr = None
        args_tr = [None] * 9
        if T > 0:
            tr = dict(delta=np.zeros((T, n)), u=np.zeros((T, n)), acc=np.zeros((T, n), np.uint8),
                      theta_prop=np.zeros((T, p)), D=np.zeros(T), logalpha=np.zeros(T), utheta=np.zeros(T),
                      tacc=np.zeros(T, np.uint8), etabar=np.zeros(T))
            args_tr = [_p(tr["delta"]), _p(tr["u"]), _p(tr["acc"], _u8p), _p(tr["theta_prop"]), _p(tr["D"]),
                       _p(tr["logalpha"]), _p(tr["utheta"]), _p(tr["tacc"], _u8p), _p(tr["etabar"])]
        rc = lib().orc_run(self.model, self.d, p, n, _p(self.y), _p(self.aux), _p(self.consts), _p(self.params),
                           self.seed, _p(self.chi), _p(self.S), _p(self.theta), _p(self.S_theta),
                           ctypes.byref(self.sweep), ctypes.byref(self.etabar), n_burn, n_iter, thin, _p(rows),
                           ctypes.byref(rows_out), ctypes.byref(self.member_accepts),
                           ctypes.byref(self.theta_accepts), T, *args_tr, _p(self.theta_pend),
                           _p(self.mom_mean) if self.mom_mean is not None else None,
                           _p(self.mom_m2) if self.mom_m2 is not None else None, ctypes.byref(self.mom_n))
        if rc != 0:
            raise RuntimeError(f"oracle run failed: {rc}")
        return rows[: rows_out.value].copy(), tr

    def member_logdens(self, theta=None):
        return member_logdens(self.model, self.y, self.aux, self.consts, self.chi,
                              self.theta if theta is None else theta)
