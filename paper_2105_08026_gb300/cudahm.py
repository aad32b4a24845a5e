"""ctypes binding of the C ABI in ``include/cudahm.h`` (argument marshalling only).

Functions keep the C names (``cudahm_create``, ``cudahm_set_data``, ``cudahm_run``,
...). Every sweep runs in the CUDA library; there is no Python or CPU fallback: if
``lib/libcudahm.so`` is missing or fails to load, every call raises.

``Sampler`` is a small convenience wrapper that owns one handle. PyTorch is only
used, when asked, as the device allocator (its caching allocator) and as the source
of the CUDA stream.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "lib", "libcudahm.so")

ABI_VERSION = 1
OK, EINVAL, ENOMEM, ECUDA, ETIMEOUT, ENUMERIC, ESTATE, EUNSUPPORTED = 0, -1, -2, -3, -4, -5, -6, -7
NN1, MVN3, LF, BB1, NN3 = 0, 1, 2, 3, 4
FP64, FP32 = 0, 1
MAX_P = 9
MAX_CONSTS = 8
MODEL_D = {NN1: 1, MVN3: 3, LF: 1, BB1: 1, NN3: 3}
MODEL_P = {NN1: 2, MVN3: 9, LF: 3, BB1: 3, NN3: 3}
SHARD_WORDS = 16  # exchange words of one shard's sweep (CUDAHM_SHARD_WORDS)

ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)


class CudahmConfig(ctypes.Structure):
    _fields_ = [
        ("abi_version", ctypes.c_uint32),
        ("model", ctypes.c_int32),
        ("precision", ctypes.c_int32),
        ("d", ctypes.c_int32),
        ("n", ctypes.c_int64),
        ("seed", ctypes.c_uint64),
        ("target_accept", ctypes.c_double),
        ("adapt_exponent", ctypes.c_double),
        ("chi_init_scale", ctypes.c_double),
        ("theta_target_accept", ctypes.c_double),
        ("adapt_theta", ctypes.c_int32),
        ("trace_sweeps", ctypes.c_int32),
        ("theta_init", ctypes.c_double * MAX_P),
        ("theta_prop_scale", ctypes.c_double * MAX_P),
        ("model_consts", ctypes.c_double * MAX_CONSTS),
        ("device", ctypes.c_int32),
        ("block_threads", ctypes.c_int32),
        ("cuda_stream", ctypes.c_void_p),
        ("dev_alloc", ALLOC_FN),
        ("dev_free", FREE_FN),
        ("alloc_ctx", ctypes.c_void_p),
        ("barrier_timeout_ns", ctypes.c_int64),
        ("debug_skip_barrier_cta", ctypes.c_int32),
        ("marginal", ctypes.c_int32),
        ("keep_chi_moments", ctypes.c_int32),
    ]


class CudahmStats(ctypes.Structure):
    _fields_ = [
        ("sweeps", ctypes.c_int64),
        ("member_accepts", ctypes.c_int64),
        ("theta_accepts", ctypes.c_int64),
        ("rows", ctypes.c_int64),
        ("last_run_ms", ctypes.c_double),
        ("etabar", ctypes.c_double),
        ("grid_blocks", ctypes.c_int32),
        ("block_threads", ctypes.c_int32),
        ("objects_per_thread", ctypes.c_int32),
        ("reserved", ctypes.c_int32),
    ]


class CudahmTune(ctypes.Structure):
    _fields_ = [
        ("block_threads", ctypes.c_int32),
        ("sweeps_per_launch", ctypes.c_int32),
        ("use_graph", ctypes.c_int32),
        ("grid_blocks", ctypes.c_int32),
    ]


class CudahmError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"cudahm error {code}: {msg}")
        self.code = code


_dp = ctypes.POINTER(ctypes.c_double)
_u8p = ctypes.POINTER(ctypes.c_uint8)
_lib = None

EXPORTED = [
    "cudahm_config_init", "cudahm_create", "cudahm_set_data", "cudahm_set_data_device", "cudahm_set_chi",
    "cudahm_run", "cudahm_get_samples", "cudahm_get_chi", "cudahm_get_theta", "cudahm_get_stats",
    "cudahm_eval_logdens", "cudahm_eval_etabar", "cudahm_eval_detection", "cudahm_get_trace", "cudahm_checkpoint", "cudahm_restore",
    "cudahm_sizeof_config", "cudahm_sizeof_stats", "cudahm_last_error", "cudahm_destroy",
    "cudahm_lf_etabar_noalloc", "cudahm_batch_run", "cudahm_server_create", "cudahm_server_submit",
    "cudahm_server_poll", "cudahm_server_wait", "cudahm_server_result", "cudahm_server_stats",
    "cudahm_server_destroy", "cudahm_ess", "cudahm_eval_marginal", "cudahm_get_chi_moments",
    "cudahm_twostate_run", "cudahm_shard_config", "cudahm_shard_begin", "cudahm_shard_pass",
    "cudahm_shard_decide", "cudahm_shard_end",
]


def lib():
    """Load libcudahm.so (built by ``paper_2105_08026_gb300.build``); raise if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"CUDA library not built: {LIB_PATH} is missing (run __graft_entry__.build())")
    L = ctypes.CDLL(LIB_PATH)
    vp, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32
    L.cudahm_config_init.argtypes = [ctypes.POINTER(CudahmConfig), i32, i64]
    L.cudahm_config_init.restype = None
    L.cudahm_create.argtypes = [ctypes.POINTER(CudahmConfig), ctypes.POINTER(vp)]
    L.cudahm_set_data.argtypes = [vp, _dp, _dp, i64]
    L.cudahm_set_data_device.argtypes = [vp, vp, vp, i64]
    L.cudahm_set_chi.argtypes = [vp, _dp, i64]
    L.cudahm_run.argtypes = [vp, i64, i64, i64]
    L.cudahm_get_samples.argtypes = [vp, _dp, i64, ctypes.POINTER(i64)]
    L.cudahm_get_chi.argtypes = [vp, _dp, _dp]
    L.cudahm_get_theta.argtypes = [vp, _dp, _dp]
    L.cudahm_get_stats.argtypes = [vp, ctypes.POINTER(CudahmStats)]
    L.cudahm_eval_logdens.argtypes = [vp, _dp, _dp]
    L.cudahm_eval_etabar.argtypes = [vp, _dp, _dp]
    L.cudahm_eval_detection.argtypes = [vp, _dp, _dp, i64]
    L.cudahm_get_trace.argtypes = [vp, _dp, _dp, _u8p, _dp, _dp, _dp, _dp, _u8p, _dp, ctypes.POINTER(i64)]
    L.cudahm_checkpoint.argtypes = [vp, vp, ctypes.c_size_t, ctypes.POINTER(ctypes.c_size_t)]
    L.cudahm_restore.argtypes = [vp, vp, ctypes.c_size_t]
    L.cudahm_sizeof_config.restype = ctypes.c_size_t
    L.cudahm_sizeof_stats.restype = ctypes.c_size_t
    L.cudahm_last_error.restype = ctypes.c_char_p
    L.cudahm_lf_etabar_noalloc.argtypes = [vp, _dp, vp, vp]
    L.cudahm_server_create.argtypes = [ctypes.c_size_t, i32, i32, i32, i32, ctypes.POINTER(vp)]
    L.cudahm_server_submit.argtypes = [vp, ctypes.POINTER(CudahmConfig), _dp, _dp, i64, i64, i64,
                                       ctypes.POINTER(ctypes.c_uint64)]
    L.cudahm_server_poll.argtypes = [vp, ctypes.c_uint64, ctypes.POINTER(i32)]
    L.cudahm_server_wait.argtypes = [vp, ctypes.c_uint64, i64]
    L.cudahm_server_result.argtypes = [vp, ctypes.c_uint64, _dp, i64, ctypes.POINTER(i64), _dp]
    L.cudahm_server_stats.argtypes = [vp, ctypes.POINTER(i64), _dp, _dp, ctypes.POINTER(i64), ctypes.POINTER(i64)]
    L.cudahm_server_destroy.argtypes = [vp]
    L.cudahm_batch_run.argtypes = [ctypes.POINTER(vp), i32, i64, i64, i64, ctypes.POINTER(CudahmTune),
                                   ctypes.POINTER(CudahmTune)]
    L.cudahm_destroy.argtypes = [vp]
    L.cudahm_destroy.restype = None
    L.cudahm_ess.argtypes = [_dp, i64, i32, _dp]
    L.cudahm_eval_marginal.argtypes = [vp, _dp, _dp]
    L.cudahm_get_chi_moments.argtypes = [vp, _dp, _dp, ctypes.POINTER(i64)]
    L.cudahm_twostate_run.argtypes = [ctypes.c_double, i32, i64, i64, ctypes.c_uint64, i32, ctypes.POINTER(i64)]
    L.cudahm_shard_config.argtypes = [vp, i64, i64, i32, i32]
    L.cudahm_shard_begin.argtypes = [vp, i64, i64, i64]
    L.cudahm_shard_pass.argtypes = [vp, vp]
    L.cudahm_shard_decide.argtypes = [vp, vp]
    L.cudahm_shard_end.argtypes = [vp, ctypes.POINTER(i64)]
    for name in EXPORTED:
        if name not in ("cudahm_config_init", "cudahm_sizeof_config", "cudahm_sizeof_stats", "cudahm_last_error",
                        "cudahm_destroy"):
            getattr(L, name).restype = ctypes.c_int
    if L.cudahm_sizeof_config() != ctypes.sizeof(CudahmConfig):
        raise RuntimeError("cudahm_config layout mismatch between the binding and the library")
    if L.cudahm_sizeof_stats() != ctypes.sizeof(CudahmStats):
        raise RuntimeError("cudahm_stats layout mismatch between the binding and the library")
    _lib = L
    return L


def _check(rc: int):
    if rc != OK:
        raise CudahmError(rc, lib().cudahm_last_error().decode(errors="replace"))


def _dptr(a):
    return a.ctypes.data_as(_dp) if a is not None else None


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


# ------------------------------------------------------------- C-named calls --
def cudahm_config_init(model: int, n: int) -> CudahmConfig:
    cfg = CudahmConfig()
    lib().cudahm_config_init(ctypes.byref(cfg), model, n)
    return cfg


def cudahm_create(cfg: CudahmConfig) -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    _check(lib().cudahm_create(ctypes.byref(cfg), ctypes.byref(h)))
    return h


def cudahm_set_data(h, y, aux):
    y, aux = _f64(y), _f64(aux)
    n = y.shape[0] if y.ndim else 0
    _check(lib().cudahm_set_data(h, _dptr(y), _dptr(aux), n))


def cudahm_set_data_device(h, y_ptr: int, aux_ptr: int, n: int):
    _check(lib().cudahm_set_data_device(h, ctypes.c_void_p(y_ptr), ctypes.c_void_p(aux_ptr), n))


def cudahm_set_chi(h, chi):
    chi = _f64(chi)
    n = chi.shape[0]
    _check(lib().cudahm_set_chi(h, _dptr(chi), n))


def cudahm_run(h, n_burn: int, n_iter: int, thin: int = 1):
    _check(lib().cudahm_run(h, n_burn, n_iter, thin))


def cudahm_get_samples(h, p: int, cap_rows: int) -> np.ndarray:
    out = np.zeros((max(cap_rows, 1), p))
    rows = ctypes.c_int64(0)
    _check(lib().cudahm_get_samples(h, _dptr(out), cap_rows, ctypes.byref(rows)))
    return out[: min(rows.value, cap_rows)].copy()


def cudahm_get_chi(h, n: int, d: int):
    chi = np.zeros(n * d)
    S = np.zeros(n * d * d)
    _check(lib().cudahm_get_chi(h, _dptr(chi), _dptr(S)))
    return chi, S


def cudahm_get_chi_moments(h, n: int, d: int):
    """(mean, var, count) of the latents over the kept sweeps; mean and var shaped (n, d)."""
    mean = np.zeros(n * d)
    var = np.zeros(n * d)
    cnt = ctypes.c_int64(0)
    _check(lib().cudahm_get_chi_moments(h, _dptr(mean), _dptr(var), ctypes.byref(cnt)))
    return mean.reshape(n, d), var.reshape(n, d), cnt.value


def cudahm_twostate_run(pi1: float, precision: int, n_chains: int, sweeps: int, seed: int = 1,
                        device: int = 0) -> np.ndarray:
    """Transition counts [[0->0, 0->1], [1->0, 1->1]] of the two-state test model of the accept rule."""
    c = (ctypes.c_int64 * 4)()
    _check(lib().cudahm_twostate_run(float(pi1), int(precision), int(n_chains), int(sweeps),
                                     int(seed) & 0xFFFFFFFFFFFFFFFF, int(device), c))
    return np.array(list(c), dtype=np.int64).reshape(2, 2)


def cudahm_get_theta(h, p: int):
    th = np.zeros(p)
    St = np.zeros(p * p)
    _check(lib().cudahm_get_theta(h, _dptr(th), _dptr(St)))
    return th, St.reshape(p, p)


def cudahm_get_stats(h) -> CudahmStats:
    s = CudahmStats()
    _check(lib().cudahm_get_stats(h, ctypes.byref(s)))
    return s


def cudahm_eval_logdens(h, theta, n: int) -> np.ndarray:
    th = _f64(theta)
    out = np.zeros(n)
    _check(lib().cudahm_eval_logdens(h, _dptr(th), _dptr(out)))
    return out


def cudahm_eval_marginal(h, theta, n: int) -> np.ndarray:
    th = _f64(theta)
    out = np.zeros(n)
    _check(lib().cudahm_eval_marginal(h, _dptr(th), _dptr(out)))
    return out


def cudahm_eval_etabar(h, theta) -> float:
    th = _f64(theta)
    out = np.zeros(1)
    _check(lib().cudahm_eval_etabar(h, _dptr(th), _dptr(out)))
    return float(out[0])


def cudahm_eval_detection(h, F) -> np.ndarray:
    F = _f64(F)
    out = np.zeros(F.size)
    _check(lib().cudahm_eval_detection(h, _dptr(F), _dptr(out), F.size))
    return out


def cudahm_ess(x) -> np.ndarray:
    """Effective sample size of each column of a sample matrix (rows x cols), host-side."""
    x = _f64(x)
    if x.ndim == 1:
        x = x[:, None]
    out = np.zeros(x.shape[1])
    _check(lib().cudahm_ess(_dptr(x), x.shape[0], x.shape[1], _dptr(out)))
    return out


def cudahm_lf_etabar_noalloc(theta_dev_ptr: int, consts, etabar_dev_ptr: int, stream_ptr: int = 0):
    """Selection integral into caller-owned device memory, with no device allocation
    (theta_dev_ptr: 3 doubles, etabar_dev_ptr: 1 double, both on the current device)."""
    c = _f64(consts).reshape(-1)
    if c.size != 6:
        raise ValueError(f"consts must hold 6 values (sigma_F, F_th, r_max, n_L, n_r, ln(upper/L*)), got {c.size}")
    _check(lib().cudahm_lf_etabar_noalloc(ctypes.c_void_p(theta_dev_ptr), _dptr(c), ctypes.c_void_p(etabar_dev_ptr),
                                          ctypes.c_void_p(stream_ptr) if stream_ptr else None))


def cudahm_batch_run(handles, n_burn: int, n_iter: int, thin: int = 1, tune: CudahmTune = None) -> CudahmTune:
    """Run several populations in one persistent launch per chunk; returns the launch shape used."""
    arr = (ctypes.c_void_p * len(handles))(*[h.value if isinstance(h, ctypes.c_void_p) else h for h in handles])
    chosen = CudahmTune()
    _check(lib().cudahm_batch_run(arr, len(handles), n_burn, n_iter, thin,
                                  ctypes.byref(tune) if tune is not None else None, ctypes.byref(chosen)))
    return chosen


def batch_run(samplers, n_burn: int, n_iter: int, thin: int = 1, tune: CudahmTune = None):
    """cudahm_batch_run over Sampler objects; returns (theta rows per sampler, launch shape)."""
    chosen = cudahm_batch_run([s.h for s in samplers], n_burn, n_iter, thin, tune)
    cap = n_iter // thin if (n_iter > 0 and thin > 0) else 0
    rows = [cudahm_get_samples(s.h, s.p, cap) if cap > 0 else np.zeros((0, s.p)) for s in samplers]
    return rows, chosen


def cudahm_shard_config(h, member_offset: int, population_n: int, part: int, parts: int):
    _check(lib().cudahm_shard_config(h, member_offset, population_n, part, parts))


def cudahm_shard_begin(h, n_burn: int, n_iter: int, thin: int = 1):
    _check(lib().cudahm_shard_begin(h, n_burn, n_iter, thin))


def cudahm_shard_pass(h, words_dev_ptr: int):
    _check(lib().cudahm_shard_pass(h, ctypes.c_void_p(words_dev_ptr)))


def cudahm_shard_decide(h, total_dev_ptr: int):
    _check(lib().cudahm_shard_decide(h, ctypes.c_void_p(total_dev_ptr)))


def cudahm_shard_end(h) -> int:
    rows = ctypes.c_int64(0)
    _check(lib().cudahm_shard_end(h, ctypes.byref(rows)))
    return rows.value


def make_config(model: int, n: int, *, theta_init, theta_prop_scale=None, model_consts=None, seed: int = 1,
                precision: int = FP64, adapt_theta: bool = True, device: int = 0) -> CudahmConfig:
    cfg = cudahm_config_init(model, n)
    cfg.precision = precision
    cfg.seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    cfg.adapt_theta = 1 if adapt_theta else 0
    cfg.device = device
    for q, v in enumerate(_f64(theta_init)):
        cfg.theta_init[q] = v
    if theta_prop_scale is not None:
        for q, v in enumerate(_f64(theta_prop_scale)):
            cfg.theta_prop_scale[q] = v
    if model_consts is not None:
        for q, v in enumerate(_f64(model_consts)):
            cfg.model_consts[q] = v
    return cfg


class Server:
    """Request loop with continuous batching (cudahm_server_*)."""

    def __init__(self, mem_budget_bytes: int, device: int = 0, precision: int = FP32, max_active: int = 256,
                 sweeps_per_step: int = 250):
        self.h = ctypes.c_void_p()
        self.precision = precision
        _check(lib().cudahm_server_create(int(mem_budget_bytes), device, precision, max_active, sweeps_per_step,
                                          ctypes.byref(self.h)))
        self.p_of = {}

    def submit(self, cfg: CudahmConfig, y, aux, n_burn: int, n_iter: int, thin: int = 1) -> int:
        y, aux = _f64(y), _f64(aux)
        t = ctypes.c_uint64(0)
        _check(lib().cudahm_server_submit(self.h, ctypes.byref(cfg), _dptr(y), _dptr(aux), n_burn, n_iter, thin,
                                          ctypes.byref(t)))
        self.p_of[t.value] = (MODEL_P[cfg.model], n_iter // thin if n_iter > 0 else 0)
        return t.value

    def poll(self, ticket: int) -> bool:
        d = ctypes.c_int32(0)
        _check(lib().cudahm_server_poll(self.h, ticket, ctypes.byref(d)))
        return bool(d.value)

    def wait(self, ticket: int, timeout_ms: int = -1):
        _check(lib().cudahm_server_wait(self.h, ticket, timeout_ms))

    def result(self, ticket: int):
        p, cap = self.p_of.pop(ticket)
        out = np.zeros((max(cap, 1), p))
        rows = ctypes.c_int64(0)
        lat = ctypes.c_double(0.0)
        _check(lib().cudahm_server_result(self.h, ticket, _dptr(out), cap, ctypes.byref(rows), ctypes.byref(lat)))
        return out[: rows.value].copy(), lat.value

    def stats(self):
        c, q, a = ctypes.c_int64(0), ctypes.c_int64(0), ctypes.c_int64(0)
        ms, busy = ctypes.c_double(0.0), ctypes.c_double(0.0)
        _check(lib().cudahm_server_stats(self.h, ctypes.byref(c), ctypes.byref(ms), ctypes.byref(busy),
                                         ctypes.byref(q), ctypes.byref(a)))
        return dict(completed=c.value, member_sweeps=ms.value, busy_ms=busy.value, queued=q.value, active=a.value)

    def close(self):
        if self.h:
            lib().cudahm_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def cudahm_get_trace(h, n: int, p: int, T: int):
    tr = dict(delta=np.zeros((T, n)), u=np.zeros((T, n)), acc=np.zeros((T, n), np.uint8),
              theta_prop=np.zeros((T, p)), D=np.zeros(T), logalpha=np.zeros(T), utheta=np.zeros(T),
              tacc=np.zeros(T, np.uint8), etabar=np.zeros(T))
    t_out = ctypes.c_int64(0)
    _check(lib().cudahm_get_trace(h, _dptr(tr["delta"]), _dptr(tr["u"]), tr["acc"].ctypes.data_as(_u8p),
                                  _dptr(tr["theta_prop"]), _dptr(tr["D"]), _dptr(tr["logalpha"]),
                                  _dptr(tr["utheta"]), tr["tacc"].ctypes.data_as(_u8p), _dptr(tr["etabar"]),
                                  ctypes.byref(t_out)))
    if t_out.value != T:
        raise CudahmError(EINVAL, f"trace holds {t_out.value} sweeps, asked for {T}")
    return tr


def cudahm_checkpoint(h) -> bytes:
    used = ctypes.c_size_t(0)
    _check(lib().cudahm_checkpoint(h, None, 0, ctypes.byref(used)))
    buf = ctypes.create_string_buffer(used.value)
    _check(lib().cudahm_checkpoint(h, buf, used.value, ctypes.byref(used)))
    return buf.raw


def cudahm_restore(h, blob: bytes):
    buf = ctypes.create_string_buffer(blob, len(blob))
    _check(lib().cudahm_restore(h, buf, len(blob)))


def cudahm_destroy(h):
    if h:
        lib().cudahm_destroy(h)


# --------------------------------------------------------------- convenience --
class _TorchAllocator:
    """Device allocator callbacks backed by torch's caching allocator."""

    def __init__(self, device: int):
        import torch
        self.torch = torch
        self.device = device
        self.alloc_cb = ALLOC_FN(self._alloc)
        self.free_cb = FREE_FN(self._free)

    def _alloc(self, nbytes, ctx):
        try:
            return int(self.torch.cuda.caching_allocator_alloc(int(nbytes), self.device))
        except Exception:  # out of memory -> the library reports ENOMEM
            return None

    def _free(self, ptr, ctx):
        if ptr:
            self.torch.cuda.caching_allocator_delete(int(ptr))


class Sampler:
    """One population and its chain (owns a cudahm handle)."""

    def __init__(self, model: int, n: int, *, theta_init, theta_prop_scale=None, model_consts=None, seed: int = 1,
                 precision: int = FP64, adapt_theta: bool = True, chi_init_scale: float = 1.0,
                 target_accept: float = 0.4, theta_target_accept: float = 0.4, adapt_exponent: float = 2.0 / 3.0,
                 trace_sweeps: int = 0, device: int = 0, block_threads: int = 0, stream=None,
                 use_torch_allocator: bool = False, barrier_timeout_ns: int = 0, debug_skip_barrier_cta: int = -1,
                 marginal: bool = False, keep_chi_moments: bool = False):
        self.model, self.n = model, int(n)
        self.d, self.p = MODEL_D[model], MODEL_P[model]
        cfg = cudahm_config_init(model, n)
        cfg.precision = precision
        cfg.seed = int(seed) & 0xFFFFFFFFFFFFFFFF
        cfg.adapt_theta = 1 if adapt_theta else 0
        cfg.chi_init_scale = chi_init_scale
        cfg.target_accept = target_accept
        cfg.theta_target_accept = theta_target_accept
        cfg.adapt_exponent = adapt_exponent
        cfg.trace_sweeps = trace_sweeps
        cfg.device = device
        cfg.block_threads = block_threads
        cfg.barrier_timeout_ns = barrier_timeout_ns
        cfg.debug_skip_barrier_cta = debug_skip_barrier_cta
        cfg.marginal = 1 if marginal else 0
        cfg.keep_chi_moments = 1 if keep_chi_moments else 0
        for q, v in enumerate(_f64(theta_init)):
            cfg.theta_init[q] = v
        if theta_prop_scale is not None:
            for q, v in enumerate(_f64(theta_prop_scale)):
                cfg.theta_prop_scale[q] = v
        if model_consts is not None:
            for q, v in enumerate(_f64(model_consts)):
                cfg.model_consts[q] = v
        if stream is not None:
            cfg.cuda_stream = ctypes.c_void_p(int(stream))
        self._alloc = None
        if use_torch_allocator:
            self._alloc = _TorchAllocator(device)
            cfg.dev_alloc = self._alloc.alloc_cb
            cfg.dev_free = self._alloc.free_cb
        self.cfg = cfg
        self.h = cudahm_create(cfg)

    def close(self):
        if self.h:
            cudahm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_data(self, y, aux):
        cudahm_set_data(self.h, y, aux)

    def set_chi(self, chi):
        cudahm_set_chi(self.h, chi)

    def run(self, n_burn: int, n_iter: int, thin: int = 1) -> np.ndarray:
        cudahm_run(self.h, n_burn, n_iter, thin)
        cap = n_iter // thin if (n_iter > 0 and thin > 0) else 0
        return cudahm_get_samples(self.h, self.p, cap) if cap > 0 else np.zeros((0, self.p))

    def chi(self):
        c, S = cudahm_get_chi(self.h, self.n, self.d)
        return c, S

    def chi_moments(self):
        """(mean, var, count): each latent component's mean and sample variance over the kept
        sweeps, shaped (n, d) (needs keep_chi_moments)."""
        return cudahm_get_chi_moments(self.h, self.n, self.d)

    def theta(self):
        return cudahm_get_theta(self.h, self.p)

    def stats(self) -> CudahmStats:
        return cudahm_get_stats(self.h)

    def marginal_logp(self, theta=None) -> np.ndarray:
        th = self.theta()[0] if theta is None else theta
        return cudahm_eval_marginal(self.h, th, self.n)

    def logdens(self, theta=None) -> np.ndarray:
        th = self.theta()[0] if theta is None else theta
        return cudahm_eval_logdens(self.h, th, self.n)

    def etabar(self, theta) -> float:
        return cudahm_eval_etabar(self.h, theta)

    def detection(self, F) -> np.ndarray:
        return cudahm_eval_detection(self.h, F)

    def trace(self, T: int):
        return cudahm_get_trace(self.h, self.n, self.p, T)

    def checkpoint(self) -> bytes:
        return cudahm_checkpoint(self.h)

    def restore(self, blob: bytes):
        cudahm_restore(self.h, blob)

    # one shard of a population split across devices (the handle holds members
    # [member_offset, member_offset + n) of population_n)
    def shard(self, member_offset: int, population_n: int, part: int, parts: int):
        cudahm_shard_config(self.h, member_offset, population_n, part, parts)

    def run_sharded(self, n_burn: int, n_iter: int, thin: int, words, exchange) -> np.ndarray:
        """A sharded run: each sweep, this shard's pass writes its exchange words into `words`
        (a device buffer of SHARD_WORDS 64-bit integers, e.g. a torch int64 tensor), then
        ``exchange(words)`` must leave the sum over all shards in it (an all-reduce), then the
        decision. Returns the kept theta rows (the same on every shard)."""
        ptr = int(words.data_ptr())
        cudahm_shard_begin(self.h, n_burn, n_iter, thin)
        try:
            for _ in range(n_burn + n_iter):
                cudahm_shard_pass(self.h, ptr)
                exchange(words)
                cudahm_shard_decide(self.h, ptr)
        except BaseException:
            try:
                cudahm_shard_end(self.h)  # ends the run; the first error is the one raised
            except CudahmError:
                pass
            raise
        rows = cudahm_shard_end(self.h)
        return cudahm_get_samples(self.h, self.p, rows) if rows > 0 else np.zeros((0, self.p))
