"""Benchmark of the CUDA MWG sampler on the thinned luminosity-function workload.

Workload (one "step" = one Metropolis-within-Gibbs sweep over all members, i.e. every
row of the hot path: theta proposal, N member RAM steps, the exact sum of
log f(chi_i;theta') - log f(chi_i;theta), the 1024 x 1024 selection-integral rule at
theta', the grid barrier, the theta accept and its RAM update, the kept-row record):
  N = 3e5 detected objects, Schechter-form population beta = -1.2, L* = 1e10,
  L_low = 1e8, distances ~ r^2 on [0, 4000], sigma_F = 0.2 F_th, F_th set for 30%
  detection; FP64 throughout. Synthetic catalog (seeded), no external data.

Metric: object-updates/s = N x sweeps / seconds (whole job over all ranks).
  value: device time of the timed sweeps (CUDA events on the sampler's stream), inputs
         resident in HBM, L2 flushed (256 MB write) before each timed launch;
  e2e:   the same metric through the public API with host buffers: set_data from host
         arrays, run, get_samples back to the host, every timed iteration.

Multi-GPU (torchrun): every rank runs an independent replica on its own catalog
(weak scaling, no collective on the data path); time = max over ranks.

--impl reference: the CPU FP64 oracle timed on the host on a bounded sample of the same
workload (rank 0 only).
"""
from __future__ import annotations

import argparse
import ctypes
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

N_OBJ = 300_000
DATA_SEED = 1002
CHAIN_SEED = 2
L2_FLUSH_BYTES = 256 << 20
# dram read+write bytes of one sweep-kernel launch (ncu, profiles/sweep_kernel_lf_n300000.md): the
# member data are read once per launch and the state stays in registers, so this does not grow
# with the sweeps of the launch.
DRAM_BYTES_PER_LAUNCH = 9.87e6

# FP64 floating-point work of one sweep of the LF workload (2 per DFMA, 1 per DADD/DMUL), from
# ncu's sm__sass_thread_inst_executed_op_d{fma,add,mul}_pred_on counters on the sweep kernel
# (profiles/sweep_kernel_lf_n300000.md; the difference between the 20- and 5-sweep launches, so
# without the launch's start-up): 115.0 per object-update including the selection rule.
FP64_FLOP_PER_SWEEP = 3.449e7

# FP64 work and DRAM traffic of one member-update of the d = 3 workload in the FP32 bulk form
# (profiles/batch_kernel_mvn3_n1000000_fp32.md).
MVN3_F32_FP64_FLOP_PER_UPDATE = 98.4
MVN3_F32_DRAM_BYTES_PER_UPDATE = 127.6

# Algorithmic HBM traffic of one member-update of the batched FP32 form (d = 1): binary32 data
# 16 B read, binary32 latent 4 B and binary64 RAM factor 8 B read and written.
BATCHED_F32_BYTES_PER_UPDATE = 40.0
HBM_FALLBACK_GBS = 6800.0


def hbm_peak():
    """The measured HBM copy bandwidth (GB/s) of this GPU type, from the peaks file beside this
    script, else the fallback figure; with a note saying which."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "of measured (copy bandwidth)"
    except (OSError, KeyError, ValueError, TypeError):
        return HBM_FALLBACK_GBS, "of fallback (6.8 TB/s)"


def batched_roofline(updates_per_s):
    """HBM roofline of the batched FP32 leg at the algorithmic 40 B per member-update."""
    peak, src = hbm_peak()
    ach = BATCHED_F32_BYTES_PER_UPDATE * updates_per_s / 1e9
    return {"bound": "hbm", "unit": "GB/s", "achieved": ach, "peak": peak, "frac": ach / peak, "peak_source": src,
            "bytes_per_update": BATCHED_F32_BYTES_PER_UPDATE, "kernel": "batch_kernel<FP32, d = 1>"}


# FP64 work of one member integral of the marginal form on the LF workload (96 nodes, with the
# step's share of the selection rule), from ncu's smsp__sass_thread_inst_executed_op_d{fma,add,mul}
# counters on marg_kernel<LF> (profiles/marg_kernel_lf_n300000.md): 2 DFMA + DADD + DMUL.
MARG_FP64_FLOP_PER_MEMBER = 4483.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5000)
    ap.add_argument("--warmup", type=int, default=1000)
    ap.add_argument("--impl", default="cuda", choices=["cuda", "reference"])
    ap.add_argument("--launch-sweeps", type=int, default=4096,
                    help="sweeps per timed run call (the library's persistent launch holds up to 4096)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-fp32", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--batched-sweeps", type=int, default=2000)
    ap.add_argument("--batched-pops", type=int, default=256)
    ap.add_argument("--batched-nlo", type=float, default=1e3, help="smallest population of the batched leg")
    ap.add_argument("--batched-block", type=int, default=0, help="batched leg launch shape (0: tuned)")
    ap.add_argument("--batched-grid", type=int, default=0)
    ap.add_argument("--batched-chunk", type=int, default=0)
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--serve-seconds", type=float, default=20.0)
    ap.add_argument("--serve-rate", type=float, default=20.0)
    ap.add_argument("--serve-sweeps", type=int, default=5000)
    ap.add_argument("--serve-pool", type=int, default=48)
    ap.add_argument("--serve-burst", type=int, default=96, help="requests of the saturated (all at t = 0) run")
    ap.add_argument("--serve-seq", type=int, default=40,
                    help="requests of the stream served by the sequential FP64 sampler")
    ap.add_argument("--cpu-sweeps", type=int, default=8)
    ap.add_argument("--no-mvn3", action="store_true")
    ap.add_argument("--no-bb1", action="store_true")
    ap.add_argument("--no-nn3", action="store_true")
    ap.add_argument("--no-marginal", action="store_true")
    ap.add_argument("--no-nn1", action="store_true")
    ap.add_argument("--no-moments", action="store_true")
    ap.add_argument("--no-shard", action="store_true")
    ap.add_argument("--marginal-burn", type=int, default=300)
    ap.add_argument("--marginal-steps", type=int, default=1500)
    ap.add_argument("--nn3-sizes", default="100,1000,10000,30000")
    ap.add_argument("--nn3-burn", type=int, default=40_000)
    ap.add_argument("--nn3-sweeps", type=int, default=75_000)
    ap.add_argument("--nn3-chains", type=int, default=64)
    ap.add_argument("--nn3-chain-sweeps", type=int, default=10_000)
    ap.add_argument("--nn3-chains-max-n", type=int, default=10_000)
    ap.add_argument("--bb1-sweeps", type=int, default=1000)
    ap.add_argument("--mvn3-sweeps", type=int, default=3000)
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def replica_seeds(rank: int):
    """(data seed, chain seed) of rank's replica: every rank samples its own catalog."""
    return DATA_SEED + rank, CHAIN_SEED + rank


def max_over_ranks(x: float, device: str = "cuda") -> float:
    """Largest x over the ranks of the default process group (x itself without one)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_value(world_size: int, units_per_rank: float, t_max_ms: float) -> float:
    """Whole-job throughput of independent replicas: all ranks' units over the slowest rank's time."""
    return world_size * units_per_rank / (t_max_ms * 1e-3)


def workload(rank):
    from paper_2105_08026_gb300 import synth
    data = synth.lf_data(N_OBJ, seed=replica_seeds(rank)[0])
    theta0, scale, consts = synth.lf_settings(data)
    return data, theta0, scale, consts


# ------------------------------------------------------------------ clocks ---
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (FileNotFoundError, OSError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 8:
                self.rows.append((time.perf_counter(), parts))

    def wait_first(self, limit_s=10.0):
        """Returns once the sampler has produced a row: the nvidia-smi process has started, so its
        start-up does not compete with the timed region's host work."""
        t_end = time.perf_counter() + limit_s
        while self.proc is not None and not self.rows and time.perf_counter() < t_end:
            time.sleep(0.05)

    def stop(self, t_lo=None, t_hi=None):
        """Median SM clock and throttle reasons over the samples taken in [t_lo, t_hi] (the timed
        region, widened by one sampling period on each side; all samples when none fall there)."""
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = self.rows
        if t_lo is not None and t_hi is not None:
            inside = [r for r in self.rows if t_lo - 0.25 <= r[0] <= t_hi + 0.25]
            rows = inside or self.rows
        rows = [r[1] for r in rows]
        sm = [float(r[0]) for r in rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[j] for r in rows for j in range(4) if r[4 + j].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# -------------------------------------------------------------- CPU oracle ---
def oracle_rate(data, theta0, scale, consts, sweeps, warmup=1):
    import oracle
    from paper_2105_08026_gb300 import synth
    chi0 = synth.lf_chi_init(data, theta0)
    ch = oracle.Chain(oracle.LF, data.fhat, data.r, consts, theta0, scale, CHAIN_SEED, chi0)
    ch.run(0, max(1, warmup))  # untimed; the first sweep also evaluates etabar at theta0
    t0 = time.perf_counter()
    ch.run(0, sweeps)
    dt = time.perf_counter() - t0
    return data.fhat.size * sweeps / dt, dt


def oracle_rate_allcores(data, theta0, scale, consts, sweeps, threads):
    """The oracle's LF chain on every host core: members split over threads, the theta step
    (with the 1024 x 1024 selection rule) serial (oracle/allcores.py)."""
    from oracle import allcores
    from paper_2105_08026_gb300 import synth
    chi0 = synth.lf_chi_init(data, theta0)
    allcores.lf_run(data.fhat, data.r, consts, theta0, scale, CHAIN_SEED, chi0, 1, threads)  # untimed
    _, _, _, dt = allcores.lf_run(data.fhat, data.r, consts, theta0, scale, CHAIN_SEED, chi0, sweeps, threads)
    return data.fhat.size * sweeps / dt, dt


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count()


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    data, theta0, scale, consts = workload(0)
    # a bounded sample of the workload: at most 15 timed and 3 untimed full sweeps (~0.1 s each on
    # one host core), so that the run ends within a few minutes whatever --steps asks
    sweeps = max(1, min(args.steps, 15))
    warm = max(1, min(args.warmup, 3))
    rate, dt = oracle_rate(data, theta0, scale, consts, sweeps, warm)
    sample = (f"{sweeps} timed full sweeps (after {warm} untimed) of the N={N_OBJ} LF workload "
              f"(1024x1024 rule), single-threaded oracle")
    line = {"impl": "reference", "metric": "object-updates/s", "value": rate, "unit": "object-updates/s",
            "n_gpus": 0, "steps": sweeps, "warmup": warm, "ms_per_step": dt * 1e3 / sweeps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "LF thinned luminosity function, N=3e5, FP64, 1024x1024 selection rule",
                       "n": N_OBJ, "sweeps_timed": sweeps},
            "cpu_baseline": {"value": rate, "unit": "object-updates/s", "cores": 1, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": rate, "unit": "object-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# -------------------------------------------------------------------- CUDA ---
PEAK_SRC = os.path.join(ROOT, "bench_fp64_peak.cu")
PEAK_LIB = os.path.join(ROOT, "_build", "libchm_peaks.so")


def build_peaks(force=False):
    """Compiles the FP64 peak probe (bench_fp64_peak.cu) that the roofline denominators use."""
    if not force and os.path.exists(PEAK_LIB) and os.path.getmtime(PEAK_LIB) >= os.path.getmtime(PEAK_SRC):
        return PEAK_LIB
    from paper_2105_08026_gb300 import build as cbuild
    os.makedirs(os.path.dirname(PEAK_LIB), exist_ok=True)
    tmp = PEAK_LIB + f".tmp{os.getpid()}"
    subprocess.check_call([cbuild.nvcc(), *cbuild.ARCH, "-O3", "-Xcompiler", "-fPIC", "-shared", "-o", tmp, PEAK_SRC])
    os.replace(tmp, PEAK_LIB)
    return PEAK_LIB


def fp64_peak(device):
    L = ctypes.CDLL(build_peaks())
    L.chm_fp64_dfma_rate.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_double)]
    r = ctypes.c_double(0.0)
    rc = L.chm_fp64_dfma_rate(device, ctypes.byref(r))
    return 2.0 * r.value if rc == 0 else None  # FP64 flop/s


def run_batched(args, cudahm, stream, device):
    """k populations (half NN1, half LF; parameters of the single-population workloads scaled
    by U[0.8, 1.2]; N log-uniform on [1e3, 1e6]), FP32 bulk form, one batched run timed with
    CUDA events on the batch stream (its autotuning launches are part of the run)."""
    import torch
    from paper_2105_08026_gb300 import synth
    specs = synth.batch_specs(args.batched_pops, seed=2000, n_lo=args.batched_nlo)
    samplers = []
    for sp in specs:
        y, aux, th, sc, c = synth.pop_data(sp)
        s = cudahm.Sampler(cudahm.NN1 if sp.kind == "nn1" else cudahm.LF, sp.n, theta_init=th, theta_prop_scale=sc,
                           model_consts=c, seed=sp.seed, precision=cudahm.FP32, device=device,
                           stream=stream.cuda_stream, use_torch_allocator=True)
        s.set_data(y, aux)
        samplers.append(s)
    members = sum(sp.n for sp in specs)
    K = args.batched_sweeps
    W = min(args.warmup, 50)
    tune = None
    if args.batched_block or args.batched_grid or args.batched_chunk:  # a fixed shape (profiling)
        tune = cudahm.CudahmTune(block_threads=args.batched_block, sweeps_per_launch=args.batched_chunk,
                                 use_graph=1, grid_blocks=args.batched_grid)
    if W > 0:
        cudahm.batch_run(samplers, W, 0, tune=tune)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    rows, chosen = cudahm.batch_run(samplers, 0, K, 1, tune=tune)
    e1.record(stream)
    e1.synchronize()
    ms = e0.elapsed_time(e1)
    assert all(r.shape[0] == K for r in rows)
    for s in samplers:
        s.close()
    value = members * K / (ms * 1e-3)
    return {"value": value, "unit": "object-updates/s", "ms_per_step": ms / K, "roofline": batched_roofline(value),
            "populations": len(specs), "members": members, "lf_populations": sum(sp.kind == "lf" for sp in specs),
            "steps": K, "launch": {"block_threads": chosen.block_threads,
                                   "sweeps_per_launch": chosen.sweeps_per_launch,
                                   "graph": bool(chosen.use_graph), "blocks": chosen.grid_blocks},
            "dtype": "f32 member terms, f64 sums/accept/RAM/selection integral (1024x1024 rule per LF population)"}


def run_shard(args, cudahm, rank, ws, local):
    """One LF population split over the ranks (every rank, a collective leg): rank r holds
    N_OBJ members (its own synthetic catalog, seed DATA_SEED + r; the model settings of catalog
    DATA_SEED on every rank), population index r N_OBJ onward, and its 1/ws share of the
    1024 x 1024 rule's outer nodes. Each sweep: the shard pass (streaming kernel), an all-reduce
    of the 16 exchange words (NCCL, int64 sum, on the sampler's stream; none at one rank), the
    decision kernel. FP64. W untimed sweeps, then K timed, CUDA events on the sampler's stream,
    max over ranks; the value is the population's member updates per second (weak scaling: the
    members per rank stay fixed)."""
    import torch
    import torch.distributed as dist
    from paper_2105_08026_gb300 import synth
    _, theta0, scale, consts = workload(0)
    data = synth.lf_data(N_OBJ, seed=replica_seeds(rank)[0])
    n_pop = N_OBJ * ws
    st = torch.cuda.Stream(device=local)
    s = cudahm.Sampler(cudahm.LF, N_OBJ, theta_init=theta0, theta_prop_scale=scale, model_consts=consts,
                       seed=CHAIN_SEED, device=local, stream=st.cuda_stream, use_torch_allocator=True)
    with torch.cuda.stream(st):
        y_dev = torch.from_numpy(data.fhat).cuda()
        r_dev = torch.from_numpy(data.r).cuda()
        cudahm.cudahm_set_data_device(s.h, y_dev.data_ptr(), r_dev.data_ptr(), N_OBJ)
        s.shard(rank * N_OBJ, n_pop, rank, ws)
        words = torch.zeros(cudahm.SHARD_WORDS, dtype=torch.int64, device=f"cuda:{local}")
        exchange = (lambda w: dist.all_reduce(w, op=dist.ReduceOp.SUM)) if ws > 1 else (lambda w: None)
        if args.warmup > 0:
            s.run_sharded(0, args.warmup, 1, words, exchange)
        torch.cuda.synchronize()
        if ws > 1:
            dist.barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        K = args.steps
        e0.record(st)
        rows = s.run_sharded(0, K, 1, words, exchange)
        e1.record(st)
        e1.synchronize()
        ms = e0.elapsed_time(e1)
    assert rows.shape[0] == K
    t = max_over_ranks(ms)
    s.close()
    return {"value": n_pop * K / (t * 1e-3), "unit": "object-updates/s", "ms_per_step": t / K,
            "population": n_pop, "shards": ws, "members_per_shard": N_OBJ, "scaling": "weak", "dtype": "f64",
            "exchange": ("NCCL all-reduce of 16 int64 words per sweep" if ws > 1 else "none (one shard)"),
            "launches_per_sweep": 2,
            "note": "one chain over the whole population; bit-identical to one handle holding it"}


def run_mvn3(args, cudahm, stream, device, flush, peak_fp64):
    """d = 3 normal population: N = 1e6, mu = (0, 1, -1), C_pop = Q diag(1, sqrt 20, 20) Q^T,
    s_ij ~ U[0.3, 1]; one run of --mvn3-sweeps sweeps (a third burn-in), inputs resident in HBM,
    L2 flushed before it, device time by CUDA events on the sampler's stream. FP32 bulk form
    and plain FP64, each from the same start."""
    import torch
    from paper_2105_08026_gb300 import synth
    data = synth.mvn3_data(1_000_000, seed=1003)
    theta0, scale, _ = synth.mvn3_settings(data)
    n = data.y.shape[0]
    y_dev = torch.from_numpy(np.ascontiguousarray(data.y)).cuda()
    s_dev = torch.from_numpy(np.ascontiguousarray(data.s)).cuda()
    K = args.mvn3_sweeps
    out = {}
    for name, prec in (("fp32", cudahm.FP32), ("fp64", cudahm.FP64)):
        sm = cudahm.Sampler(cudahm.MVN3, n, theta_init=theta0, theta_prop_scale=scale, seed=3, precision=prec,
                            device=device, stream=stream.cuda_stream, use_torch_allocator=True)
        cudahm.cudahm_set_data_device(sm.h, y_dev.data_ptr(), s_dev.data_ptr(), n)
        if args.warmup > 0:
            sm.run(min(args.warmup, 100), 0)
        flush.zero_()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        rows = sm.run(K // 3, K - K // 3, 1)
        e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        assert rows.shape == (K - K // 3, 9)
        st = sm.stats()
        out[name] = {"value": n * K / (ms * 1e-3), "unit": "object-updates/s", "ms_per_step": ms / K,
                     "member_accept": st.member_accepts / (n * (K + min(args.warmup, 100)))}
        if prec == cudahm.FP32 and peak_fp64:
            ach = MVN3_F32_FP64_FLOP_PER_UPDATE * n * K / (ms * 1e-3)
            out[name]["roofline"] = {"bound": "alu", "unit": "TFLOP/s", "achieved": ach / 1e12,
                                     "peak": peak_fp64 / 1e12, "frac": ach / peak_fp64,
                                     "peak_source": "FP64 DFMA stream measured live on this GPU (x2 flops)",
                                     "hbm_GBps": MVN3_F32_DRAM_BYTES_PER_UPDATE * n * K / (ms * 1e-3) / 1e9,
                                     "kernel": "batch_kernel<FP32> (MVN3 member step)"}
        sm.close()
    out.update({"n": n, "d": 3, "steps": K, "workload": "MVN3 d=3 normal population, N=1e6, cond(C_pop)=20",
                "dtype": {"fp32": "f32 member terms, f64 v = S U, RAM factor, sums, theta step", "fp64": "f64"},
                "l2": "256 MB flush before the run; state and data (~170 MB) exceed L2"})
    return out


def run_bb1(args, cudahm, stream, device, flush, peak_fp64):
    """The paper's own simulation model (BB1 luminosity function, flux-dependent measurement error,
    detection at nu = 5 times the error; Sec. 5.1-5.2) at its case-study size, N = 1e5 detected
    objects, FP64, 1024 x 1024 selection rule with sigma(F) inside Phi; one run of --bb1-sweeps
    sweeps, inputs resident in HBM, L2 flushed before it, CUDA events on the sampler's stream."""
    import torch
    from paper_2105_08026_gb300 import synth
    data = synth.bb1_data(100_000, seed=1004)
    theta0, scale, consts = synth.bb1_settings(data)
    n = data.fhat.size
    s = cudahm.Sampler(cudahm.BB1, n, theta_init=theta0, theta_prop_scale=scale, model_consts=consts, seed=5,
                       device=device, stream=stream.cuda_stream, use_torch_allocator=True)
    y_dev = torch.from_numpy(data.fhat).cuda()
    r_dev = torch.from_numpy(data.r).cuda()
    cudahm.cudahm_set_data_device(s.h, y_dev.data_ptr(), r_dev.data_ptr(), n)
    if args.warmup > 0:
        s.run(min(args.warmup, 200), 0)
    K = args.bb1_sweeps
    flush.zero_()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    rows = s.run(0, K, 1)
    e1.record(stream)
    e1.synchronize()
    ms = e0.elapsed_time(e1)
    st = s.stats()
    s.close()
    # the same data in the marginal form (latents integrated out by cubature, FP64)
    m = cudahm.Sampler(cudahm.BB1, n, theta_init=theta0, theta_prop_scale=scale, model_consts=consts, seed=5,
                       device=device, stream=stream.cuda_stream, use_torch_allocator=True, marginal=True)
    cudahm.cudahm_set_data_device(m.h, y_dev.data_ptr(), r_dev.data_ptr(), n)
    m.run(20, 0)
    Km = 100
    torch.cuda.synchronize()
    e0.record(stream)
    m.run(0, Km, 1)
    e1.record(stream)
    e1.synchronize()
    mms = e0.elapsed_time(e1)
    m.close()
    marg = {"ms_per_step": mms / Km, "member_integrals_per_s": n * Km / (mms * 1e-3), "steps": Km, "dtype": "f64"}
    # the paper's headline size (3e5 objects; its K40c took about an hour, run length not printed),
    # timed on the N = 1e5 catalog repeated three times (drawing a new 3e5 catalog takes minutes on
    # the host: about 2,600 simulated objects per detection; a member's work does not depend on
    # which other members repeat), 500 timed sweeps after 100 untimed
    b3 = cudahm.Sampler(cudahm.BB1, 300_000, theta_init=theta0, theta_prop_scale=scale, model_consts=consts, seed=6,
                        device=device, stream=stream.cuda_stream, use_torch_allocator=True)
    y3 = torch.from_numpy(np.tile(data.fhat, 3)).cuda()
    r3 = torch.from_numpy(np.tile(data.r, 3)).cuda()
    cudahm.cudahm_set_data_device(b3.h, y3.data_ptr(), r3.data_ptr(), 300_000)
    b3.run(100, 0)
    flush.zero_()
    torch.cuda.synchronize()
    e0.record(stream)
    b3.run(0, 500, 1)
    e1.record(stream)
    e1.synchronize()
    ms3 = e0.elapsed_time(e1)
    b3.close()
    big = {"n": 300_000, "value": 300_000 * 500 / (ms3 * 1e-3), "unit": "object-updates/s", "ms_per_step": ms3 / 500,
           "steps": 500, "seconds_per_1e6_sweeps": ms3 / 500 * 1e3, "data": "the N=1e5 catalog x 3"}
    return {"value": n * K / (ms * 1e-3), "unit": "object-updates/s", "ms_per_step": ms / K, "n": n, "steps": K,
            "marginal": marg, "n300000": big,
            "theta_mean": rows.mean(axis=0).tolist(), "theta_true": theta0.tolist(),
            "launch_shape": [st.grid_blocks, st.block_threads, st.objects_per_thread],
            "workload": "BB1 luminosity function (paper Sec. 5), N=1e5, FP64, 1024x1024 rule with sigma(F)",
            "dtype": "f64"}


def run_nn3_ess(args, cudahm, stream, device):
    """The paper's normal-normal benchmark (Sec. 3: d = 3, mu_pop, C_pop = D R D and sigma_j as
    printed, C_pop and sigma_j known, flat prior on mu) measured as the paper measures it: the
    post-burn-in time to an effective sample size of 1000 for the slowest of the three mu
    components. Per population size: --nn3-burn untimed sweeps, then --nn3-sweeps timed ones
    (the paper's 4e4 burn-in and 7.5e4 kept sweeps), CUDA events on the sampler's stream, ESS of
    the kept theta rows by the library's estimator. FP64, and FP32 at N = 1e4. Then the same
    with --nn3-chains independent chains on the same data in one batched run (the paper's Stan
    protocol pools parallel chains; ESS of the pooled draws = the sum of the chains' ESS), for
    N <= --nn3-chains-max-n, each chain --nn3-chain-sweeps timed sweeps after the same burn-in."""
    import torch
    from paper_2105_08026_gb300 import synth
    out = []
    sizes = [int(float(v)) for v in args.nn3_sizes.split(",") if v]
    for n in sizes:
        data = synth.nn3_data(n, seed=1004)
        theta0, scale, consts = synth.nn3_settings(data)
        precs = [("f64", cudahm.FP64)] + ([("f32", cudahm.FP32)] if n == 10_000 else [])
        for name, prec in precs:
            s = cudahm.Sampler(cudahm.NN3, n, theta_init=theta0, theta_prop_scale=scale, model_consts=consts,
                               seed=7, precision=prec, device=device, stream=stream.cuda_stream,
                               use_torch_allocator=True)
            s.set_data(data.y, data.s)
            s.run(args.nn3_burn, 0)
            K = args.nn3_sweeps
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            rows = s.run(0, K, 1)
            e1.record(stream)
            e1.synchronize()
            ms = e0.elapsed_time(e1)
            ess = cudahm.cudahm_ess(rows)
            st = s.stats()
            s.close()
            out.append({"n": n, "dtype": name, "sweeps": K, "burn_in": args.nn3_burn, "ms": ms,
                        "us_per_sweep": 1e3 * ms / K, "ess": ess.tolist(),
                        "time_to_ess1000_s": 1e-3 * ms * 1000.0 / float(ess.min()),
                        "object_updates_per_s": n * K / (ms * 1e-3),
                        "theta_accept": st.theta_accepts / st.sweeps,
                        "member_accept": st.member_accepts / (st.sweeps * n),
                        "launch_shape": [st.grid_blocks, st.block_threads, st.objects_per_thread]})
        R = args.nn3_chains
        if R > 1 and n <= args.nn3_chains_max_n:
            chains = []
            for r in range(R):
                c = cudahm.Sampler(cudahm.NN3, n, theta_init=theta0, theta_prop_scale=scale, model_consts=consts,
                                   seed=1000 + r, device=device, stream=stream.cuda_stream, use_torch_allocator=True)
                c.set_data(data.y, data.s)
                chains.append(c)
            _, tune = cudahm.batch_run(chains, args.nn3_burn, 0)
            K = args.nn3_chain_sweeps
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            rows, _ = cudahm.batch_run(chains, 0, K, 1, tune=tune)
            e1.record(stream)
            e1.synchronize()
            ms = e0.elapsed_time(e1)
            ess = np.sum([cudahm.cudahm_ess(r_) for r_ in rows], axis=0)
            for c in chains:
                c.close()
            out.append({"n": n, "dtype": "f64", "chains": R, "sweeps": K, "burn_in": args.nn3_burn, "ms": ms,
                        "us_per_sweep": 1e3 * ms / K, "ess": ess.tolist(),
                        "time_to_ess1000_s": 1e-3 * ms * 1000.0 / float(ess.min()),
                        "object_updates_per_s": R * n * K / (ms * 1e-3),
                        "launch": {"block_threads": tune.block_threads, "sweeps_per_launch": tune.sweeps_per_launch,
                                   "graph": bool(tune.use_graph), "blocks": tune.grid_blocks}})
    return {"workload": "normal-normal benchmark (paper Sec. 3), d=3, C_pop known, theta=mu",
            "metric": "post-burn-in seconds to ESS=1000 (min over mu components)", "runs": out}


def run_marginal(args, cudahm, stream, device, data, theta0, scale, consts, peak_fp64):
    """The marginal form on the LF workload (N = 3e5, 1024 x 1024 rule): every member's latent
    integrated out by the cubature rule (96 nodes per member) and a theta-only chain, in FP64 and
    in the FP32 bulk form (binary32 node terms). --marginal-burn untimed steps, then
    --marginal-steps timed (CUDA events on the sampler's stream); reports theta steps/s, member
    integrals/s and the theta ESS per second."""
    import torch
    n = data.fhat.size
    y_dev = torch.from_numpy(data.fhat).cuda()
    r_dev = torch.from_numpy(data.r).cuda()
    out = {"workload": "LF N=3e5, latents integrated out by cubature (64 + 32 Gauss-Legendre nodes per member), "
                       "theta-only chain, 1024x1024 selection rule"}
    for name, prec in (("f64", cudahm.FP64), ("f32", cudahm.FP32)):
        s = cudahm.Sampler(cudahm.LF, n, theta_init=theta0, theta_prop_scale=scale, model_consts=consts, seed=11,
                           precision=prec, device=device, stream=stream.cuda_stream, use_torch_allocator=True,
                           marginal=True)
        cudahm.cudahm_set_data_device(s.h, y_dev.data_ptr(), r_dev.data_ptr(), n)
        s.run(args.marginal_burn, 0)
        K = args.marginal_steps * (1 if prec == cudahm.FP64 else 10)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        rows = s.run(0, K, 1)
        e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        ess = cudahm.cudahm_ess(rows)
        st = s.stats()
        s.close()
        r = {"steps": K, "burn_in": args.marginal_burn, "ms_per_step": ms / K, "steps_per_s": K / (ms * 1e-3),
             "member_integrals_per_s": n * K / (ms * 1e-3), "theta_accept": st.theta_accepts / st.sweeps,
             "ess": ess.tolist(), "ess_per_s_min": float(ess.min()) / (ms * 1e-3),
             "launch_shape": [st.grid_blocks, st.block_threads],
             "dtype": "f64" if prec == cudahm.FP64 else "f32 node terms, f64 window/reference/sums/theta step"}
        if prec == cudahm.FP64 and MARG_FP64_FLOP_PER_MEMBER is not None and peak_fp64:
            ach = MARG_FP64_FLOP_PER_MEMBER * n * K / (ms * 1e-3)
            r["roofline"] = {"bound": "alu", "unit": "TFLOP/s", "achieved": ach / 1e12, "peak": peak_fp64 / 1e12,
                             "frac": ach / peak_fp64, "kernel": "marg_kernel<LF>",
                             "peak_source": "FP64 DFMA stream measured live on this GPU (x2 flops)"}
        out[name] = r
    return out


def run_nn1_small(args, cudahm, stream, device):
    """The d = 1 normal-normal configuration (N = 1000, mu = 2, tau = 0.8, sigma_i ~ U[0.5, 1.5],
    data seed 1001, chain seed 1, FP64): 500 burn-in sweeps untimed, 2000 timed. At this N a
    sweep is latency-bound (one member per thread, the theta step and the grid barrier)."""
    import torch
    from paper_2105_08026_gb300 import synth
    d = synth.nn1_data(1000, seed=1001)
    th, sc, c = synth.nn1_settings(d)
    s = cudahm.Sampler(cudahm.NN1, 1000, theta_init=th, theta_prop_scale=sc, model_consts=c, seed=1,
                       device=device, stream=stream.cuda_stream, use_torch_allocator=True)
    s.set_data(d.y, d.sigma)
    s.run(500, 0)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    rows = s.run(0, 2000, 1)
    e1.record(stream)
    e1.synchronize()
    ms = e0.elapsed_time(e1)
    st = s.stats()
    s.close()
    return {"workload": "normal-normal d=1, N=1000, FP64", "value": 1000 * 2000 / (ms * 1e-3),
            "unit": "object-updates/s", "us_per_sweep": 1e3 * ms / 2000, "steps": 2000, "burn_in": 500,
            "theta_mean": rows.mean(axis=0).tolist(),
            "launch_shape": [st.grid_blocks, st.block_threads, st.objects_per_thread]}


def _serve_pool(args):
    """Pre-generated request catalogs: NN1 or LF alternately, N log-uniform on [1e3, 3e5], the
    single-population workloads' parameters scaled by U[0.8, 1.2]."""
    from paper_2105_08026_gb300 import synth
    g = np.random.default_rng(3000)
    pool = []
    for q in range(args.serve_pool):
        n = int(round(math.exp(g.uniform(math.log(1e3), math.log(3e5)))))
        kind = "nn1" if q % 2 == 0 else "lf"
        f = g.uniform(0.8, 1.2, 5)
        if kind == "nn1":
            sp = synth.PopSpec("nn1", n, 3100 + q, dict(mu=2.0 * f[0], tau=0.8 * f[1]))
        else:
            sp = synth.PopSpec("lf", n, 3100 + q, dict(beta=-1.2 * f[0], L_star=1e10 * f[1], L_low=1e8 * f[2],
                                                       r_max=4000.0 * f[3], detect_frac=0.30 * f[4]))
        y, aux, th, sc, c = synth.pop_data(sp)
        pool.append((sp, y, aux, th, sc, c))
    return pool


def _pct(lat):
    lat = np.asarray(lat, dtype=np.float64)
    return {"p50": float(np.percentile(lat, 50)), "p95": float(np.percentile(lat, 95)),
            "p99": float(np.percentile(lat, 99)), "max": float(lat.max())}


def _serve_stream(cudahm, device, pool, arrivals, sweeps):
    """Feeds (arrival s, pool index, seed) requests to a fresh continuous-batching server at their
    arrival times (all at once when every arrival time is 0); returns latencies, work, wall time,
    the server's stats and the largest number of requests seen on the device together."""
    import threading as th_
    sv = cudahm.Server(60 << 30, device=device, precision=cudahm.FP32, max_active=512, sweeps_per_step=250)
    tickets = []
    peak = [0]
    done = [False]

    def producer():
        t0 = time.perf_counter()
        for (ta, pi, seed) in arrivals:
            dt = ta - (time.perf_counter() - t0)
            if dt > 0:
                time.sleep(dt)
            sp, y, aux, th, sc, c = pool[pi]
            cfg = cudahm.make_config(cudahm.NN1 if sp.kind == "nn1" else cudahm.LF, sp.n, theta_init=th,
                                     theta_prop_scale=sc, model_consts=c, seed=seed, precision=cudahm.FP32,
                                     device=device)
            tickets.append((sv.submit(cfg, y, aux, 0, sweeps, sweeps), sp.n))

    def sampler():  # how many requests share the device
        while not done[0]:
            peak[0] = max(peak[0], sv.stats()["active"])
            time.sleep(0.005)
    t_start = time.perf_counter()
    mon = th_.Thread(target=sampler)
    mon.start()
    prod = th_.Thread(target=producer)
    prod.start()
    prod.join()
    lat = []
    work = 0.0
    for tk, n in tickets:
        sv.wait(tk, -1)
        rows, ms = sv.result(tk)
        lat.append(ms)
        work += n * sweeps
    wall = time.perf_counter() - t_start
    done[0] = True
    mon.join()
    st = sv.stats()
    sv.close()
    return lat, work, wall, st, peak[0]


def run_served(args, cudahm, device):
    """Config 4: a Poisson request stream (rate --serve-rate for --serve-seconds) into the
    continuous-batching server: each request is NN1 or LF with probability 1/2, N log-uniform on
    [1e3, 3e5], 5000 sweeps, FP32, 60 GB budget; request data come from a pre-generated pool of
    catalogs (each request has its own chain seed). Reports completion-latency percentiles and
    aggregate throughput. Beside it:
    - saturated: --serve-burst requests of the same mix all arriving at once, so the server's own
      capacity (not the offered load) sets the throughput;
    - sequential_fp64: the plain FP64 sampler serving the same stream one request at a time in
      arrival order (the first --serve-seq requests; each request's service time measured on the
      GPU, the first-come-first-served queue then gives each completion time)."""
    pool = _serve_pool(args)
    sweeps = args.serve_sweeps
    g = np.random.default_rng(3001)
    arrivals = []
    t = 0.0
    while True:
        t += g.exponential(1.0 / args.serve_rate)
        if t > args.serve_seconds:
            break
        arrivals.append((t, int(g.integers(0, len(pool))), int(g.integers(1, 2**31))))
    lat, work, wall, st, peak = _serve_stream(cudahm, device, pool, arrivals, sweeps)
    offered = args.serve_rate * float(np.mean([pool[pi][0].n for _, pi, _ in arrivals])) * sweeps
    out = {"value": work / wall, "unit": "object-updates/s", "requests": len(lat),
           "arrival_rate_per_s": args.serve_rate, "window_s": args.serve_seconds, "sweeps_per_request": sweeps,
           "latency_ms": _pct(lat), "offered_object_updates_per_s": offered, "wall_s": wall,
           "device_busy_s": st["busy_ms"] / 1e3, "peak_requests_on_device": peak,
           "dtype": "f32 member terms, f64 sums/accept/RAM/selection integral", "budget_bytes": 60 << 30}
    if args.serve_burst > 0:
        burst = [(0.0, pi, seed) for (_, pi, seed) in arrivals[: args.serve_burst]]
        blat, bwork, bwall, bst, bpeak = _serve_stream(cudahm, device, pool, burst, sweeps)
        out["saturated"] = {"value": bwork / bwall, "unit": "object-updates/s", "requests": len(blat),
                            "latency_ms": _pct(blat), "wall_s": bwall, "peak_requests_on_device": bpeak,
                            "note": "every request arrives at t = 0: the throughput is the server's capacity"}
    if args.serve_seq > 0:
        seq = arrivals[: args.serve_seq]
        service = []
        swork = 0.0
        for (ta, pi, seed) in seq:
            sp, y, aux, th, sc, c = pool[pi]
            t0 = time.perf_counter()
            sm = cudahm.Sampler(cudahm.NN1 if sp.kind == "nn1" else cudahm.LF, sp.n, theta_init=th,
                                theta_prop_scale=sc, model_consts=c, seed=seed, precision=cudahm.FP64, device=device)
            sm.set_data(y, aux)
            rows = sm.run(0, sweeps, sweeps)
            sm.close()
            service.append(time.perf_counter() - t0)
            assert rows.shape[0] == 1
            swork += sp.n * sweeps
        end = 0.0
        slat = []
        for (ta, _, _), sv_s in zip(seq, service):
            end = max(end, ta) + sv_s
            slat.append((end - ta) * 1e3)
        out["sequential_fp64"] = {"value": swork / sum(service), "unit": "object-updates/s", "requests": len(seq),
                                  "latency_ms": _pct(slat), "busy_s": sum(service),
                                  "note": "plain FP64 sampler, one request at a time in arrival order (handle "
                                          "creation, data upload, run and result read per request); latency from "
                                          "the first-come-first-served queue of the measured service times"}
        # the server on the same prefix of the stream, for a like-for-like comparison
        plat, pwork, pwall, _, ppeak = _serve_stream(cudahm, device, pool, seq, sweeps)
        out["served_same_prefix"] = {"value": pwork / pwall, "unit": "object-updates/s", "requests": len(plat),
                                     "latency_ms": _pct(plat), "peak_requests_on_device": ppeak}
    return out


def run_cuda(args):
    import torch
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    from paper_2105_08026_gb300 import cudahm

    data, theta0, scale, consts = workload(rank)
    n = data.fhat.size
    stream = torch.cuda.current_stream()
    chain_seed = replica_seeds(rank)[1]
    s = cudahm.Sampler(cudahm.LF, n, theta_init=theta0, theta_prop_scale=scale, model_consts=consts,
                       seed=chain_seed, device=local, stream=stream.cuda_stream, use_torch_allocator=True)
    # inputs resident in HBM before timing (device-to-device set_data from torch tensors)
    y_dev = torch.from_numpy(data.fhat).cuda()
    r_dev = torch.from_numpy(data.r).cuda()
    cudahm.cudahm_set_data_device(s.h, y_dev.data_ptr(), r_dev.data_ptr(), n)
    torch.cuda.synchronize()
    # the clock sampler runs from before the warm-up, so that its start-up is over when timing starts
    clocks = ClockSampler(local)
    clocks.start()
    clocks.wait_first()
    # warm-up: W untimed sweeps through the same call as the timed steps (run, rows read back)
    if args.warmup > 0:
        s.run(0, args.warmup, 1)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    K = args.steps
    # timed run calls of up to one persistent launch each (4096 sweeps), the L2 flushed before each
    L = max(1, args.launch_sweeps)
    chunks = [min(L, K - j) for j in range(0, K, L)]
    R = len(chunks)
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    t_timed0 = time.perf_counter()
    total_ms = 0.0
    host_ms = 0.0
    launches = 0
    rows_total = 0
    kept = []
    for ns in chunks:
        flush.zero_()  # write 256 MB > L2 between timed launches
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        rows = s.run(0, ns, 1)
        e1.record(stream)
        e1.synchronize()
        # the step's device time: the library's events on the stream, from before its first kernel
        # to after the kept rows' copy to the host (the torch events also hold the host's enqueue
        # and return latency, when the device is idle: reported beside it)
        total_ms += s.stats().last_run_ms
        host_ms += e0.elapsed_time(e1)
        nl = math.ceil(ns / 4096)
        launches += 2 * nl  # per chunk of <= 4096 sweeps: theta-table kernel + persistent sweep kernel
        rows_total += rows.shape[0]
        kept.append(rows)
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    clk = clocks.stop(t_timed0, time.perf_counter())
    assert rows_total == K
    t_max_ms = max_over_ranks(total_ms)
    value = replica_value(ws, n * K, t_max_ms)

    # the same workload in the FP32 bulk form (binary32 member terms, binary64 sums/accept/RAM/etabar)
    fp32 = None
    if not args.no_fp32:
        s3 = cudahm.Sampler(cudahm.LF, n, theta_init=theta0, theta_prop_scale=scale, model_consts=consts,
                            seed=chain_seed, device=local, stream=stream.cuda_stream,
                            use_torch_allocator=True, precision=cudahm.FP32)
        cudahm.cudahm_set_data_device(s3.h, y_dev.data_ptr(), r_dev.data_ptr(), n)
        if args.warmup > 0:
            s3.run(0, args.warmup, 1)
        f_ms = 0.0
        for ns in chunks:
            flush.zero_()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            s3.run(0, ns, 1)
            e1.record(stream)
            e1.synchronize()
            f_ms += s3.stats().last_run_ms  # device time, as the headline's
        f_ms = max_over_ranks(f_ms)
        # and one longer run, where the launch's fixed start-up cost (~0.1 ms: tables, the first
        # proposal, the first half-step) no longer weighs on the per-sweep figure
        L_long = 400
        flush.zero_()
        torch.cuda.synchronize()
        s3.run(0, L_long, 1)
        l_ms = max_over_ranks(s3.stats().last_run_ms)
        fp32 = {"value": replica_value(ws, n * K, f_ms), "unit": "object-updates/s", "ms_per_step": f_ms / K,
                "steady": {"sweeps": L_long, "value": replica_value(ws, n * L_long, l_ms),
                           "ms_per_step": l_ms / L_long},
                "dtype": "f32 member terms, f64 sums/accept/RAM/selection integral"}
        s3.close()

    # the same FP64 workload keeping every member's running mean and variance of chi over the kept
    # sweeps (thin 1: every sweep adds its latents; one read and one write of 16 B per member)
    moments = None
    if not args.no_moments and rank == 0:
        s4 = cudahm.Sampler(cudahm.LF, n, theta_init=theta0, theta_prop_scale=scale, model_consts=consts,
                            seed=chain_seed, device=local, stream=stream.cuda_stream,
                            use_torch_allocator=True, keep_chi_moments=True)
        cudahm.cudahm_set_data_device(s4.h, y_dev.data_ptr(), r_dev.data_ptr(), n)
        if args.warmup > 0:
            s4.run(args.warmup, 0)  # burn-in: its sweeps are not kept in the moments
        m_ms = 0.0
        for ns in chunks:
            flush.zero_()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            s4.run(0, ns, 1)
            e1.record(stream)
            e1.synchronize()
            m_ms += e0.elapsed_time(e1)
        mean, var, cnt = s4.chi_moments()
        assert cnt == K
        moments = {"value": n * K / (m_ms * 1e-3), "unit": "object-updates/s", "ms_per_step": m_ms / K,
                   "kept_sweeps": int(cnt), "relative_to_plain": (n * K / (m_ms * 1e-3)) / value,
                   "dtype": "f64", "median_posterior_sd_chi": float(np.median(np.sqrt(var)))}
        s4.close()

    # one population split over the ranks (all ranks: an all-reduce per sweep)
    shard = None
    if not args.no_shard:
        shard = run_shard(args, cudahm, rank, ws, local)

    # batched FP32 form: 256 NN1/LF populations of uneven size in one persistent launch per chunk
    batched = None
    if not args.no_batched and rank == 0:
        batched = run_batched(args, cudahm, stream, local)

    served = None
    if not args.no_serve and rank == 0:
        served = run_served(args, cudahm, local)

    peak = fp64_peak(local) if rank == 0 else None
    mvn3 = None
    if not args.no_mvn3 and rank == 0:
        mvn3 = run_mvn3(args, cudahm, stream, local, flush, peak)

    bb1 = None
    if not args.no_bb1 and rank == 0:
        bb1 = run_bb1(args, cudahm, stream, local, flush, peak)
    nn3 = None
    if not args.no_nn3 and rank == 0:
        nn3 = run_nn3_ess(args, cudahm, stream, local)
    nn1 = None
    if not args.no_nn1 and rank == 0:
        nn1 = run_nn1_small(args, cudahm, stream, local)
    marg = None
    if not args.no_marginal and rank == 0:
        marg = run_marginal(args, cudahm, stream, local, data, theta0, scale, consts, peak)
        all_rows = np.concatenate(kept, axis=0)
        ess = cudahm.cudahm_ess(all_rows)
        marg["member_form_same_workload"] = {"ess": ess.tolist(), "sweeps": int(all_rows.shape[0]),
                                             "ess_per_s_min": float(ess.min()) / (total_ms * 1e-3)}

    # e2e through the public API with host buffers (every iteration: H2D data, run, D2H samples)
    e2e = None
    if not args.no_e2e:
        s2 = cudahm.Sampler(cudahm.LF, n, theta_init=theta0, theta_prop_scale=scale, model_consts=consts,
                            seed=chain_seed, device=local, stream=stream.cuda_stream,
                            use_torch_allocator=True)
        host_y = np.ascontiguousarray(data.fhat)
        host_r = np.ascontiguousarray(data.r)
        s2.set_data(host_y, host_r)
        s2.run(0, max(1, min(args.warmup, 200)), 1)  # untimed: the same call path as the timed steps
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for ns in chunks:  # the same run calls as the device-timed leg
            s2.set_data(host_y, host_r)          # host -> device copy of the inputs
            out = s2.run(0, ns, 1)               # device -> host copy of the theta rows
            assert out.shape == (ns, 3)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        e2e_val = replica_value(ws, n * K, max_over_ranks(wall * 1e3))
        e2e = {"value": e2e_val, "unit": "object-updates/s", "h2d_bytes_per_step": 2 * n * 8 * R / K,
               "d2h_bytes_per_step": 3 * 8 + 4 * R / K}
        s2.close()

    if rank != 0:
        s.close()
        if ws > 1:
            torch.distributed.destroy_process_group()
        return 0

    st = s.stats()
    sweep_launch_ms = total_ms / max(1, launches // 2)  # (with the table kernel and the rows' copy)
    sweeps_per_launch = K / max(1, launches // 2)
    roofline = {"bound": "alu", "unit": "TFLOP/s", "peak": peak / 1e12 if peak else None,
                "peak_source": "FP64 DFMA stream measured live on this GPU (x2 flops)",
                "achieved": None, "frac": None, "traffic": DRAM_BYTES_PER_LAUNCH,
                "kernel": "sweep_kernel<LF,4>", "launch_ms": sweep_launch_ms}
    if FP64_FLOP_PER_SWEEP is not None and peak:
        ach = FP64_FLOP_PER_SWEEP * sweeps_per_launch / (sweep_launch_ms * 1e-3)
        roofline.update(achieved=ach / 1e12, frac=ach / peak)
    cpu = None
    if not args.no_cpu:
        sweeps = max(1, args.cpu_sweeps)
        rate, dt = oracle_rate(data, theta0, scale, consts, sweeps)
        cpu = {"value": rate, "unit": "object-updates/s", "cores": 1, "kind": "oracle",
               "sample": f"{sweeps} full sweeps of the same N={n} workload ({dt:.1f} s, single-threaded)"}
        ncore = host_cores()
        rate_all, dt_all = oracle_rate_allcores(data, theta0, scale, consts, sweeps, ncore)
        cpu["all_cores"] = {"value": rate_all, "unit": "object-updates/s", "cores": ncore, "kind": "oracle",
                            "sample": f"{sweeps} full sweeps of the same workload ({dt_all:.1f} s): members split "
                                      f"over {ncore} threads, the theta step and its selection rule serial"}
    line = {"metric": "object-updates/s", "value": value, "unit": "object-updates/s", "n_gpus": ws, "steps": K,
            "warmup": args.warmup, "ms_per_step": t_max_ms / K, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "LF thinned luminosity function, N=3e5, FP64, 1024x1024 selection rule",
                       "n": n, "parallelism": f"replicas x{ws}", "l2": "256 MB flush before each timed launch; "
                       "member state register-resident within a launch", "timed_launches": R,
                       "timing": "device time per run call: the library's CUDA events on the stream, before the "
                                 "theta-table kernel to after the kept rows' copy to the host",
                       "host_inclusive_ms_per_step": host_ms / K,
                       "launch_shape": [st.grid_blocks, st.block_threads, st.objects_per_thread]},
            "e2e": e2e, "gpu_launches": launches, "roofline": roofline, "cpu_baseline": cpu, "clocks": clk,
            "fp32_bulk": fp32, "batched_fp32": batched, "served_fp32": served, "mvn3": mvn3, "bb1": bb1, "nn3_ess": nn3,
            "marginal": marg, "nn1_n1000": nn1, "chi_moments": moments, "shard": shard}
    print(json.dumps(line), flush=True)
    s.close()
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    return run_cuda(args)


if __name__ == "__main__":
    sys.exit(main())
