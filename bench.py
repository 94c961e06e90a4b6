"""Benchmark of the FK-convolution fit step on B300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--prec P] [--impl ours|reference]

A fit step is one pass of the whole hot path over the global-shaped fit set
(40 synthetic datasets, 12 DIS + 28 hadronic, ~4500 data points, R = 100
replicas on a shared 50-point x grid): forward convolution of every table,
chi^2 with its gradient, adjoint of every table into dchi2/dF.  In the
non-FP64 modes the tables and data are whitened once at set-up (each
covariance block's inverse Cholesky factor folded in, --whiten), so the
step's chi^2 needs no triangular solve; the FP64 modes (and --whiten off)
run the FP64 substitutions in the step.  A bench
step is --inner (default 10) consecutive fit steps, so that the timed region
of the driver's step count lasts a quarter of a second or more.  The metric
is datapoint*replicas per second (sum of ndata * R over the fit steps,
divided by their time).  Tables are device resident; the timed region
replays the step's CUDA graphs.  Under torchrun each rank runs its own copy
of the workload (weak scaling, no collective on the data path); rank 0
prints one JSON line.

With one GPU the line also carries: `accuracy` (the fit step's chi^2 and
gradient against the FP64 oracle, from the CPU-baseline leg's own run),
`kernels` (kernel-level lines with their own rooflines: stress table R = 1
streaming and R = 1000 tensor cores, configs 0-2, Table 3's R = 1 rows, the
FP64 chi^2 substitutions alone) and
`serve` (a bounded run of the served mixed workload: 2000 Poisson arrivals
at 2000/s, p50/p99/max latency, saturation and per-request throughput).
"""
import argparse
import faulthandler
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, HERE)

METRIC = "FK conv datapoint·replicas/s"
UNIT = "datapoint·replicas/s"
REPLICAS = 100
SEED = 10547 + 3


_T0 = time.perf_counter()


def stage(msg):
    """Progress on stderr (the JSON line alone goes to stdout)."""
    print(f"[bench {time.perf_counter() - _T0:7.1f} s] {msg}", file=sys.stderr, flush=True)


def save_arg(args):
    """GlobalFit's save_products for --save."""
    return {"auto": "auto", "on": True, "off": False}[getattr(args, "save", "auto")]


def whiten_arg(args):
    """GlobalFit's whiten for --whiten."""
    return {"auto": None, "on": True, "off": False}[getattr(args, "whiten", "auto")]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--prec", default="bf16x3", choices=["fp64", "fp32", "bf16", "bf16x3", "tf32", "fp64tc"])
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--save", choices=("auto", "on", "off"), default="auto",
                    help="fit case: keep the forward's tensor-core products for the adjoint (GlobalFit's "
                         "save_products: auto = where the table's ratio of table to product bytes pays)")
    ap.add_argument("--whiten", choices=("auto", "on", "off"), default="auto",
                    help="fit case: fold each covariance block's inverse factor into its table at set-up "
                         "(GlobalFit's whiten: auto = every mode but the FP64 ones)")
    ap.add_argument("--watchdog-s", type=float, default=900.0,
                    help="print every thread's stack to stderr and exit if the run has not finished after this "
                         "many seconds (the default run takes a few minutes); 0 disables")
    ap.add_argument("--inner", type=int, default=10,
                    help="fit case: fit steps per bench step (the timed region is steps x inner fit steps)")
    ap.add_argument("--no-extras", action="store_true",
                    help="fit case: skip the kernel-level lines and the served-mix block")
    ap.add_argument("--phases", action="store_true",
                    help="fit case: run the step as three separate phases (per-phase timing) "
                         "instead of the pipelined per-table chains")
    ap.add_argument("--waves", type=int, default=1, help="fit case: forward waves of the pipelined step")
    ap.add_argument("--streams", type=int, default=0,
                    help="fit case: streams the tables are spread over (0: one per table)")
    ap.add_argument("--case", default="fit", choices=["fit", "stress", "serve", "descent", "dense", "peaks", "dis"],
                    help="fit: the fit step (default, the headline line); stress: one convolution "
                         "of the hadronic stress table (2000 x 196 channels x 50 x 50) for kernel rooflines; "
                         "serve: the served mixed workload (Poisson arrivals over 41 resident tables); "
                         "descent: Adam on the PDF parameters of every replica, iterations of the fit; "
                         "dense: the paper's Table 3 product FK[ndata x 35721] . PDF[35721 x R] "
                         "(--ndata, --replicas; default 2000 x 2000); "
                         "peaks: measures the TF32 (cuBLAS), FP32 and FP64 (multiply-add loops) peaks; "
                         "dis: the config-0 DIS table (64 x 9 x 40), --stack copies stacked along the data "
                         "points, --replicas (default 1), --prec (default fp64 here)")
    ap.add_argument("--stack", type=int, default=1, help="dis case: config-0 tables stacked")
    ap.add_argument("--kdense", type=int, default=0,
                    help="dense case: a seeded random table [ndata][kdense] instead of Table 3's base table")
    ap.add_argument("--requests", type=int, default=2000, help="serve case: number of requests")
    ap.add_argument("--rate", type=float, default=2000.0, help="serve case: arrivals per second")
    ap.add_argument("--ndata", type=int, default=2000, help="stress case: data points")
    ap.add_argument("--form", default="factored", choices=["factored", "lumi"],
                    help="stress case, reduced modes: the hadronic forward's formulation (FK_TABLE_LUMI)")
    ap.add_argument("--table", default="stress", choices=["stress", "config1"],
                    help="stress case: the stress table, or the plain hadronic table of configs 1-2 "
                         "(200 data points, 60 channels, nx = 30; R = 512 is config 2)")
    ap.add_argument("--replicas", type=int, default=None,
                    help="stress case: replicas (default 1); dense case: columns of the PDF matrix (default 2000)")
    return ap.parse_args()


def peaks():
    """HBM and BF16 peaks from MEASURED_PEAKS.json (driver-measured), plus the
    TF32, FP32 and FP64 peaks this repository measured the same way
    (profiles/peaks.txt, written from `bench.py --case peaks`)."""
    p = os.path.join(HERE, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            m = json.load(f)
        src = "measured"
    else:
        m = {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "bf16_tflops_sustained": 1400.0, "sm_max_mhz": 2032.0}
        src = "fallback"
    try:
        for ln in open(os.path.join(HERE, "profiles", "peaks.txt")):
            w = ln.split()
            if len(w) >= 2 and not ln.startswith("#") and w[0].endswith("_tflops"):
                m[w[0]] = float(w[1])
    except OSError:
        pass
    return m, src


def peak_of(prec, pk, sustained=False):
    """(TFLOP/s, source) of the arithmetic a mode runs on: the tensor pipe for
    BF16 / BF16 hi+lo (BF16 peak) and TF32, the CUDA cores for FP32 and FP64."""
    mhz = pk.get("sm_max_mhz", 2032.0)
    if prec in ("bf16", "bf16x3", "fp64tc"):
        return (pk["bf16_tflops_sustained"] if sustained else pk["bf16_tflops"]), "measured (cuBLAS BF16)"
    if prec == "tf32":
        if "tf32_tflops" in pk:
            return pk["tf32_tflops"], "measured (cuBLAS TF32, profiles/peaks.txt)"
        return pk["bf16_tflops"] / 2.0, "BF16 measured / 2 (nominal ratio)"
    if prec == "fp32":
        if "fp32_tflops" in pk:
            return pk["fp32_tflops"], "measured (FP32 FMA loop, profiles/peaks.txt)"
        return 148 * 128 * 2 * mhz * 1e6 / 1e12, "derived: 148 SMs x 128 FMA/clock x max clock"
    if "fp64_tflops" in pk:
        return pk["fp64_tflops"], "measured (FP64 FMA loop, profiles/peaks.txt)"
    return 148 * 2 * 2 * mhz * 1e6 / 1e12, "derived: 148 SMs x 2 FP64 FMA/clock x max clock"


def dist_init(n):
    import torch
    import torch.distributed as dist
    if n <= 1 or "RANK" not in os.environ:
        return 0, 1, None
    rank = int(os.environ["RANK"])
    world = int(os.environ["WORLD_SIZE"])
    local = int(os.environ.get("LOCAL_RANK", rank))
    backend = "nccl" if torch.cuda.is_available() else "gloo"
    if torch.cuda.is_available():
        torch.cuda.set_device(local)
    dist.init_process_group(backend)
    return rank, world, dist


def max_over_ranks(dist, x):
    import torch
    if dist is None:
        return x
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank, world, ms_max):
    """Whole-job rate: every rank processes units_per_rank per step (weak
    scaling, replicas only), the job's step time is the slowest rank's."""
    return units_per_rank * world / (ms_max * 1e-3)


def workload():
    from paper_1909_10547_b300 import workloads as W
    g = W.config3(R=REPLICAS, seed=SEED)
    return g


class Clocks:
    """Samples SM clocks and throttle reasons during a region: through NVML
    every 5 ms from a thread (read-only queries), else with nvidia-smi at its
    100 ms interval.  Nothing here changes a GPU setting."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    NAMES = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]

    def __init__(self, index):
        self.index = index
        self.p = None
        self.nv = None
        self.samples = []  # (sm MHz, max sm MHz, reasons)

    class _CNVML:
        """The few read-only NVML calls used here, through ctypes (when the
        pynvml module is not installed)."""
        NVML_CLOCK_SM = 1
        nvmlClocksEventReasonSwPowerCap = 0x4
        nvmlClocksEventReasonHwSlowdown = 0x8
        nvmlClocksEventReasonSwThermalSlowdown = 0x20
        nvmlClocksEventReasonHwThermalSlowdown = 0x40

        def __init__(self):
            import ctypes
            self.ct = ctypes
            self.lib = ctypes.CDLL("libnvidia-ml.so.1")
            if self.lib.nvmlInit_v2() != 0:
                raise OSError("nvmlInit failed")

        def _check(self, rc):
            if rc != 0:
                raise OSError(f"NVML error {rc}")

        def nvmlDeviceGetHandleByIndex(self, i):
            h = self.ct.c_void_p()
            self._check(self.lib.nvmlDeviceGetHandleByIndex_v2(self.ct.c_uint(i), self.ct.byref(h)))
            return h

        def nvmlDeviceGetHandleByUUID(self, uuid):
            h = self.ct.c_void_p()
            self._check(self.lib.nvmlDeviceGetHandleByUUID(self.ct.c_char_p(uuid.encode()), self.ct.byref(h)))
            return h

        def nvmlDeviceGetClockInfo(self, h, kind):
            v = self.ct.c_uint()
            self._check(self.lib.nvmlDeviceGetClockInfo(h, self.ct.c_int(kind), self.ct.byref(v)))
            return v.value

        def nvmlDeviceGetMaxClockInfo(self, h, kind):
            v = self.ct.c_uint()
            self._check(self.lib.nvmlDeviceGetMaxClockInfo(h, self.ct.c_int(kind), self.ct.byref(v)))
            return v.value

        def nvmlDeviceGetCurrentClocksEventReasons(self, h):
            v = self.ct.c_ulonglong()
            f = getattr(self.lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
                self.lib.nvmlDeviceGetCurrentClocksThrottleReasons
            self._check(f(h, self.ct.byref(v)))
            return v.value

    def _nvml_handle(self):
        try:
            import pynvml
            pynvml.nvmlInit()
        except ImportError:
            pynvml = self._CNVML()
        try:
            import torch
            uuid = str(torch.cuda.get_device_properties(self.index).uuid)
            return pynvml, pynvml.nvmlDeviceGetHandleByUUID(uuid if uuid.startswith("GPU-") else "GPU-" + uuid)
        except Exception:
            return pynvml, pynvml.nvmlDeviceGetHandleByIndex(self.index)

    def _poll(self):
        nv, h = self.nv
        bits = [nv.nvmlClocksEventReasonHwSlowdown, nv.nvmlClocksEventReasonHwThermalSlowdown,
                nv.nvmlClocksEventReasonSwThermalSlowdown, nv.nvmlClocksEventReasonSwPowerCap]
        mx = nv.nvmlDeviceGetMaxClockInfo(h, nv.NVML_CLOCK_SM)
        while not self.stop.is_set():
            try:
                sm = nv.nvmlDeviceGetClockInfo(h, nv.NVML_CLOCK_SM)
                r = nv.nvmlDeviceGetCurrentClocksEventReasons(h)
                self.samples.append((sm, mx, {n for n, b in zip(self.NAMES, bits) if r & b}))
            except Exception:
                break
            self.stop.wait(0.005)

    def __enter__(self):
        try:
            import threading
            self.nv = self._nvml_handle()
            self.stop = threading.Event()
            self.th = threading.Thread(target=self._poll, daemon=True)
            self.th.start()
            return self
        except Exception:
            self.nv = None
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "100"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.p = None
        return self

    def __exit__(self, *a):
        if self.nv is not None:
            self.stop.set()
            self.th.join(timeout=5)
        if self.p is not None:
            self.p.terminate()
            try:
                self.out, _ = self.p.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.p.kill()
                self.out = ""
            for line in self.out.strip().splitlines():
                f = [x.strip() for x in line.split(",")]
                if len(f) < 9:
                    continue
                try:
                    self.samples.append((float(f[1]), float(f[2]),
                                         {n for n, v in zip(self.NAMES, f[5:9]) if v.lower().startswith("active")}))
                except ValueError:
                    continue
        return False

    def summary(self):
        if not self.samples:
            return None
        reasons = set().union(*(r for _, _, r in self.samples))
        return {"sm_mhz": statistics.median(s for s, _, _ in self.samples),
                "sm_max_mhz": max(m for _, m, _ in self.samples), "reasons": sorted(reasons),
                "samples": len(self.samples), "source": "nvml" if self.nv is not None else "nvidia-smi"}


def cpu_baseline(g, blocks, D_parts, replicas_all=16, replicas_one=1):
    """The FP64 oracle (as it stands) on bounded samples of the same fit step
    (same tables, covariance blocks and pseudo-data as the GPU run): the first
    `replicas_all` replicas on all host cores (best of 5) and `replicas_one`
    on one core (best of 3).  Also returns the oracle's chi^2 and dchi2/dF of
    the all-core sample, which the accuracy block compares with the GPU."""
    import oracle
    Ls = [oracle.cholesky(b) for b in blocks]

    def run(F):
        chi = np.zeros(F.shape[0])
        gF = np.zeros_like(F)
        for t, L, d in zip(g.tables, Ls, D_parts):
            O, _ = oracle.conv(t, F)
            c, gO = oracle.chi2(L, O, d)
            chi += c
            gF += oracle.conv_grad(t, F, gO)
        return chi, gF

    def best(F, n):
        b = float("inf")
        out = None
        for _ in range(n):
            t0 = time.perf_counter()
            out = run(F)
            b = min(b, time.perf_counter() - t0)
        return b, out

    ntot = sum(t.ndata for t in g.tables)
    cores = oracle.threads()
    t_all, (chi, gF) = best(g.F[:replicas_all], 5)
    oracle.set_threads(1)
    try:
        t_one, _ = best(g.F[:replicas_one], 3)
    finally:
        oracle.set_threads(cores)
    return {"value": ntot * replicas_all / t_all, "cores": cores, "seconds": t_all, "replicas": replicas_all,
            "value_1core": ntot * replicas_one / t_one, "seconds_1core": t_one, "replicas_1core": replicas_one,
            "chi2": chi, "gF": gF}


def time_calls(fn, steps, flush=None):
    """Milliseconds per call of fn (one CUDA graph of it, replayed).  Warm:
    `steps` replays back to back between two events.  With flush (a tensor
    larger than L2): before every call flush is overwritten, then that call
    alone is timed; the mean of the calls is returned."""
    import torch
    fn()
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        fn()
    for _ in range(3):
        g.replay()
    torch.cuda.synchronize()
    if flush is None:
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            g.replay()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / steps
    tot = 0.0
    for _ in range(steps):
        flush.add_(1.0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        g.replay()
        e1.record()
        torch.cuda.synchronize()
        tot += e0.elapsed_time(e1)
    return tot / steps


def roof_entry(prec, byts, flops, ms, kernel, traffic=None):
    """Roofline of one timed call: HBM when flops/bytes is below the ridge of
    the mode's peak, else the tensor pipe (reduced modes) or the CUDA cores."""
    pk, src = peaks()
    tpeak, psrc = peak_of(prec, pk)
    ridge = tpeak * 1e12 / (pk["hbm_gbs"] * 1e9)
    tc = prec in ("bf16", "bf16x3", "tf32", "fp64tc")
    if prec == "fp64tc":
        # FP64 results from 36 BF16 digit products per multiply-add: the
        # tensor pipe's issued rate against the BF16 peak, and the useful FP64
        # rate against the FP64 pipe's
        iss = ISSUED[prec] * flops / (ms * 1e-3) / 1e12
        f64pk, f64src = peak_of("fp64", pk)
        return {"bound": "tensor", "achieved": iss, "peak": tpeak, "unit": "TFLOP/s", "frac": iss / tpeak,
                "issued": True, "useful_tflops": flops / (ms * 1e-3) / 1e12,
                "useful_vs_fp64_peak": flops / (ms * 1e-3) / 1e12 / f64pk, "fp64_peak_source": f64src,
                "algorithmic_flops": flops, "peak_source": psrc, "traffic": traffic, "kernel": kernel}
    if flops / byts < ridge:
        ach = byts / (ms * 1e-3) / 1e9
        r = {"bound": "hbm", "achieved": ach, "peak": pk["hbm_gbs"], "unit": "GB/s", "frac": ach / pk["hbm_gbs"],
             "algorithmic_bytes": byts, "peak_source": src}
    else:
        ach = flops / (ms * 1e-3) / 1e12
        r = {"bound": "tensor" if tc else "alu", "achieved": ach, "peak": tpeak, "unit": "TFLOP/s",
             "frac": ach / tpeak, "algorithmic_flops": flops, "peak_source": psrc}
    r["traffic"] = traffic
    r["kernel"] = kernel
    return r


def chi2_line(args, cov, o_true, D, R=REPLICAS):
    """The FP64 chi^2 with its gradient (blocked forward and back
    substitutions, fk_chi2) on the global set's 40 covariance blocks, R = 100
    replicas of FP32 observables: the fit step itself runs on whitened tables,
    so the solve is timed here.  Roofline: the FP64 pipe, sum n_k^2 R
    multiply-adds (both substitutions)."""
    import torch
    import paper_1909_10547_b300 as fk
    dcov = fk.Cov(cov.blocks)
    o = np.concatenate(o_true)
    rng = np.random.default_rng(SEED + 2)
    O = torch.tensor(o[None, :] * rng.uniform(0.9, 1.1, (R, o.size)), dtype=torch.float32, device="cuda")
    Dd = torch.tensor(np.asarray(D, np.float64), device="cuda")
    c = torch.empty(R, dtype=torch.float64, device="cuda")
    g = torch.empty_like(O)
    ms = time_calls(lambda: fk.chi2(dcov, O, Dd, out=c, gO=g), max(args.steps, 20))
    nn = int(sum(b.shape[0] ** 2 for b in cov.blocks))
    return {"name": f"FP64 chi^2 + gradient, blocked substitutions, {len(cov.blocks)} blocks ({o.size} points), "
                    f"R={R}", "prec": "fp64", "value": o.size * R / (ms * 1e-3), "unit": UNIT, "ms": ms,
            "roofline": roof_entry("fp64", 2 * nn * 8, 2.0 * nn * R, ms, "k_chi2_solve (one launch per call)")}


def kernel_lines(args, stress_tab=None, stress_t=None, stress_oz=None):
    """Kernel-level lines: each one call of one path, timed on its own with
    its own roofline.  Stress table (2000 x 196 channels x 50 x 50; resident
    tables far larger than L2): R = 1 FP32 streaming and R = 1000 BF16 on the
    tensor cores.  Configs 1-2 table (200 x 60 x 30 x 30, 43 MB in FP32: it
    fits in L2, so each line is given warm, back to back, and cold, L2 flushed
    by a 256 MB write before every call).  Config 0 (DIS, 64 x 9 x 40, FP64,
    R = 1): one call's latency, and 4096 such tables stacked into one table
    (262144 data points, 755 MB) for bandwidth.  Table 3's R = 1 rows with
    K = 10^6 and 10^7 (ndata = 8, FP32 streaming of the dense table)."""
    import torch
    import paper_1909_10547_b300 as fk
    from paper_1909_10547_b300 import workloads as W
    out = []
    steps = max(args.steps, 20)
    flush = torch.empty(64 << 20, dtype=torch.float32, device="cuda")  # 256 MB > L2

    def line(name, prec, units, ms, roof, **extra):
        d = {"name": name, "prec": prec, "value": units / (ms * 1e-3), "unit": UNIT, "ms": ms,
             "roofline": roof}
        d.update(extra)
        out.append(d)

    # stress table
    if stress_tab is not None:
        nd = stress_t.ndata
        elems = stress_t.fk.size
        F1 = torch.tensor(W.pdf_replicas(W.xgrid(50, 1e-7), W.pdf_params(np.random.default_rng(1)), 1, None),
                          dtype=torch.float32, device="cuda")
        O1 = torch.empty((1, nd), dtype=torch.float32, device="cuda")
        ms = time_calls(lambda: fk.conv(stress_tab, F1, "fp32", out=O1), steps)
        line("stress table 2000x196x50x50, R=1, FP32 streaming", "fp32", nd, ms,
             roof_entry("fp32", elems * 4, 2.0 * elems, ms, "k_stream",
                        traffic_of("k_stream", "fp32", nd, 1)))
        R = 1000
        FR = torch.tensor(W.pdf_replicas(W.xgrid(50, 1e-7), W.pdf_params(np.random.default_rng(1)), R,
                                         np.random.default_rng(2)), dtype=torch.float32, device="cuda")
        OR = torch.empty((R, nd), dtype=torch.float32, device="cuda")
        for prec in ("bf16", "bf16x3"):
            ms = time_calls(lambda: fk.conv(stress_tab, FR, prec, out=OR), max(5, steps // 4))
            line(f"stress table, R=1000, {prec} tensor cores", prec, nd * R, ms,
                 roof_entry(prec, elems * ESZ[prec], 2.0 * elems * R, ms,
                            "k_tc (whole call: operand packing + tcgen05 kernel)", traffic_of("k_tc", prec, nd, R)))
        del FR, OR
        if stress_oz is not None:
            R = 100
            F64 = torch.tensor(W.pdf_replicas(W.xgrid(50, 1e-7), W.pdf_params(np.random.default_rng(1)), R,
                                              np.random.default_rng(2)), device="cuda")
            O64 = torch.empty((R, nd), dtype=torch.float64, device="cuda")
            ms = time_calls(lambda: fk.conv(stress_oz, F64, "fp64tc", out=O64), 3)
            line("stress table, R=100, FP64 results on the tensor cores (fp64tc)", "fp64tc", nd * R, ms,
                 roof_entry("fp64tc", elems * 8, 2.0 * elems * R, ms,
                            "k_oz_slice + k_tc digit pairs + k_oz_combine (whole call)"),
                 fp64_pipe_ms_reference="249 ms (k_fac FP64, bench.py --case stress --prec fp64 --replicas 100)")
            del F64, O64
    # configs 1-2 table
    t1, F1h = W.config1(R=512)
    tab1 = fk.Table.from_workload(t1, precs=("fp64", "fp32", "bf16", "bf16x3", "tf32", "fp64tc"))
    e1 = t1.fk.size
    nd1 = t1.ndata
    Fa = torch.tensor(F1h, dtype=torch.float32, device="cuda")
    Oa = torch.empty((512, nd1), dtype=torch.float32, device="cuda")
    Fs = Fa[:1].contiguous()
    Os = torch.empty((1, nd1), dtype=torch.float32, device="cuda")
    for cold in (False, True):
        ms = time_calls(lambda: fk.conv(tab1, Fs, "fp32", out=Os), steps, flush if cold else None)
        line(f"config 1 table 200x60x30x30, R=1, FP32 streaming, {'cold L2' if cold else 'warm L2'}", "fp32", nd1,
             ms, roof_entry("fp32", e1 * 4, 2.0 * e1, ms, "k_stream"))
    for prec in ("bf16", "tf32", "bf16x3"):
        for cold in (False, True):
            ms = time_calls(lambda: fk.conv(tab1, Fa, prec, out=Oa), steps, flush if cold else None)
            line(f"config 2: config 1 table, R=512, {prec} tensor cores, {'cold L2' if cold else 'warm L2'}", prec,
                 nd1 * 512, ms, roof_entry(prec, e1 * ESZ[prec], 2.0 * e1 * 512, ms,
                                           "k_tc (whole call: operand packing + tcgen05 kernel)"))
    # config 1 at R = 100 with FP64 results: the FP64 pipe against the tensor cores
    F100 = torch.tensor(F1h[:100], device="cuda")
    O100 = torch.empty((100, nd1), dtype=torch.float64, device="cuda")
    for prec, kern in (("fp64", "k_fac (FP64 pipe)"), ("fp64tc", "k_oz_slice + k_tc digit pairs + k_oz_combine")):
        ms = time_calls(lambda: fk.conv(tab1, F100, prec, out=O100), steps)
        line(f"config 1: R=100, FP64 results, {prec}", prec, nd1 * 100, ms,
             roof_entry(prec, e1 * 8, 2.0 * e1 * 100, ms, kern))
    del tab1
    # config 0 (DIS, FP64, R = 1) and 4096 of its tables stacked
    t0, F0h = W.config0()
    tab0 = fk.Table.from_workload(t0, precs=("fp64",))
    F0 = torch.tensor(F0h, device="cuda")
    O0 = torch.empty((1, t0.ndata), dtype=torch.float64, device="cuda")
    used0 = t0.ndata * len(t0.flav) * t0.nx
    for cold in (False, True):
        ms = time_calls(lambda: fk.dis_conv(tab0, F0, "fp64", out=O0), steps, flush if cold else None)
        line(f"config 0: DIS 64x9x40, R=1, FP64, one call ({'cold L2' if cold else 'warm L2'})", "fp64", t0.ndata, ms,
             roof_entry("fp64", used0 * 8, 2.0 * used0, ms, "k_stream<DIS> + k_reduce_parts"),
             latency_us=ms * 1e3)
    del tab0
    nb = 4096
    rng = np.random.default_rng(10547)
    big = np.abs(rng.standard_normal((nb * t0.ndata, len(t0.flav), t0.nx))) * (W.xgrid(t0.nx, 1e-7) ** 0.3)[None, None, :]
    tabb = fk.Table.dis(big, t0.flav, None, t0.nx, precs=("fp64", "fp32"))
    del big
    ub = used0 * nb
    F0s = F0.float()
    for prec, Fx in (("fp64", F0), ("fp32", F0s)):
        Ob = torch.empty((1, nb * t0.ndata), dtype=Fx.dtype, device="cuda")
        ms = time_calls(lambda: fk.dis_conv(tabb, Fx, prec, out=Ob), steps)
        line(f"config 0 x 4096: 4096 DIS tables 64x9x40 stacked (262144 points), R=1, {prec}", prec,
             nb * t0.ndata, ms, roof_entry(prec, ub * ESZ[prec], 2.0 * ub, ms, "k_stream<DIS> + k_reduce_parts"))
    del tabb
    # Table 3 rows with R = 1: ndata = 8, K = 1e6, 1e7, 1e8 (the last table is 3.2 GB in FP32; its
    # values are drawn in FP32, which the table's FP32 copy holds exactly)
    for K in (10 ** 6, 10 ** 7, 10 ** 8):
        fkd = np.random.default_rng(K).standard_normal((8, K), dtype=np.float32)
        tabd = fk.Table.dense(fkd, precs=("fp32",))
        del fkd
        L = torch.rand((1, K), dtype=torch.float32, device="cuda")
        Od = torch.empty((1, 8), dtype=torch.float32, device="cuda")
        ms = time_calls(lambda: fk.dense_conv(tabd, L, "fp32", out=Od), steps, flush if 8 * K * 4 < 126e6 else None)
        line(f"Table 3 row: dense 8 x {K:.0e} . PDF [{K:.0e} x 1], FP32 streaming", "fp32", 8, ms,
             roof_entry("fp32", 8 * K * 4 + K * 4, 2.0 * 8 * K, ms, "k_stream<DENSE> + k_reduce_parts"),
             paper_seconds={10 ** 6: 5.0e-3, 10 ** 7: 5.7e-2, 10 ** 8: 5.7e-1}[K])
        del tabd, L
    # Table 3's last line (2000 x 35721 x 2000) with FP64 results on the tensor cores
    t3, F3 = W.table3(2000, 2000)
    K3 = t3.fk[0].size
    tab3 = fk.Table.dense(t3.fk.reshape(2000, K3), precs=("fp64tc",))
    ht3 = fk.Table.from_workload(t3, precs=("fp64",))
    del t3
    L3 = fk.luminosity(ht3, torch.tensor(F3, device="cuda"), "fp64")
    O3 = torch.empty((2000, 2000), dtype=torch.float64, device="cuda")
    ms = time_calls(lambda: fk.dense_conv(tab3, L3, "fp64tc", out=O3), 3)
    line("Table 3 line 147: dense 2000 x 35721 . PDF [35721 x 2000], FP64 results on the tensor cores", "fp64tc",
         2000 * 2000, ms, roof_entry("fp64tc", 2000 * K3 * 8, 2.0 * 2000 * K3 * 2000, ms,
                                     "k_oz_slice + k_tc digit pairs + k_oz_combine"),
         paper_seconds=1.38, fp64_pipe_ms_reference="254 ms (k_tile FP64, bench.py --case dense --prec fp64)")
    del tab3, ht3, L3, O3
    return out


def serve_block(args, g, tabs, tprec, stress_tab=None, n=2000, rate=2000.0, plain_prec=None):
    """The served mixed workload, bounded: n requests with Poisson arrivals at
    `rate` over the global-set tables (+ the stress table), R from
    {1, 10, 100, 1000}, resident tables, 150 GB budget.  Reports open-loop
    p50/p99/max latency (submit to the poll that sees the result), the
    saturation throughput (closed loop, 64 in flight) and the same requests
    one at a time through the plain per-request path (H2D, conv, D2H)."""
    import threading
    import torch
    import paper_1909_10547_b300 as fk
    from paper_1909_10547_b300 import workloads as W
    alltabs = list(tabs) + ([stress_tab] if stress_tab is not None else [])
    allprec = list(tprec) + ([args.prec] if stress_tab is not None else [])
    nxg = [t.nxg for t in alltabs]
    srv = fk.Server(budget_bytes=150 << 30, max_inflight=8)
    ids = [srv.add_table(t) for t in alltabs]
    rng = np.random.default_rng(SEED + 1)
    which = rng.integers(0, len(alltabs), n)
    Rs = rng.choice(W.REPLICA_CHOICES, n)
    arr = W.arrivals(rng, rate, n)
    pool = {}
    for k in range(n):
        key = (nxg[which[k]], int(Rs[k]), allprec[which[k]])
        if key not in pool:
            x = g.x if key[0] == 50 else W.xgrid(key[0], 1e-7)
            F = W.pdf_replicas(x, g.params, key[1], np.random.default_rng(key[1]))
            pool[key] = F.astype(np.float64 if key[2] in ("fp64", "fp64tc") else np.float32)
    work = [(int(which[k]), pool[(nxg[which[k]], int(Rs[k]), allprec[which[k]])], allprec[which[k]])
            for k in range(n)]
    units = sum(alltabs[w].ndata * F.shape[0] for w, F, _ in work)
    # warm-up: every (table, R) pair of the run once through the server and
    # once through the plain path, so that no kernel is loaded (the CUDA
    # runtime loads each kernel on its first launch) inside the timed runs
    stage(f"  serve: warm-up of {len(alltabs)} tables")
    seen = {}
    for w, F, p in work:
        seen.setdefault((w, F.shape[0]), (w, F, p))
    for w, F, p in seen.values():
        srv.wait(srv.submit(ids[w], F, p), 120000)
        fk.conv(alltabs[w], torch.from_numpy(F).to("cuda"), plain_prec or p).cpu()
    tickets = [None] * n
    t_sub = np.zeros(n)
    t_done = np.zeros(n)

    poll_err = []

    def poller():
        outstanding = set()
        nxt = 0
        deadline = time.perf_counter() + 300.0
        while nxt < n or outstanding:
            if time.perf_counter() > deadline:
                poll_err.append(f"{len(outstanding)} requests unresolved after 300 s")
                return
            while nxt < n and tickets[nxt] is not None:
                outstanding.add(nxt)
                nxt += 1
            for k in list(outstanding):
                ok, _ = srv.poll(tickets[k])
                if ok:
                    t_done[k] = time.perf_counter()
                    outstanding.discard(k)
            time.sleep(0.0001)

    th = threading.Thread(target=poller, daemon=True)
    stage(f"  serve: open loop, {n} requests")
    th.start()
    t0 = time.perf_counter()
    for k, (w, F, p) in enumerate(work):
        delay = t0 + arr[k] - time.perf_counter()
        if delay > 0:
            time.sleep(delay)
        t_sub[k] = time.perf_counter()
        tickets[k] = srv.submit(ids[w], F, p)
    th.join()
    if poll_err:
        raise TimeoutError("served mix: " + poll_err[0])
    lat = (t_done - t_sub) * 1e3
    span = t_done.max() - t_sub.min()
    s0 = time.perf_counter()
    inflight = []
    for w, F, p in work:
        if len(inflight) >= 64:
            srv.wait(inflight.pop(0), 120000)
        inflight.append(srv.submit(ids[w], F, p))
    for tk in inflight:
        srv.wait(tk, 120000)
    sat = time.perf_counter() - s0
    st = srv.stats()
    srv.close()
    t1 = time.perf_counter()
    plain = []
    for w, F, p in work:
        a = time.perf_counter()
        Fd = torch.from_numpy(F).to("cuda")
        fk.conv(alltabs[w], Fd, plain_prec or p).cpu()
        plain.append((time.perf_counter() - a) * 1e3)
    plain_span = time.perf_counter() - t1
    return {"requests": n, "offered_rate": rate, "tables": len(alltabs), "mode": allprec[0],
            "per_request_mode": plain_prec or allprec[0],
            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "max_ms": float(lat.max()), "achieved_rate": n / span, "open_loop_value": units / span,
            "saturation_value": units / sat, "unit": UNIT, "launches": st["launches"],
            "per_request": {"value": units / plain_span, "p50_ms": float(np.percentile(plain, 50)),
                            "p99_ms": float(np.percentile(plain, 99)),
                            "what": "one request at a time: H2D, fk conv, D2H, synchronise"}}


def run_peaks(args):
    """TF32 tensor-core peak by the MEASURED_PEAKS method (cuBLAS 8192^3 GEMM
    through torch, best of 10 and back to back for 4 s), and the FP32 / FP64
    CUDA-core multiply-add rates with fk_fma_probe (8 chains per thread, one
    wave of 8 CTAs of 256 threads per SM, best of 10 and 4 s back to back).
    The clock is sampled throughout."""
    import ctypes
    import torch
    import paper_1909_10547_b300 as fk
    from paper_1909_10547_b300 import _lib
    res = {}
    torch.backends.cuda.matmul.allow_tf32 = True
    a = torch.randn(8192, 8192, device="cuda")
    b = torch.randn(8192, 8192, device="cuda")
    c = torch.empty(8192, 8192, device="cuda")

    def rate(fn, flops):
        fn()
        torch.cuda.synchronize()
        best = 0.0
        for _ in range(10):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            fn()
            e1.record()
            torch.cuda.synchronize()
            best = max(best, flops / (e0.elapsed_time(e1) * 1e-3) / 1e12)
        n = 0
        t0 = time.perf_counter()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        while time.perf_counter() - t0 < 4.0:
            fn()
            n += 1
            if n % 8 == 0:
                torch.cuda.synchronize()
        e1.record()
        torch.cuda.synchronize()
        return best, flops * n / (e0.elapsed_time(e1) * 1e-3) / 1e12

    with Clocks(torch.cuda.current_device()) as clk:
        res["tf32_tflops"], res["tf32_tflops_sustained"] = rate(lambda: torch.matmul(a, b, out=c), 2.0 * 8192 ** 3)
        del a, b, c
        sms = torch.cuda.get_device_properties(0).multi_processor_count
        blocks = 8 * sms
        lib = _lib.load()
        for name, prec, dt, iters in (("fp32", _lib.FK_FP32, torch.float32, 1 << 16),
                                      ("fp64", _lib.FK_FP64, torch.float64, 1 << 11)):
            sink = torch.zeros(blocks, dtype=dt, device="cuda")
            stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
            fl = 2.0 * 8 * iters * 256 * blocks
            res[f"{name}_tflops"], res[f"{name}_tflops_sustained"] = rate(
                lambda: lib.fk_fma_probe(prec, blocks, iters, ctypes.c_void_p(sink.data_ptr()), stream), fl)
        # cycles one BF16 tcgen05.mma (M = 128, K = 16) takes, by N: best of 5 runs of 4096
        cyc = torch.zeros(1, dtype=torch.int64, device="cuda")
        stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        for fill, key in ((1, "tcgen05_f16_mma_cycles_by_n"), (0, "tcgen05_f16_mma_cycles_by_n_zero_operands")):
            per = {}
            for n in (64, 128, 192, 240, 256):
                best = None
                for _ in range(5):
                    _lib.call("fk_mma_probe", n, 4096, fill, ctypes.c_void_p(cyc.data_ptr()), stream)
                    torch.cuda.synchronize()
                    v = cyc.item() / 4096
                    best = v if best is None else min(best, v)
                per[str(n)] = round(best, 1)
            res[key] = per
    res["clocks"] = clk.summary()
    res["how"] = ("TF32: torch.matmul fp32 8192^3 with TF32 allowed (cuBLAS), 2 N^3 flops; FP32 / FP64: "
                  "fk_fma_probe, 8 independent FMA chains per thread, 8 x SMs CTAs of 256 threads; best of 10 "
                  "(burst) and back to back for 4 s (sustained), CUDA events; MMA cycles: fk_mma_probe, one CTA, "
                  "4096 back-to-back BF16 tcgen05.mma of 128 x N x 16, SM cycles per instruction, best of 5")
    print(json.dumps(res), flush=True)


def run_reference(args, rank, world, dist):
    """Reference arm: the FP64 CPU oracle on the host cores (rank 0 only)."""
    if rank != 0:
        return
    g = workload()
    per_step = max(1, min(8, int(150.0 / (0.5 * (args.steps + args.warmup)))))
    import oracle
    from paper_1909_10547_b300 import workloads as W
    o_true = [oracle.conv(t, g.F_true)[0][0] for t in g.tables]
    cov = W.covariance(o_true, SEED)
    D = W.pseudo_data(o_true, SEED)
    Ls = [oracle.cholesky(b) for b in cov.blocks]
    F = g.F[:per_step]

    def step():
        for t, L, d in zip(g.tables, Ls, D):
            O, _ = oracle.conv(t, F)
            _, gO = oracle.chi2(L, O, d)
            oracle.conv_grad(t, F, gO)

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = (time.perf_counter() - t0) / max(1, args.steps)
    ntot = sum(t.ndata for t in g.tables)
    v = ntot * per_step / dt
    sample = f"{per_step} of {REPLICAS} replicas per step, all 40 tables, FP64"
    line = {"metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": config_dict(g, "fp64", graphs=False),
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": oracle.threads(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# table bytes per element of the definition in each mode (FP64_TC: the FP64 values it reproduces)
ESZ = {"fp64": 8, "fp32": 4, "bf16": 2, "bf16x3": 4, "tf32": 4, "fp64tc": 8}
# MMAs issued per multiply-add of the definition
ISSUED = {"bf16x3": 3, "fp64tc": 36}


def roofline(fit, seg, prec):
    """Roofline entry for the pipelined step as a whole, or (phase-separated
    step) for the phase that takes longest.

    Algorithmic bytes of a convolution phase: every table element streamed
    once in the mode's storage (BF16 hi+lo: 4 B).  Algorithmic flops: 2 per
    multiply-add of the definition.
    The bound is HBM when flops/bytes is below the ridge of the measured
    peaks, else the tensor pipe (reduced modes) or the ALUs (FP32 / FP64 on
    the CUDA cores).  The FP64 chi^2 phase is bound by the FP64 multiply-add
    rate (peak_of: measured with fk_fma_probe when profiles/peaks.txt has it)."""
    pk, src = peaks()
    dom = max(seg, key=seg.get)
    t = seg[dom] * 1e-3
    tc = prec in ("bf16", "bf16x3", "tf32")
    if dom == "step":
        # pipelined: the phases overlap; every table is streamed once by the
        # forward and once by the adjoint within the step
        flops = sum(fit.flops.values())
        byts = 2 * (fit.elems["had"] + fit.elems["dis"]) * ESZ[prec]
        ach = byts / t / 1e9
        return {"bound": "hbm", "achieved": ach, "peak": pk["hbm_gbs"], "unit": "GB/s",
                "frac": ach / pk["hbm_gbs"], "traffic": None,
                "kernel": "whole pipelined step (forward, FP64 chi^2 and adjoint overlapped)",
                "algorithmic_bytes": byts, "algorithmic_flops": flops, "peak_source": src}
    flops = fit.flops[dom]
    if dom == "loss":
        peak, psrc = peak_of("fp64", pk)
        return {"bound": "alu", "achieved": flops / t / 1e12, "peak": peak, "unit": "TFLOP/s",
                "frac": flops / t / 1e12 / peak, "traffic": None, "kernel": "loss phase (FP64 chi^2)",
                "peak_source": psrc, "phase_ms": seg}
    had_b = fit.elems["had"] * ESZ[prec]
    dis_b = fit.elems["dis"] * ESZ[prec]
    byts = had_b + dis_b
    tpeak, _ = peak_of(prec, pk, sustained=True)
    ridge = tpeak * 1e12 / (pk["hbm_gbs"] * 1e9)
    if flops / byts < ridge:
        ach = byts / t / 1e9
        return {"bound": "hbm", "achieved": ach, "peak": pk["hbm_gbs"], "unit": "GB/s",
                "frac": ach / pk["hbm_gbs"], "traffic": None, "kernel": f"{dom} phase",
                "algorithmic_bytes": byts, "peak_source": src, "phase_ms": seg}
    ach = flops / t / 1e12
    return {"bound": "tensor" if tc else "alu", "achieved": ach, "peak": tpeak, "unit": "TFLOP/s",
            "frac": ach / tpeak, "traffic": None, "kernel": f"{dom} phase", "peak_source": src,
            "phase_ms": seg}


def config_dict(g, prec, table_bytes=None, graphs=True):
    ntot = sum(t.ndata for t in g.tables)
    elems = sum(t.fk.size for t in g.tables)
    l2 = (f"inputs larger than L2 (resident FK tables {table_bytes / 1e9:.2f} GB on the device)"
          if table_bytes else f"inputs larger than L2 ({elems / 1e6:.0f}M FK elements, {8 * elems / 1e9:.2f} GB in FP64)")
    return {"workload": "global-shaped chi2 fit step (forward + FP64 chi2 + adjoint): 40 datasets "
                        "(12 DIS, 28 hadronic), nx 20..50 on a 50-point grid, 20..120 channels",
            "ndata_total": ntot, "replicas": REPLICAS, "tables": len(g.tables), "prec": prec,
            "l2": l2, "graphs": graphs, "parallelism": "replicas only (one independent copy per rank)"}


def traffic_of(kernel, prec, ndata, replicas):
    """DRAM bytes per launch of `kernel` for this workload, from the
    committed one-kernel ncu capture list
    (profiles/dram_traffic.txt), or None when no capture matches or the
    source has changed since it was taken."""
    here = os.path.dirname(os.path.abspath(__file__))
    csrc = os.path.join(here, "paper_1909_10547_b300", "csrc")
    srcs = ({"k_tc": ["k_tc.cu"], "k_tc_dense": ["k_tc.cu"], "k_stream": ["k_cc.cu"], "k_fac": ["k_cc.cu"]}.get(kernel) or
            sorted(f for f in os.listdir(csrc) if f.endswith(".cu")))
    h = hashlib.sha256()
    for src in srcs:
        with open(os.path.join(csrc, src), "rb") as f:
            h.update(f.read())
    sha = h.hexdigest()[:16]
    try:
        lines = open(os.path.join(here, "profiles", "dram_traffic.txt")).read().splitlines()
    except OSError:
        return None
    for ln in lines:
        w = ln.split()
        if len(w) >= 6 and not ln.startswith("#") and w[:5] == [kernel, sha, prec, str(ndata), str(replicas)]:
            return float(w[5])
    return None


# The paper's Table 3 (Sec. 3) times this product; its fastest line at
# ndata = 2000, K = 35721, R = 2000 is TensorFlow on a GPU in 1.38 s including
# the transfer to the device: 2000 * 2000 / 1.38 s datapoint*replicas/s.
TABLE3_LAST = {"ndata": 2000, "R": 2000, "seconds": 1.38}


def run_dense(args):
    """The dense product of the paper's timing study: the Table 3 base table
    (49 flavour combinations x 27 x points, K = 35721) flattened to
    [ndata][K] times the PDF matrix [K][R] built on the device from R
    replicas.  `value`: the product alone, timed over graph replays with the
    PDF matrix resident; `e2e`: per step the PDF matrix is copied from pinned
    host memory and O copied back (the table stays resident)."""
    import torch
    import paper_1909_10547_b300 as fk
    from paper_1909_10547_b300 import workloads as W
    R = args.replicas or 2000
    nd = args.ndata
    prec = args.prec
    f64 = prec in ("fp64", "fp64tc")
    io = torch.float64 if f64 else torch.float32
    if args.kdense:
        K = args.kdense
        tab = fk.Table.dense(np.random.default_rng(K).standard_normal((nd, K)), precs=(prec,))
        L = torch.rand((R, K), dtype=io, device="cuda")
    else:
        t, F = W.table3(nd, R)
        K = t.fk[0].size
        ht = fk.Table.from_workload(t, precs=("fp64" if f64 else "fp32",))
        tab = fk.Table.dense(t.fk.reshape(nd, K), precs=(prec,))
        del t
        Fd = torch.tensor(F, dtype=io, device="cuda")
        L = fk.luminosity(ht, Fd, "fp64" if f64 else "fp32")
    O = fk.dense_conv(tab, L, prec)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        fk.dense_conv(tab, L, prec, out=O)
    for _ in range(max(3, args.warmup)):
        g.replay()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.cudart().cudaProfilerStart()
    with Clocks(torch.cuda.current_device()) as clk:
        e0.record()
        for _ in range(args.steps):
            g.replay()
        e1.record()
        torch.cuda.synchronize()
    torch.cuda.cudart().cudaProfilerStop()
    ms = e0.elapsed_time(e1) / args.steps
    # end to end: the PDF matrix from pinned host memory, O back to the host
    Lh = L.cpu().pin_memory()
    Oh = torch.empty(O.shape, dtype=io).pin_memory()
    for _ in range(2):
        L.copy_(Lh, non_blocking=True)
        fk.dense_conv(tab, L, prec, out=O)
        Oh.copy_(O, non_blocking=True)
    torch.cuda.synchronize()
    e2, e3 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e2.record()
    for _ in range(args.steps):
        L.copy_(Lh, non_blocking=True)
        fk.dense_conv(tab, L, prec, out=O)
        Oh.copy_(O, non_blocking=True)
    e3.record()
    torch.cuda.synchronize()
    ms_e2e = e2.elapsed_time(e3) / args.steps
    flops = 2.0 * nd * K * R
    byts = nd * K * ESZ[prec]
    pk, src = peaks()
    tc = prec in ("bf16", "bf16x3", "tf32")
    tpeak, _ = peak_of(prec, pk)
    ridge = tpeak * 1e12 / (pk["hbm_gbs"] * 1e9)
    kern = "k_tc" if tc else ("k_stream" if R <= 4 else "k_tile")
    if flops / byts < ridge:
        ach = byts / (ms * 1e-3) / 1e9
        roof = {"bound": "hbm", "achieved": ach, "peak": pk["hbm_gbs"], "unit": "GB/s",
                "frac": ach / pk["hbm_gbs"], "algorithmic_bytes": byts}
    else:
        ach = flops / (ms * 1e-3) / 1e12
        roof = {"bound": "tensor" if tc else "alu", "achieved": ach, "peak": tpeak, "unit": "TFLOP/s",
                "frac": ach / tpeak, "algorithmic_flops": flops}
    roof.update({"traffic": traffic_of("k_tc_dense", prec, nd, R) if tc else None, "peak_source": src,
                 "kernel": f"{kern} (timed as the whole product call, operand packing included)"})
    value = nd * R / (ms * 1e-3)
    exact = nd == TABLE3_LAST["ndata"] and R == TABLE3_LAST["R"]
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak",
            "vs_baseline": value / (TABLE3_LAST["ndata"] * TABLE3_LAST["R"] / TABLE3_LAST["seconds"]) if exact else None,
            "dtype": prec, "data": "synthetic",
            "config": {"workload": f"dense product of the paper's Table 3: FK [{nd} x {K}] . PDF matrix "
                                   f"[{K} x {R}] (49 flavour combinations x 27 x points)",
                       "l2": "table larger than L2" if byts > 126e6 else "table fits in L2 (warm: replayed back to back)",
                       "graphs": True,
                       "baseline": "paper Table 3, TensorFlow GPU 1.38 s incl. transfer (other hardware)" if exact else None},
            "roofline": roof,
            "e2e": {"value": nd * R / (ms_e2e * 1e-3), "unit": UNIT,
                    "h2d_bytes_per_step": int(L.numel() * L.element_size()),
                    "d2h_bytes_per_step": int(O.numel() * O.element_size())},
            "clocks": clk.summary()}
    print(json.dumps(line), flush=True)


def run_stress(args):
    """One convolution of the stress table, timed over graph replays: the
    kernel-level roofline (HBM for the streaming path at small R, tensor pipe
    for the tcgen05 path at large R)."""
    import torch
    import paper_1909_10547_b300 as fk
    from paper_1909_10547_b300 import workloads as W
    R = args.replicas or 1
    if args.table == "config1":
        t, F = W.config1(R=R)
        args.ndata = t.ndata
        name = f"plain hadronic table (configs 1-2) 200 x 60 channels x 30 x 30, one convolution, R={R}"
    else:
        t = W.stress_table(ndata=args.ndata)
        x = W.xgrid(50, 1e-7)
        F = W.pdf_replicas(x, W.pdf_params(np.random.default_rng(1)), R, np.random.default_rng(2) if R > 1 else None)
        name = f"hadronic stress table {args.ndata} x 196 channels x 50 x 50, one convolution, R={R}"
    lumi = args.form == "lumi" and args.prec in ("bf16", "bf16x3", "tf32")
    tab = fk.Table.from_workload(t, precs=(args.prec,), form="lumi" if lumi else None)
    if lumi:
        name += ", dense form (PDF matrix formed in shared memory)"
    dt = torch.float64 if args.prec in ("fp64", "fp64tc") else torch.float32
    Fd = torch.tensor(F, dtype=dt, device="cuda")
    O = fk.conv(tab, Fd, args.prec)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        fk.conv(tab, Fd, args.prec, out=O)
    for _ in range(max(3, args.warmup)):
        g.replay()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.cudart().cudaProfilerStart()
    with Clocks(torch.cuda.current_device()) as clk:
        e0.record()
        for _ in range(args.steps):
            g.replay()
        e1.record()
        torch.cuda.synchronize()
    torch.cuda.cudart().cudaProfilerStop()
    ms = e0.elapsed_time(e1) / args.steps
    elems = t.fk.size
    byts = elems * ESZ[args.prec]
    flops = 2.0 * elems * R
    tc = args.prec in ("bf16", "bf16x3", "tf32", "fp64tc")
    kern = ("k_oz_slice + k_tc digit pairs + k_oz_combine" if args.prec == "fp64tc" else
            "k_tc" if tc else ("k_stream" if R == 1 else "k_fac"))
    roof = roof_entry(args.prec, byts, flops, ms, f"{kern} (timed as the whole convolution call)",
                      traffic_of(kern, args.prec, args.ndata, R) if args.table == "stress" and args.prec != "fp64tc"
                      else None)
    line = {"metric": METRIC, "value": args.ndata * R / (ms * 1e-3), "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": args.prec, "data": "synthetic",
            "config": {"workload": name, "l2": "table larger than L2" if byts > 126e6 else
                       "table fits in L2 (warm: replayed back to back)", "graphs": True},
            "roofline": roof, "clocks": clk.summary()}
    print(json.dumps(line), flush=True)


def run_dis(args):
    """The DIS convolution of config 0 (64 data points, 9 of 14 flavours, 40 x
    points, one PDF), --stack copies of the table stacked along the data
    points, timed over graph replays (back to back)."""
    import torch
    import paper_1909_10547_b300 as fk
    from paper_1909_10547_b300 import workloads as W
    prec = args.prec
    R = args.replicas or 1
    t0, _ = W.config0()
    x = W.xgrid(40, 1e-7)
    rng = np.random.default_rng(5)
    F = W.pdf_replicas(x, W.pdf_params(rng), R, rng if R > 1 else None)
    comp = t0.compact()
    if args.stack > 1:
        comp = np.abs(np.random.default_rng(10547).standard_normal((args.stack * t0.ndata,) + comp.shape[1:])) * \
            (x ** 0.3)[None, None, :]
    tab = fk.Table.dis(comp, t0.flav, None, 40, precs=(prec,))
    nd = comp.shape[0]
    used = comp.size
    del comp
    dt = torch.float64 if prec in ("fp64", "fp64tc") else torch.float32
    Fd = torch.tensor(F, dtype=dt, device="cuda")
    O = torch.empty((R, nd), dtype=dt, device="cuda")
    ms = time_calls(lambda: fk.dis_conv(tab, Fd, prec, out=O), args.steps)
    roof = roof_entry(prec, used * ESZ[prec], 2.0 * used * R, ms, "DIS convolution call")
    line = {"metric": METRIC, "value": nd * R / (ms * 1e-3), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": prec, "data": "synthetic",
            "config": {"workload": f"DIS 64 x 9 x 40 (config 0) x {args.stack} stacked, R={R}", "graphs": True},
            "roofline": roof, "latency_us": ms * 1e3}
    print(json.dumps(line), flush=True)


def run_serve(args):
    """Served mixed workload: open-loop Poisson arrivals of convolution requests
    on the 40 global-set tables plus the stress table, replica counts from
    {1, 10, 100, 1000}, all tables resident, admission by a 150 GB budget.
    Latency is measured by the client from submit to the poll that sees the
    result; throughput is datapoint*replicas over first submit -> last
    completion.  The same requests are then run one at a time through the
    plain per-request path (H2D, fk_*_conv, D2H, synchronise) for comparison."""
    import threading
    import torch
    import paper_1909_10547_b300 as fk
    from paper_1909_10547_b300 import workloads as W
    g = workload()
    prec = args.prec
    tc = prec in ("bf16", "bf16x3", "tf32")
    tables = list(g.tables) + [W.stress_table()]
    tabs = [fk.Table.from_workload(t, precs=(prec,)) for t in tables]
    tprec = [prec for _ in tables]
    nxg = [t.nxg for t in tables]
    del tables
    srv = fk.Server(budget_bytes=150 << 30, max_inflight=8)
    ids = [srv.add_table(t) for t in tabs]
    rng = np.random.default_rng(SEED + 1)
    n = args.requests
    which = rng.integers(0, len(tabs), n)
    Rs = rng.choice(W.REPLICA_CHOICES, n)
    arr = W.arrivals(rng, args.rate, n)
    pool = {}  # a few PDF sets per (grid size, R), reused across requests
    for k in range(n):
        key = (nxg[which[k]], int(Rs[k]), tprec[which[k]])
        if key not in pool:
            x = g.x if key[0] == 50 else W.xgrid(key[0], 1e-7)
            F = W.pdf_replicas(x, g.params, key[1], np.random.default_rng(key[1]))
            pool[key] = F.astype(np.float64 if key[2] in ("fp64", "fp64tc") else np.float32)
    work = [(int(which[k]), pool[(nxg[which[k]], int(Rs[k]), tprec[which[k]])], tprec[which[k]]) for k in range(n)]
    units = sum(tabs[w].ndata * F.shape[0] for w, F, _ in work)

    # warm-up: every table once
    for k in range(len(tabs)):
        srv.wait(srv.submit(ids[k], pool[next(key for key in pool if key[0] == nxg[k] and key[2] == tprec[k])], tprec[k]))

    tickets = [None] * n
    t_sub = np.zeros(n)
    t_done = np.zeros(n)
    done_flag = [False]

    def poller():
        outstanding = set()
        nxt = 0
        deadline = time.perf_counter() + 300.0
        while nxt < n or outstanding:
            if time.perf_counter() > deadline:
                return  # done_flag stays False: reported below
            while nxt < n and tickets[nxt] is not None:
                outstanding.add(nxt)
                nxt += 1
            for k in list(outstanding):
                ok, _ = srv.poll(tickets[k])
                if ok:
                    t_done[k] = time.perf_counter()
                    outstanding.discard(k)
            time.sleep(0.0001)
        done_flag[0] = True

    th = threading.Thread(target=poller, daemon=True)
    th.start()
    t0 = time.perf_counter()
    for k, (w, F, p) in enumerate(work):
        delay = t0 + arr[k] - time.perf_counter()
        if delay > 0:
            time.sleep(delay)
        t_sub[k] = time.perf_counter()
        tickets[k] = srv.submit(ids[w], F, p)
    th.join()
    if not done_flag[0]:
        raise TimeoutError("served mix: requests unresolved after 300 s")
    lat = (t_done - t_sub) * 1e3
    span = t_done.max() - t_sub.min()
    st = srv.stats()
    # saturation: the same requests in a closed loop that keeps WINDOW of them
    # in flight (capacity of the server, independent of the arrival process)
    WINDOW = 64
    s0 = time.perf_counter()
    inflight = []
    for w, F, p in work:
        if len(inflight) >= WINDOW:
            srv.wait(inflight.pop(0), 120000)
        inflight.append(srv.submit(ids[w], F, p))
    for tk in inflight:
        srv.wait(tk, 120000)
    sat_span = time.perf_counter() - s0
    srv.close()

    # the plain per-request path, one request at a time, same requests
    stream = torch.cuda.current_stream()
    dev_cache = {}
    t1 = time.perf_counter()
    plain_lat = []
    for w, F, p in work:
        s0 = time.perf_counter()
        dt = torch.float64 if p in ("fp64", "fp64tc") else torch.float32
        Fd = torch.from_numpy(F).to("cuda", non_blocking=False)
        O = fk.conv(tabs[w], Fd, p)
        O.cpu()
        plain_lat.append((time.perf_counter() - s0) * 1e3)
    plain_span = time.perf_counter() - t1
    line = {"metric": METRIC, "value": units / sat_span, "unit": UNIT, "n_gpus": 1, "steps": n,
            "warmup": len(tabs), "ms_per_step": sat_span * 1e3 / n, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": prec, "data": "synthetic",
            "config": {"workload": f"served mix: {n} requests, Poisson {args.rate:g}/s, 40 global-set tables + "
                                   "stress table 2000 x 196 x 50 x 50 resident, R in {1,10,100,1000}, "
                                   "budget 150 GB", "max_inflight": 8,
                       "value": "saturation throughput (closed loop, 64 requests in flight)"},
            "serve": {"p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                      "max_ms": float(lat.max()), "offered_rate": args.rate,
                      "achieved_rate": n / span, "open_loop_value": units / span,
                      "launches": st["launches"], "peak_bytes": st["peak_bytes"]},
            "per_request_baseline": {"value": units / plain_span, "unit": UNIT,
                                     "p50_ms": float(np.percentile(plain_lat, 50)),
                                     "p99_ms": float(np.percentile(plain_lat, 99)),
                                     "what": "one request at a time: H2D, fk conv, D2H, synchronise"}}
    print(json.dumps(line), flush=True)


def run_descent(args):
    """Gradient descent on the PDF parameters of the R = 100 replicas over the
    global set: per iteration, parametrisation -> pipelined fit step ->
    parameter gradient -> Adam.  Replicas start from parameters jittered
    around the ones the pseudo-data were drawn from; reports iterations per
    second (as datapoint*replicas/s of the fit step they contain) and the
    chi^2/ndata of the replicas before and after."""
    import torch
    import paper_1909_10547_b300 as fk
    from paper_1909_10547_b300 import workloads as W
    from paper_1909_10547_b300.descent import PDFDescent
    from paper_1909_10547_b300.fitstep import GlobalFit
    g = workload()
    tabs64 = [fk.Table.from_workload(t, ("fp64",)) for t in g.tables]
    Ft = torch.tensor(g.F_true, device="cuda")
    o_true = [fk.conv(t, Ft, "fp64")[0].cpu().numpy() for t in tabs64]
    del tabs64
    cov = W.covariance(o_true, SEED)
    D = np.concatenate(W.pseudo_data(o_true, SEED))
    rng = np.random.default_rng(SEED + 2)
    t0 = np.empty((REPLICAS, 14, 3))
    t0[..., 0] = np.log(g.params.A)[None, :] + rng.uniform(-0.3, 0.3, (REPLICAS, 14))
    t0[..., 1] = g.params.alpha[None, :] * rng.uniform(0.8, 1.2, (REPLICAS, 14))
    t0[..., 2] = g.params.beta[None, :] * rng.uniform(0.8, 1.2, (REPLICAS, 14))
    fit = GlobalFit(g.tables, g.F, cov.blocks, D, prec=args.prec, nstreams=args.streams or None,
                    save_products=save_arg(args), whiten=whiten_arg(args))
    fit.capture()
    gd = PDFDescent(fit, t0, g.x, lr=0.02)
    for _ in range(max(3, args.warmup)):
        gd.step()
    gd.__init__(fit, t0, g.x, lr=0.02)  # restart from t0 after the warm-up
    torch.cuda.synchronize()
    gd.step()
    chi_first = fit.chi2.cpu().numpy().copy()
    iters = max(args.steps, 200)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with Clocks(torch.cuda.current_device()) as clk:
        e0.record()
        for _ in range(iters):
            gd.step()
        e1.record()
        torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / iters
    chi_last = fit.chi2.cpu().numpy()
    line = {"metric": METRIC, "value": fit.ntot * fit.R / (ms * 1e-3), "unit": UNIT, "n_gpus": 1,
            "steps": iters, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": args.prec, "data": "synthetic",
            "config": dict(config_dict(g, args.prec, sum(t.device_bytes() for t in fit.tabs)),
                           workload="gradient descent on the PDF parameters of "
                           "100 replicas over the global-shaped set (one fit step per iteration)",
                           optimizer="Adam, lr 0.02"),
            "descent": {"chi2_per_point_first_median": float(np.median(chi_first) / fit.ntot),
                        "chi2_per_point_last_median": float(np.median(chi_last) / fit.ntot),
                        "iterations_timed": iters + 1},
            "clocks": clk.summary()}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.watchdog_s > 0:
        faulthandler.dump_traceback_later(args.watchdog_s, exit=True)
    import torch
    if args.case == "stress":
        run_stress(args)
        return
    if args.case == "serve":
        run_serve(args)
        return
    if args.case == "descent":
        run_descent(args)
        return
    if args.case == "dense":
        run_dense(args)
        return
    if args.case == "peaks":
        run_peaks(args)
        return
    if args.case == "dis":
        run_dis(args)
        return
    rank, world, dist = dist_init(args.gpus)
    if args.impl == "reference":
        run_reference(args, rank, world, dist)
        if dist is not None:
            dist.destroy_process_group()
        return
    import paper_1909_10547_b300 as fk
    from paper_1909_10547_b300 import workloads as W
    from paper_1909_10547_b300.fitstep import GlobalFit

    dev = torch.cuda.current_device()
    g = workload()
    # pseudo-data: D = O(f_true) + correlated noise, O(f_true) from the FP64 path
    tabs64 = [fk.Table.from_workload(t, ("fp64",)) for t in g.tables]
    Ft = torch.tensor(g.F_true, device="cuda")
    o_true = [fk.conv(t, Ft, "fp64")[0].cpu().numpy() for t in tabs64]
    del tabs64
    cov = W.covariance(o_true, SEED)
    D = np.concatenate(W.pseudo_data(o_true, SEED))
    fit = GlobalFit(g.tables, g.F, cov.blocks, D, prec=args.prec, nstreams=args.streams or None,
                    pipelined=not args.phases, waves=args.waves, save_products=save_arg(args),
                    whiten=whiten_arg(args))
    stage("fit step set up (tables, whitening, saved-product buffers)")
    fit.capture()
    launches = fit.launches_per_step()
    stream = torch.cuda.current_stream()

    inner = max(1, args.inner)
    for _ in range(max(3, args.warmup) * inner):
        fit.step()
    torch.cuda.synchronize()
    names = list(fit.graphs)
    # a bench step is `inner` consecutive fit steps: events between the
    # graphs of the first fit step of each bench step give the per-graph split
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(len(names) + 2)] for _ in range(args.steps)]
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    # the timed region is also the profiler range (ncu --profile-from-start off)
    torch.cuda.cudart().cudaProfilerStart()
    with Clocks(dev) as clk:
        for k in range(args.steps):
            ev[k][0].record(stream)
            for i, n in enumerate(names):
                fit.graphs[n].replay()
                ev[k][i + 1].record(stream)
            for _ in range(inner - 1):
                fit.step()
            ev[k][-1].record(stream)
        torch.cuda.synchronize()
    torch.cuda.cudart().cudaProfilerStop()
    if dist is not None:
        dist.barrier()
    seg = {n: sum(ev[k][i].elapsed_time(ev[k][i + 1]) for k in range(args.steps)) / args.steps
           for i, n in enumerate(names)}
    ms = sum(ev[k][0].elapsed_time(ev[k][-1]) for k in range(args.steps)) / args.steps
    ms = max_over_ranks(dist, ms)
    fit_ms = ms / inner
    if len(names) == 1:
        seg = {names[0]: fit_ms}  # the pipelined step: the mean over all timed fit steps

    # end to end: per fit step, pinned host F in, chi2 and gF out, through the same calls
    F_host = torch.tensor(g.F, dtype=fit.io).pin_memory()
    chi2_host = torch.empty(fit.R, dtype=torch.float64).pin_memory()
    gF_host = torch.empty(fit.gF.shape, dtype=fit.io).pin_memory()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for _ in range(3):
        fit.F.copy_(F_host, non_blocking=True)
        fit.step()
        chi2_host.copy_(fit.chi2, non_blocking=True)
        gF_host.copy_(fit.gF, non_blocking=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(args.steps * inner):
        fit.F.copy_(F_host, non_blocking=True)
        fit.step()
        chi2_host.copy_(fit.chi2, non_blocking=True)
        gF_host.copy_(fit.gF, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_e2e = max_over_ranks(dist, e0.elapsed_time(e1) / args.steps)
    stage("fit step timed (device and end to end)")

    units = fit.ntot * fit.R * inner
    value = job_throughput(units, world, ms)
    roof = roofline(fit, seg, args.prec)
    roof["traffic"] = None
    roof["traffic_note"] = ("whole-step DRAM counters are not captured (one kernel at a time on small cases "
                            "only); per-kernel traffic is in the kernels block")

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": {"fp64": "f64", "fp32": "f32", "bf16": "bf16",
                                           "bf16x3": "bf16x3", "tf32": "tf32", "fp64tc": "f64 (bf16 digit slices)"}[args.prec],
            "data": "synthetic",
            "config": dict(config_dict(g, args.prec, sum(t.device_bytes() for t in fit.tabs)), streams=fit.nstreams,
                           schedule="per-phase" if args.phases else f"pipelined, {fit.waves} forward waves",
                           fit_steps_per_step=inner, ms_per_fit_step=fit_ms,
                           chi2=("whitened tables: L_k^-1 folded into each table and its data at set-up, "
                                 "chi^2 = |Z - Dw|^2 per step" if fit.whiten else
                                 "FP64 blocked substitutions per step"),
                           saved_products=f"{sum(b is not None for b in fit.saved)} of "
                                          f"{sum(k == 'had' for k in fit.kinds)} hadronic tables, "
                                          f"{sum(b.numel() * 4 for b in fit.saved if b is not None) / 1e6:.0f} MB "
                                          f"(--save {args.save})"),
            "roofline": roof,
            "e2e": {"value": job_throughput(units, world, ms_e2e), "unit": UNIT,
                    "h2d_bytes_per_step": inner * F_host.numel() * F_host.element_size(),
                    "d2h_bytes_per_step": inner * (chi2_host.numel() * 8 + gF_host.numel() * gF_host.element_size())},
            "gpu_launches": launches * args.steps * inner, "clocks": clk.summary()}
    if rank == 0 and world == 1 and not args.no_extras:
        # the served mixes first (the server's threads then meet a quiet
        # host), then the kernel-level lines
        from paper_1909_10547_b300 import workloads as W
        try:
            st = W.stress_table()
            stress_tab = fk.Table.from_workload(st, precs=("fp32", "bf16", "bf16x3"))
            stress_oz = fk.Table.from_workload(st, precs=("fp64tc",))
            # only the shape is needed from here on: the 7.8 GB host copy goes
            st = W.HadTable(np.empty((st.fk.shape[0], st.fk.shape[1], st.fk.shape[2], st.fk.shape[3]),
                                     dtype=np.uint8), st.ca, st.cb, st.xmap, st.nxg)
            # the global-set tables as they are (the fit's own are whitened)
            serve_tabs = fit.tabs if not fit.whiten else [fk.Table.from_workload(t, (args.prec,)) for t in g.tables]
            stage("serving block")
            line["serve"] = serve_block(args, g, serve_tabs, fit.tprec, stress_tab)
            del serve_tabs
            # FP64-contract serving: FP64 results on the tensor cores, served,
            # against the plain FP64 path one request at a time (global set)
            tabs64 = [fk.Table.from_workload(t, precs=("fp64", "fp64tc")) for t in g.tables]
            stage("FP64-contract serving block")
            line["serve_fp64"] = serve_block(args, g, tabs64, ["fp64tc"] * len(tabs64), None, n=400,
                                             plain_prec="fp64")
            del tabs64
            stage("kernel lines")
            line["kernels"] = kernel_lines(args, stress_tab, st, stress_oz)
            line["kernels"].append(chi2_line(args, cov, o_true, D))
            del st, stress_oz, stress_tab
            torch.cuda.synchronize()
        except Exception as exc:  # the headline stands; say what failed
            line["extras_error"] = f"{type(exc).__name__}: {exc}"
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        D_parts = np.split(D, np.cumsum([t.ndata for t in g.tables])[:-1])
        stage("CPU baseline (oracle)")
        cb = cpu_baseline(g, cov.blocks, D_parts)
        nr = cb["replicas"]
        line["cpu_baseline"] = {"value": cb["value"], "unit": UNIT, "cores": cb["cores"], "kind": "oracle",
                                "sample": f"{nr} of {REPLICAS} replicas, whole fit step (all 40 tables), FP64, "
                                          f"best of 5: {cb['seconds']:.2f} s",
                                "value_1core": cb["value_1core"],
                                "sample_1core": f"{cb['replicas_1core']} replica, one core, best of 3: "
                                                f"{cb['seconds_1core']:.2f} s"}
        fit.F.copy_(torch.tensor(g.F, dtype=fit.io))
        fit.step()
        torch.cuda.synchronize()
        chi = fit.chi2[:nr].cpu().numpy()
        gF = fit.gF[:nr].double().cpu().numpy()
        line["accuracy"] = {"reference": "FP64 oracle, same tables, covariance and pseudo-data",
                            "replicas_compared": nr, "mode": args.prec,
                            "chi2_max_rel_err": float(np.max(np.abs(chi / cb["chi2"] - 1))),
                            "grad_max_err_rel_to_max": float(np.abs(gF - cb["gF"]).max() / np.abs(cb["gF"]).max())}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
