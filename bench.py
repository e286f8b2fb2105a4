"""Benchmark of the GB300 block-LOBPCG plane-wave eigensolver.

Workload (default): the 120^3 Gamma-point cell -- a = 25 bohr, 113081 plane
waves, 108 Gaussian atoms on a jittered fcc lattice with 432 Kleinman-Bylander
projectors, 1024 bands in blocks of 128 plus one block of buffer bands,
nline = 4 (seeded synthetic inputs, no pseudopotential data).  This is the
cell on which the mixed-precision schedule is compared with the FP64 path
and the FP64 oracle.

One step = one full ``lobpcg_solve`` from the same seeded start block until
every one of the 1024 bands has an FP64 residual <= 1e-8 Ha (mixed
FP32/FP64 schedule).  ``value`` is the seconds to 1e-8 Ha (lower is better);
``ms_per_step`` the same in ms.  The line also carries the eigenvalue error
against the oracle's golden eigenvalues of the cell, the standalone
``apply_H`` throughput (band-applies/s, the metric's second quantity), the
CUDA-event roofline of the dominant kernel, the per-phase device times, the
CPU-oracle baseline and the SM clocks seen during the timed region.  The
FP64-only solve of the same problem (``--fp64``; on by default for the cells
where it takes under a minute) gives the mixed-vs-FP64 comparison.

Multi-GPU: a workload with several k-points is sharded -- each rank solves its
own k-points (Sec. 5.2), the eigenvalues are gathered once at the end -- and
the line reports the slowest rank's time ("strong" scaling: the total work is
fixed).  A single-k-point workload runs one replica per rank ("weak").

``--impl reference`` times the CPU FP64 oracle on the same workload and metric
(a bounded sample, extrapolated to a full solve as its ``sample`` states).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "LOBPCG s to 1e-8 Ha residual, mixed vs FP64 on GB300; H·psi band-applies/s"
UNIT = "s"
RATE_UNIT = "band-applies/s"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
FP64_PEAK_TFLOPS = 1.25          # GB300 FP64 (CUDA cores), nominal per GPU
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12   # SMs x FP32 lanes x FMA x max SM clock = 80.5
FALLBACK = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="gamma120")
    ap.add_argument("--precision", default="mixed", choices=["fp64", "mixed"])
    ap.add_argument("--nbuf", type=int, default=-1, help="buffer bands above the wanted ones (-1: one block)")
    ap.add_argument("--tol", type=float, default=1e-8)
    ap.add_argument("--max-sweeps", type=int, default=60)
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64-only comparison solve")
    ap.add_argument("--fp64", action="store_true",
                    help="run the FP64-only comparison solve also on cells where it takes minutes")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-gamma-real", action="store_true",
                    help="skip the Gamma-point real-orbital solve of a Gamma cell (reported beside the headline)")
    ap.add_argument("--ncu", action="store_true",
                    help="profiling run: only the warm-up and timed steps of --mode, no other legs")
    ap.add_argument("--mode", default="sweep", choices=["sweep", "solve", "apply", "apply_df32", "fp64gemm", "tf32gemm"],
                    help="with --ncu: LOBPCG sweeps, full solves to --tol, standalone apply_H, the "
                         "double-FP32 apply_H of the FP64-class H X, or the FP64-class tensor-core A B "
                         "(npw x nb x nb; nb = --nb, default the solve's band count)")
    ap.add_argument("--nb", type=int, default=0, help="with --ncu and an apply mode: bands (0 = all)")
    return ap.parse_args()


def ncu_run(args):
    """Minimal launch sequence for ncu captures: build the handle, then
    warm-up + timed steps of one kind (prints a short JSON line, not a bench value)."""
    import torch
    import paper_0707_3405_gb300 as lg
    import __graft_entry__
    __graft_entry__.build()
    w = make(args.workload)
    nbuf = nbuf_of(w, args.nbuf)
    if args.mode == "fp64gemm":
        lg.load()
        import dataclasses
        s0 = solver_for(dataclasses.replace(w, proj_E=np.zeros(0), kpts=w.kpts[:1]), "mixed")
        M = s0.npw(0)
        s0.close()
        nb = args.nb if args.nb > 0 else w.nbands + nbuf
        g = torch.Generator(device="cuda")
        g.manual_seed(3)
        A = torch.randn((nb, M), dtype=torch.complex128, device="cuda", generator=g)
        B = torch.randn((nb, nb), dtype=torch.complex128, device="cuda", generator=g)
        D = torch.empty((nb, M), dtype=torch.complex128, device="cuda")
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.warmup + args.steps):
            lg.gemm_nn(A, B, D=D, tc=True)
        torch.cuda.synchronize()
        lg.check_timeouts()
        print(json.dumps({"ncu_run": True, "mode": args.mode, "shape": [M, nb, nb], "launches": lg.launch_count(),
                          "s": time.perf_counter() - t0}))
        return 0
    if args.mode == "tf32gemm":
        # the 3xTF32 A B of a block update at the bench shape (npw x m x 2m, complex64)
        lg.load()
        import dataclasses
        s0 = solver_for(dataclasses.replace(w, proj_E=np.zeros(0), kpts=w.kpts[:1]), "mixed")
        M = s0.npw(0)
        s0.close()
        m = w.block
        A = torch.randn((2 * m, M), dtype=torch.complex64, device="cuda")
        B = torch.randn((m, 2 * m), dtype=torch.complex64, device="cuda")
        D = torch.empty((m, M), dtype=torch.complex64, device="cuda")
        lg.set_gemm_mode(0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.warmup + args.steps):
            lg.gemm_nn(A, B, D=D)
        torch.cuda.synchronize()
        lg.check_timeouts()
        print(json.dumps({"ncu_run": True, "mode": args.mode, "shape": [M, m, 2 * m], "launches": lg.launch_count(),
                          "s": time.perf_counter() - t0}))
        return 0
    if args.mode == "solve":
        s = solver_for(w, args.precision, timing=False, max_sweeps=args.max_sweeps, tol=args.tol, nbuf=nbuf)
    else:
        s = solver_for(w, args.precision, timing=False, max_sweeps=1, tol=1e-30, nbuf=nbuf)
    X = start_block(w, s)
    if args.mode.startswith("apply") and args.nb > 0:
        X = X[:args.nb].contiguous()
    if args.mode == "apply" and args.precision == "mixed":
        X = X.to(torch.complex64)
    Y = torch.empty_like(X)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.warmup + args.steps):
        if args.mode in ("sweep", "solve"):
            s.solve([X.clone()] if args.mode == "solve" else [X])
        else:
            s.apply_H(0, X, Y, df32=args.mode == "apply_df32")
    torch.cuda.synchronize()
    print(json.dumps({"ncu_run": True, "mode": args.mode, "precision": args.precision, "workload": w.name,
                      "launches": lg.launch_count(), "s": time.perf_counter() - t0}))
    s.close()
    return 0


def peaks():
    try:
        with open(PEAKS_FILE) as f:
            p = json.load(f)
        return p, "measured"
    except Exception:
        return dict(FALLBACK), "fallback"


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ workload
GOLDEN_DIR = os.path.join(ROOT, "tests", "golden")
# Sweeps the FP64 schedule (the same Algorithm 1 sweeps as the oracle's) needs to 1e-8 Ha from
# the seeded start with one block of buffer bands, measured on the GB300; the reference arm
# scales its sampled block visit to a full solve with it.
SWEEPS_TO_TOL = {"gamma24": 12, "k96": 7, "gamma120": 9, "mp72x10": 6, "large160": 9}


def make(workload: str):
    import synth
    return synth.make_workload(workload)


def nbuf_of(w, nbuf_arg):
    return w.block if nbuf_arg < 0 else nbuf_arg


def solver_for(w, precision, timing=False, max_sweeps=1, tol=1e-8, nbuf=0, autotune=False, use_graph=False,
               kidx=None, gamma_real=False):
    """A library handle for the k-points ``kidx`` of workload ``w`` (all when None)."""
    import dataclasses
    import paper_0707_3405_gb300 as lg
    ks = list(range(w.nk)) if kidx is None else list(kidx)
    wl = dataclasses.replace(w, kpts=w.kpts[ks])
    return lg.Solver(wl.a, wl.N, wl.ecut, wl.kpts, wl.vloc(), wl.proj_E if wl.nproj else None,
                     beta=(lambda mil, k: wl.beta(mil, k)) if wl.nproj else None, block_size=w.block,
                     nline=w.nline, max_sweeps=max_sweeps, precision=precision, tol=tol, timing=timing,
                     nbuf=nbuf, autotune=autotune, use_graph=use_graph, gamma_real=gamma_real)


def start_block(w, s, k=0, device=True, pinned=False, kglobal=None):
    """Seeded start vectors of k-point ``k`` of handle ``s`` (``kglobal``: its index in the workload)."""
    import torch
    x = torch.from_numpy(np.ascontiguousarray(w.x0(s.npw(k), k if kglobal is None else kglobal).T))
    if device:
        return x.cuda()
    return x.pin_memory() if pinned else x


def golden_eigs(w):
    """{k: eigenvalues} from the oracle goldens of this workload (tests/golden, written by
    tests/golden/make_golden.py from the oracle); empty when none is stored."""
    out = {}
    names = {"gamma24": {0: "gamma24_eig.txt"}, "k96": {0: "k96_eig.txt"}, "gamma120": {0: "gamma120_eig.txt"},
             "mp72x10": {k: f"mp72x10_k{k}_eig.txt" for k in range(10)}}.get(w.name, {})
    for k, f in names.items():
        path = os.path.join(GOLDEN_DIR, f)
        if os.path.exists(path):
            out[k] = np.loadtxt(path)
    return out


# ------------------------------------------------------------------ oracle (CPU) sample
def oracle_setup(w):
    """The oracle's Hamiltonian of the first k-point and its first start block (set-up, untimed,
    like the library's create)."""
    from oracle import hamiltonian
    H = hamiltonian.for_workload(w)
    return H, w.x0(H.npw, 0, w.block)


def oracle_sample(w, seconds_target=15.0, setup=None):
    """Bounded sample of the oracle's own solve of the same cell: visits of the first block
    (block start + nline Algorithm 1 iterations on m bands, H applications included), repeated
    until about ``seconds_target`` of CPU work.  Returns (seconds per block visit, elapsed, visits)."""
    from oracle import lobpcg as olob
    H, X0 = setup if setup is not None else oracle_setup(w)
    t0 = time.perf_counter()
    reps = 0
    while True:
        olob.block_lobpcg(H, X0, H.T, None, nline=w.nline)
        reps += 1
        el = time.perf_counter() - t0
        if el >= seconds_target or reps >= 50:
            break
    return el / reps, el, reps


def oracle_s_to_tol(w, t_visit, nbuf):
    """The oracle's seconds to 1e-8 Ha extrapolated from its block-visit time: sweeps x blocks
    (wanted + buffer) x k-points visits.  It leaves out the constraint against earlier blocks and
    the all-band Rayleigh-Ritz step, so it is a lower bound of the oracle's time."""
    nblk = (w.nbands + nbuf) // w.block
    return SWEEPS_TO_TOL.get(w.name, 10) * nblk * w.nk * t_visit


def cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


# ------------------------------------------------------------------ distributed
def dist_init(n):
    if n <= 1 or "RANK" not in os.environ:
        return 0, 1
    import torch
    import torch.distributed as dist
    dist.init_process_group("nccl")
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
    return dist.get_rank(), dist.get_world_size()


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def _all_reduce(x, ws, op):
    """One float reduced over the ranks (on the GPU under NCCL, on the host under gloo)."""
    if ws <= 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=op)
    return float(t.item())


def max_over_ranks(x, ws):
    import torch.distributed as dist
    return _all_reduce(x, ws, dist.ReduceOp.MAX) if ws > 1 else x


def sum_over_ranks(x, ws):
    import torch.distributed as dist
    return _all_reduce(x, ws, dist.ReduceOp.SUM) if ws > 1 else x


def whole_job_rate(units, seconds, ws):
    """Replicas: every rank solves its own copy of the workload, so the whole-job rate is the
    units of all ranks over the slowest rank's time. Returns (rate, slowest time)."""
    t_max = max_over_ranks(seconds, ws)
    return sum_over_ranks(units, ws) / t_max, t_max


# ------------------------------------------------------------------ reference arm
def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    w = make(args.workload)
    nbuf = nbuf_of(w, args.nbuf)
    per_step = max(4.0, 40.0 / max(1, args.steps + args.warmup))
    setup = oracle_setup(w)
    H, X0 = setup
    for _ in range(args.warmup):       # warm-up: one H application to a few bands of the block
        H.apply(X0[:, :min(8, X0.shape[1])])
    vals, els, visits = [], [], 0
    for _ in range(args.steps):
        tv, el, reps = oracle_sample(w, per_step, setup)
        vals.append(oracle_s_to_tol(w, tv, nbuf))
        els.append(el)
        visits += reps
    value = float(np.mean(vals))
    sample = (f"oracle block LOBPCG on the same cell: visits of the first block ({w.block} bands, block start + "
              f"{w.nline} Algorithm 1 iterations), at least one per step, {visits} visits in {sum(els):.1f} s "
              f"(the oracle's H built once before them); extrapolated to a full solve "
              f"as {SWEEPS_TO_TOL.get(w.name, 10)} sweeps x {(w.nbands + nbuf) // w.block} blocks x {w.nk} k-points "
              f"visits (constraint and all-band Rayleigh-Ritz left out: a lower bound)")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * value,
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "c128/f64",
        "data": "synthetic", "config": config_of(w, H.npw, nbuf, args, 1),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cpu_cores(), "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def config_of(w, npw, nbuf, args, ws, sharded=False):
    return {"workload": w.name, "a_bohr": w.a, "N": w.N, "npw": npw, "nk": w.nk,
            "kpts": [list(map(float, k)) for k in w.kpts], "natoms": len(w.pos), "nproj": w.nproj,
            "nbands": w.nbands, "block": w.block, "nbuf": nbuf, "nline": w.nline, "precision": args.precision,
            "tol_Ha": args.tol, "step": f"one lobpcg_solve to max residual <= {args.tol:g} Ha from the same start",
            "l2": "inputs larger than L2 (the start block alone is "
                  f"{16 * (npw or 0) * w.nbands / 1e6:.0f} MB per k-point)",
            "parallelism": (f"k-points sharded over {ws} ranks" if sharded else f"replicas x{ws}")}


# ------------------------------------------------------------------ our arm
def phase_rates(ph_ms, ph_ms64, ph_fl, ph_fl64, ph_by, ph_by64, steps):
    """Algorithmic rates of every (phase, arithmetic) segment of the library's phase timers.

    ``fp64`` is native FP64 arithmetic.  ``other`` mixes, per phase, the FP32 work (register
    FFTs, 3xTF32 tensor-core and CUDA-core GEMMs) and the FP64-class work done on the FP32 units
    or the tensor cores, so no single ceiling applies to it; the kernel rooflines are measured
    apart.  Rates are useful flops and algorithmic DRAM bytes over event time."""
    out = {}
    for p in ph_ms:
        for prec in ("other", "fp64"):
            t_ms = ph_ms64[p] if prec == "fp64" else ph_ms[p] - ph_ms64[p]
            fl = ph_fl64[p] if prec == "fp64" else ph_fl[p] - ph_fl64[p]
            by = ph_by64[p] if prec == "fp64" else ph_by[p] - ph_by64[p]
            if t_ms <= 0.0 or (fl <= 0.0 and by <= 0.0):
                continue
            t = t_ms / 1e3
            out[f"{p}/{prec}"] = {"ms_per_step": t_ms / max(1, steps), "tflops": fl / t / 1e12,
                                  "gbs": by / t / 1e9}
    return out


# FP32 instruction rate: SMs x FP32 lanes x max SM clock; a double-FP32 complex multiply-add
# costs about 48 FP32 instructions (split operands, TwoProd by FMA, TwoSum accumulation)
FP32_INSTR_PER_S = 152 * 128 * 2.07e9
DF32_INSTR_PER_CMAC = 48.0
TF32_PER_BF16 = 1.1 / 2.25        # nominal dense TF32 / BF16 tensor rates
OZ_PAIRS = 21                     # digit-slice products per real product of the FP64-class tensor-core GEMM
# Dominant kernel of the mixed solve on the benchmark cell (launch list in profiles/): the 3xTF32
# A B of the block updates, k_tc_nn<128> (14% of device time), timed here at a block update's
# shape; the FP64-class tensor GEMMs (22% as a family) are reported beside it under kernels.
DOMINANT = "update_3xtf32"


def _event_time(fn, reps, stream):
    """Mean seconds per call of ``fn`` by CUDA events on ``stream`` (2 warm-up calls)."""
    import torch
    for _ in range(2):
        fn()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(reps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / 1e3 / reps


def kernel_rooflines(w, npw, nbands, pk, reps=3):
    """CUDA-event timings of the kernels the solve is made of, standalone at the solve's shapes
    on operands larger than L2, each against its own ceiling:

    * ``fp64class_gemm``: the FP64-class A B of the sweep-end rotation X C (npw x nbands x
      nbands, complex128) on the tensor cores, the engine the mixed schedule uses: BF16 tensor
      flops (21 digit-slice products per real product) against the measured BF16 rate; beside it
      ``fp64class_gemm_df32``, the double-FP32 CUDA-core engine at the same shape;
    * ``gram_3xtf32``: the 3xTF32 tensor-core A^H B Gram of a block's [R W P] (3m x 3m x npw,
      complex64), tensor flops 3 x 8 m n K against the TF32 rate (measured BF16 x 1.1 / 2.25);
    * ``update_3xtf32``: the 3xTF32 A B of a block's update P = [W P] C (npw x m x 2m, complex64),
      the same flop count and ceiling;
    * ``fft_c64``: the FP32 FFT passes A, B, C of H psi for one block (m bands) on a handle of the
      same cell without projectors, algorithmic bytes (half box written, read + written, read;
      sphere in and out, kinetic table; V once per band batch) against the HBM copy rate.

    Each entry: shape, ms per call, achieved, peak, frac.  Failures are recorded, never raised."""
    import torch
    import paper_0707_3405_gb300 as lg
    out = {}
    try:
        stream = torch.cuda.current_stream()
    except Exception as e:  # no device: every entry records the error
        return {k: {"error": f"{type(e).__name__}: {e}"}
                for k in ("fp64class_gemm", "fp64class_gemm_df32", "gram_3xtf32", "update_3xtf32", "fft_c64")}
    hbm = pk.get("hbm_gbs", FALLBACK["hbm_gbs"])
    tf32 = pk.get("bf16_tflops", FALLBACK["bf16_tflops"]) * TF32_PER_BF16
    m = w.block
    try:
        g = torch.Generator(device="cuda")
        g.manual_seed(1234)
        M, n, k = npw, nbands, nbands
        A = torch.randn((k, M), dtype=torch.complex128, device="cuda", generator=g)
        B = torch.randn((n, k), dtype=torch.complex128, device="cuda", generator=g)
        D = torch.empty((n, M), dtype=torch.complex128, device="cuda")
        t = _event_time(lambda: lg.gemm_nn(A, B, D=D, tc=True), reps, stream)
        fl = 8.0 * M * n * k
        tfl = OZ_PAIRS * fl
        bf16 = pk.get("bf16_tflops", FALLBACK["bf16_tflops"])
        out["fp64class_gemm"] = {
            "kernel": "k_oz_split + k_oz_mma<1>", "shape": [M, n, k], "bound": "tensor", "unit": "TFLOP/s",
            "ms": t * 1e3, "achieved": tfl / t / 1e12, "peak": bf16, "frac": tfl / t / 1e12 / bf16,
            "fp64class_tflops": fl / t / 1e12,
            "work_per_launch": f"{tfl:.4g} BF16 tensor flops ({OZ_PAIRS} digit-slice products x 8 M n k)",
            "peak_source": "MEASURED_PEAKS.json bf16_tflops"}
        t_df = _event_time(lambda: lg.gemm_nn(A, B, D=D, df32=True), 2, stream)
        peak_df = FP32_INSTR_PER_S / DF32_INSTR_PER_CMAC * 8.0 / 1e12
        out["fp64class_gemm_df32"] = {
            "kernel": "k_gemm_df<0,0,4>", "shape": [M, n, k], "bound": "alu", "unit": "TFLOP/s", "ms": t_df * 1e3,
            "achieved": fl / t_df / 1e12, "peak": peak_df, "frac": fl / t_df / 1e12 / peak_df,
            "work_per_launch": f"{fl:.4g} FP64-class flops (8 M n k)",
            "peak_source": "152 SMs x 128 FP32 lanes x 2.07 GHz / 48 FP32 instructions per complex multiply-add"}
        del A, B, D
    except Exception as e:  # a failed side measurement must not cost the bench line
        out["fp64class_gemm"] = {"error": f"{type(e).__name__}: {e}"}
    try:
        m3 = 3 * m
        A = torch.randn((m3, npw), dtype=torch.complex64, device="cuda")
        B = torch.randn((m3, npw), dtype=torch.complex64, device="cuda")
        C = torch.empty((m3, m3), dtype=torch.complex64, device="cuda")
        lg.set_gemm_mode(0)
        t = _event_time(lambda: lg.gemm_cn(A, B, C=C), max(reps, 5), stream)
        fl = 3.0 * 8.0 * m3 * m3 * npw
        out["gram_3xtf32"] = {
            "kernel": "k_tc_cn + k_tc_reduce", "shape": [m3, m3, npw], "bound": "tensor", "unit": "TFLOP/s",
            "ms": t * 1e3, "achieved": fl / t / 1e12, "peak": tf32, "frac": fl / t / 1e12 / tf32,
            "work_per_launch": f"{fl:.4g} tensor flops (3 x 8 m n K)",
            "peak_source": "MEASURED_PEAKS.json bf16_tflops x nominal TF32/BF16 ratio 1.1/2.25"}
        del A, B, C
    except Exception as e:
        out["gram_3xtf32"] = {"error": f"{type(e).__name__}: {e}"}
    try:
        k2 = 2 * m
        A = torch.randn((k2, npw), dtype=torch.complex64, device="cuda")
        B = torch.randn((m, k2), dtype=torch.complex64, device="cuda")
        D = torch.empty((m, npw), dtype=torch.complex64, device="cuda")
        lg.set_gemm_mode(0)
        t = _event_time(lambda: lg.gemm_nn(A, B, D=D), max(reps, 5), stream)
        fl = 3.0 * 8.0 * npw * m * k2
        out["update_3xtf32"] = {
            "kernel": f"k_tc_nn<{128 if m > 64 else 64}>", "shape": [npw, m, k2], "bound": "tensor",
            "unit": "TFLOP/s", "ms": t * 1e3, "achieved": fl / t / 1e12, "peak": tf32, "frac": fl / t / 1e12 / tf32,
            "work_per_launch": f"{fl:.4g} tensor flops (3 x 8 M n k)",
            "peak_source": "MEASURED_PEAKS.json bf16_tflops x nominal TF32/BF16 ratio 1.1/2.25"}
        del A, B, D
    except Exception as e:
        out["update_3xtf32"] = {"error": f"{type(e).__name__}: {e}"}
    try:
        import dataclasses
        wl = dataclasses.replace(w, proj_E=np.zeros(0), kpts=w.kpts[:1])
        s = solver_for(wl, "mixed")
        try:
            X = torch.randn((m, s.npw(0)), dtype=torch.complex64, device="cuda")
            Y = torch.empty_like(X)
            t = _event_time(lambda: s.apply_H(0, X, Y), max(reps, 5), stream)
            mil = s.gvectors(0)
            px = int(mil[:, 0].max() - mil[:, 0].min() + 1)
            by = m * (4.0 * 8 * px * w.N * w.N + 3.0 * 8 * s.npw(0) + 4.0 * s.npw(0)) + 4.0 * w.N ** 3
            out["fft_c64"] = {
                "kernel": f"k_ra<{w.N}> + k_rb<{w.N}> + k_rc<{w.N}>", "shape": [m, s.npw(0), w.N], "bound": "hbm",
                "unit": "GB/s", "ms": t * 1e3, "achieved": by / t / 1e9, "peak": hbm, "frac": by / t / 1e9 / hbm,
                "band_applies_per_s": m / t, "work_per_launch": f"{by:.4g} algorithmic bytes",
                "peak_source": "MEASURED_PEAKS.json hbm_gbs"}
        finally:
            s.close()
    except Exception as e:
        out["fft_c64"] = {"error": f"{type(e).__name__}: {e}"}
    return out


# DRAM bytes per launch (read + write) from one ncu capture, by kernel entry and shape; valid only
# while the kernel is unchanged since the capture (the summary names the command).
TRAFFIC = {("fp64class_gemm", (113081, 1152, 1152)): (1.905e10, "profiles/fp64class_tensor_gemm_traffic_gamma120.md"),
           ("update_3xtf32", (113081, 128, 256)): (3.16e8, "profiles/tc_nn_3xtf32_update_gamma120.md")}


def roofline_of(kr, dominant=DOMINANT):
    """The contract's roofline object: the dominant kernel's CUDA-event rate against its peak."""
    d = kr.get(dominant, {})
    if "achieved" not in d:
        return {"bound": None, "achieved": None, "peak": None, "unit": None, "frac": None, "traffic": None,
                "kernel": dominant, "error": d.get("error", "not measured")}
    traffic, tsrc = TRAFFIC.get((dominant, tuple(d["shape"])), (None, None))
    return {"bound": d["bound"], "achieved": d["achieved"], "peak": d["peak"], "unit": d["unit"],
            "frac": d["frac"], "traffic": traffic, "traffic_source": tsrc, "kernel": d["kernel"], "shape": d["shape"],
            "work_per_launch": d["work_per_launch"], "peak_source": d["peak_source"] + " (of measured)"
            if "MEASURED" in d["peak_source"] else d["peak_source"]}


def run_fp64_default(w):
    """Whether the FP64-only comparison solve runs without --fp64: only where it takes under a minute."""
    return w.name in ("gamma24", "k96", "mp72x10")


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.ncu:
        return ncu_run(args)
    import torch
    import paper_0707_3405_gb300 as lg
    from paper_0707_3405_gb300 import kshard
    import __graft_entry__
    rank, ws = dist_init(args.gpus)
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
    if rank == 0:
        __graft_entry__.build()
    barrier(ws)
    lg.load()
    w = make(args.workload)
    nbuf = nbuf_of(w, args.nbuf)
    pk, pk_kind = peaks()
    sharded = w.nk > 1 and ws > 1
    if sharded and ws > w.nk:
        raise SystemExit(f"{w.name} has {w.nk} k-points: k-point sharding runs on at most {w.nk} ranks")
    mine = kshard.partition(w.nk, ws)[rank] if sharded else list(range(w.nk))

    # the autotuner runs in the first warm-up solve (its time is reported apart)
    s = solver_for(w, args.precision, timing=False, max_sweeps=args.max_sweeps, tol=args.tol, nbuf=nbuf,
                   autotune=True, use_graph=True, kidx=mine)
    npw = s.npw(0)
    X0 = [start_block(w, s, i, kglobal=k) for i, k in enumerate(mine)]
    X = [torch.empty_like(x) for x in X0]
    stream = torch.cuda.current_stream()

    def step():
        for xb, x0 in zip(X, X0):
            xb.copy_(x0)
        return s.solve(X)

    ms_autotune = 0.0
    for _ in range(max(args.warmup, 3)):
        ms_autotune += step().stats.get("ms_autotune", 0.0)
    torch.cuda.synchronize()
    barrier(ws)
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    l0 = lg.launch_count()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    sweeps, converged, maxres, applies = [], True, 0.0, 0
    for _ in range(args.steps):
        r = step()
        sweeps.append(r.stats["sweeps"])
        converged = converged and r.status == 0
        maxres = max(maxres, float(r.resid.max()))
        applies += r.stats["band_applies_fp64"] + r.stats["band_applies_fp32"]
    e1.record(stream)
    torch.cuda.synchronize()
    launches = lg.launch_count() - l0
    clk = clocks.stop()
    t = e0.elapsed_time(e1) / 1e3
    barrier(ws)
    t_max = max_over_ranks(t, ws)
    s_to_tol = t_max / args.steps
    local = {k: (r.eig[i], r.resid[i]) for i, k in enumerate(mine)}
    if sharded:
        eig_all, res_all = kshard.gather_results(local, w.nk, ws)
    else:
        eig_all, res_all = r.eig, r.resid
    eig_main = eig_all.copy()
    gold = golden_eigs(w)
    eig_err = None
    if gold:
        eig_err = {f"k{k}": float(np.abs(eig_main[k][:len(v)] - v[:w.nbands]).max()) for k, v in gold.items()
                   if k < eig_main.shape[0]}

    # per-phase device times of one more solve with the library's CUDA-event phase timers
    s.set_options(block_size=w.block, nline=w.nline, max_sweeps=args.max_sweeps, precision=args.precision,
                  tol=args.tol, timing=True, nbuf=nbuf)
    rp = step()
    st = rp.stats
    phases = {p: st["ph_ms"][p] for p in lg.PHASES}
    prl = phase_rates(st["ph_ms"], st["ph_ms_fp64"], st["ph_flops"], st["ph_fp64_flops"], st["ph_bytes"],
                      st["ph_bytes_fp64"], 1)
    s.set_options(block_size=w.block, nline=w.nline, max_sweeps=args.max_sweeps, precision=args.precision,
                  tol=args.tol, timing=False, nbuf=nbuf, use_graph=True)

    # end to end through the same public call: start vectors in pinned host memory
    # (the host buffers are filled before the clock starts: the solve overwrites them with the
    # result, and refilling them is a host-to-host copy of the caller's, not part of the call)
    Xh = [x.cpu().pin_memory() for x in X0]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    s.solve(Xh)
    t_e2e = max_over_ranks(time.perf_counter() - t0, ws)
    nb_bytes = sum(16 * s.npw(i) * w.nbands for i in range(len(mine)))
    e2e = {"value": t_e2e, "unit": UNIT, "h2d_bytes_per_step": nb_bytes,
           "d2h_bytes_per_step": nb_bytes + 16 * w.nbands * len(mine)}

    # standalone apply_H throughput (the metric's band-applies/s), all bands of the first k-point
    applyh = {}
    for dt, name, df in ((torch.complex128, "c128", False), (torch.complex64, "c64", False),
                         (torch.complex128, "c128_df32", True)):
        Xa = X0[0].to(dt)
        Ya = torch.empty_like(Xa)
        ta = _event_time(lambda: s.apply_H(0, Xa, Ya, df32=df), 3, stream)
        applyh[f"{name}_band_applies_per_s"] = w.nbands / ta
        del Xa, Ya
    s.close()
    kroof = kernel_rooflines(w, npw, w.nbands + nbuf, pk)
    roof = roofline_of(kroof)

    # Gamma-point real-orbital form (options.gamma_real) of the same solve, on Gamma cells
    gamma_real = None
    if not sharded and w.nk == 1 and not np.any(w.kpts[0]) and not args.no_gamma_real:
        s3 = solver_for(w, args.precision, timing=False, max_sweeps=args.max_sweeps, tol=args.tol, nbuf=nbuf,
                        use_graph=True, gamma_real=True)
        X3 = X0[0].clone()
        for rep in range(2):   # the first solve is a warm-up
            X3.copy_(X0[0])
            torch.cuda.synchronize()
            g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            g0.record(stream)
            r3 = s3.solve([X3])
            g1.record(stream)
            torch.cuda.synchronize()
        el = g0.elapsed_time(g1) / 1e3
        gamma_real = {"s_to_tol": el, "sweeps": r3.stats["sweeps"], "converged": bool(r3.status == 0),
                      "max_resid": float(r3.resid.max()),
                      "max_eig_diff_vs_complex_Ha": float(np.abs(r3.eig[0] - eig_main[0]).max()),
                      "speedup_vs_complex": s_to_tol / el}
        if gold and 0 in gold:
            gamma_real["eig_err_vs_oracle_golden_Ha"] = float(np.abs(r3.eig[0][:len(gold[0])] -
                                                                   gold[0][:w.nbands]).max())
        s3.close()

    # the FP64-only path on the same problem from the same start
    fp64 = None
    if not args.no_fp64 and args.precision != "fp64" and (args.fp64 or run_fp64_default(w)):
        s2 = solver_for(w, "fp64", timing=False, max_sweeps=args.max_sweeps, tol=args.tol, nbuf=nbuf, kidx=mine)
        X2 = [x.clone() for x in X0]
        torch.cuda.synchronize()
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        r2 = s2.solve(X2)
        f1.record(stream)
        torch.cuda.synchronize()
        el = max_over_ranks(f0.elapsed_time(f1) / 1e3, ws)
        loc2 = {k: (r2.eig[i], r2.resid[i]) for i, k in enumerate(mine)}
        e2, _ = kshard.gather_results(loc2, w.nk, ws) if sharded else (r2.eig, r2.resid)
        fp64 = {"s_to_tol": el, "sweeps": r2.stats["sweeps"], "converged": bool(r2.status == 0),
                "max_resid": float(r2.resid.max()),
                "max_eig_diff_vs_mixed_Ha": float(np.abs(e2 - eig_main).max()),
                "speedup_mixed_vs_fp64": el / s_to_tol}
        s2.close()

    cpu = None
    if rank == 0 and not args.no_cpu:
        tv, el, reps = oracle_sample(w, 15.0)
        est = oracle_s_to_tol(w, tv, nbuf)
        cpu = {"value": est, "unit": UNIT, "cores": cpu_cores(), "kind": "oracle",
               "sample": f"oracle block LOBPCG on the same cell: {reps} visits of the first block ({w.block} bands, "
                         f"block start + {w.nline} Algorithm 1 iterations) in {el:.1f} s, extrapolated to "
                         f"{SWEEPS_TO_TOL.get(w.name, 10)} sweeps x {(w.nbands + nbuf) // w.block} blocks x {w.nk} "
                         f"k-points (a lower bound of the oracle's solve)"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": s_to_tol, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": max(args.warmup, 3), "ms_per_step": 1e3 * s_to_tol, "higher_is_better": False,
            "scaling": "strong" if sharded else "weak", "vs_baseline": None,
            "dtype": "c128/f64" if args.precision == "fp64" else "c64/f32 + c128/f64",
            "data": "synthetic",
            "config": config_of(w, npw, nbuf, args, ws, sharded),
            "sweeps": sweeps, "converged": converged, "max_resid_Ha": maxres,
            "eig_err_vs_oracle_golden_Ha": eig_err,
            "band_applies_per_s_in_solve": applies / max(1e-9, t),
            "gpu_launches": launches,
            "clocks": clk,
            "roofline": roof,
            "kernels": kroof,
            "e2e": e2e,
            "cpu_baseline": cpu,
            "apply_H": applyh,
            "autotune_ms_first_solve": ms_autotune,
            "fp64_path": fp64,
            "gamma_real_form": gamma_real,
            "phases_ms_per_solve": phases,
            "phase_rates": prl,
        }
        print(json.dumps(line))
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
