"""Benchmark of the GB300 block-LOBPCG plane-wave eigensolver.

Workload (default): the 96^3 cell -- a = 20 bohr, 57925 plane waves at
k = (1/4, 1/4, 1/4), 64 Gaussian atoms on a jittered rock-salt lattice with
256 Kleinman-Bylander projectors, 256 bands in blocks of 64, nline = 4,
complex128 (seeded synthetic inputs, no pseudopotential data).

One step = one LOBPCG sweep (every block visited for nline iterations of
Algorithm 1 with the block constraint, closed by the all-band Rayleigh-Ritz
step and FP64 residuals), through ``lobpcg_solve`` with max_sweeps = 1.
``value`` is H psi band-applies per second over the timed sweeps.  The JSON
line also carries the time to a 1e-8 Ha residual of the FP64 and the mixed
schedules (full solves from the same start), the standalone ``apply_H``
throughput, the roofline of the dominant phase, the CPU-oracle baseline and
the SM clocks seen during the timed region.

``--impl reference`` times the CPU FP64 oracle on the same workload and metric
(bounded samples on the host cores).
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
UNIT = "band-applies/s"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
FP64_PEAK_TFLOPS = 1.25          # GB300 FP64 (CUDA cores), nominal per GPU
FALLBACK = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="k96")
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed"])
    ap.add_argument("--no-ttt", action="store_true", help="skip the time-to-tolerance solves")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--ttt-max-sweeps", type=int, default=120)
    ap.add_argument("--ncu", action="store_true",
                    help="profiling run: only the warm-up and timed steps of --mode, no other legs")
    ap.add_argument("--mode", default="sweep", choices=["sweep", "apply"],
                    help="with --ncu: time LOBPCG sweeps or standalone apply_H on all bands")
    return ap.parse_args()


def ncu_run(args):
    """Minimal launch sequence for ncu captures: build the handle, then
    warm-up + timed steps of one kind (prints a short JSON line, not a bench value)."""
    import torch
    import paper_0707_3405_gb300 as lg
    import __graft_entry__
    __graft_entry__.build()
    w = make(args.workload)
    s = solver_for(w, args.precision, timing=False, max_sweeps=1, tol=1e-30)
    X = start_block(w, s)
    if args.mode == "apply" and args.precision == "mixed":
        X = X.to(torch.complex64)
    Y = torch.empty_like(X)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.warmup + args.steps):
        if args.mode == "sweep":
            s.solve([X])
        else:
            s.apply_H(0, X, Y)
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
def make(workload: str):
    import synth
    return synth.make_workload(workload)


def solver_for(w, precision, timing=False, max_sweeps=1, tol=1e-8):
    import paper_0707_3405_gb300 as lg
    return lg.Solver(w.a, w.N, w.ecut, w.kpts, w.vloc(), w.proj_E if w.nproj else None,
                     beta=(lambda mil, k: w.beta(mil, k)) if w.nproj else None, block_size=w.block,
                     nline=w.nline, max_sweeps=max_sweeps, precision=precision, tol=tol, timing=timing)


def start_block(w, s, k=0, device=True, pinned=False):
    import torch
    x = torch.from_numpy(np.ascontiguousarray(w.x0(s.npw(k), k).T))
    if device:
        return x.cuda()
    return x.pin_memory() if pinned else x


# ------------------------------------------------------------------ oracle (CPU) sample
def oracle_sample(w, seconds_target=15.0):
    """Oracle band-applies/s inside its own LOBPCG iteration on the same cell:
    first block (m bands), one Algorithm 1 iteration (H X and H W, Gram,
    Rayleigh-Ritz, update), repeated until about `seconds_target` of CPU work."""
    from oracle import hamiltonian, lobpcg as olob
    H = hamiltonian.for_workload(w)
    X0 = w.x0(H.npw, 0, w.block)
    applies, t0 = 0, time.perf_counter()
    reps = 0
    while True:
        olob.block_lobpcg(H, X0, H.T, None, nline=1)
        applies += 2 * w.block
        reps += 1
        el = time.perf_counter() - t0
        if el >= seconds_target or reps >= 50:
            break
    return applies / el, el, reps


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


def max_over_ranks(x, ws):
    if ws <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x, ws):
    if ws <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda")
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


# ------------------------------------------------------------------ reference arm
def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    w = make(args.workload)
    per_step = max(4.0, 40.0 / max(1, args.steps + args.warmup))
    for _ in range(args.warmup):
        oracle_sample(w, per_step / 2)
    vals, els = [], []
    for _ in range(args.steps):
        v, el, _ = oracle_sample(w, per_step)
        vals.append(v)
        els.append(el)
    value = float(np.mean(vals))
    sample = (f"oracle block LOBPCG, first block of {w.block} bands, one Algorithm 1 iteration "
              f"(2 x {w.block} band-applies + Gram + RR + update) repeated for ~{per_step:.0f} s per step")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * float(np.mean(els)),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c128/f64",
        "data": "synthetic", "config": {"workload": w.name, "a_bohr": w.a, "N": w.N, "nbands": w.nbands,
                                         "block": w.block, "nproj": w.nproj},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cpu_cores(), "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


# ------------------------------------------------------------------ our arm
def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.ncu:
        return ncu_run(args)
    import torch
    import paper_0707_3405_gb300 as lg
    import __graft_entry__
    rank, ws = dist_init(args.gpus)
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
    if rank == 0:
        __graft_entry__.build()
    barrier(ws)
    lg.load()
    w = make(args.workload)
    pk, pk_kind = peaks()

    s = solver_for(w, args.precision, timing=True, max_sweeps=1, tol=1e-30)
    npw = s.npw(0)
    X = start_block(w, s)
    stream = torch.cuda.current_stream()

    def step(Xbuf):
        return s.solve([Xbuf])

    for _ in range(max(args.warmup, 3)):
        step(X)
    torch.cuda.synchronize()
    barrier(ws)
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    l0 = lg.launch_count()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    applies = 0
    ph_ms = {p: 0.0 for p in lg.PHASES}
    ph_fl = {p: 0.0 for p in lg.PHASES}
    ph_by = {p: 0.0 for p in lg.PHASES}
    ph_calls = {p: 0 for p in lg.PHASES}
    ph_f64 = {p: 0.0 for p in lg.PHASES}
    for _ in range(args.steps):
        r = step(X)
        st = r.stats
        applies += st["band_applies_fp64"] + st["band_applies_fp32"]
        for p in lg.PHASES:
            ph_ms[p] += st["ph_ms"][p]
            ph_fl[p] += st["ph_flops"][p]
            ph_by[p] += st["ph_bytes"][p]
            ph_calls[p] += st["ph_calls"][p]
            ph_f64[p] += st["ph_fp64_flops"][p]
    e1.record(stream)
    torch.cuda.synchronize()
    launches = lg.launch_count() - l0
    clk = clocks.stop()
    t = e0.elapsed_time(e1) / 1e3
    barrier(ws)
    t_max = max_over_ranks(t, ws)
    total_applies = sum_over_ranks(applies, ws)
    value = total_applies / t_max

    # roofline of the dominant phase (device time from the library's CUDA events)
    dom = max(ph_ms, key=lambda p: ph_ms[p])
    dom_s = ph_ms[dom] / 1e3
    if dom == "fft" and args.precision == "mixed":
        roof = {"bound": "hbm", "achieved": ph_by[dom] / dom_s / 1e9, "peak": pk["hbm_gbs"], "unit": "GB/s"}
    elif ph_f64[dom] >= 0.5 * ph_fl[dom]:
        roof = {"bound": "alu", "achieved": ph_fl[dom] / dom_s / 1e12, "peak": FP64_PEAK_TFLOPS,
                "unit": "TFLOP/s", "alu": "fp64"}
    else:
        roof = {"bound": "alu", "achieved": ph_fl[dom] / dom_s / 1e12, "peak": 74.0, "unit": "TFLOP/s",
                "alu": "fp32"}
    roof["frac"] = roof["achieved"] / roof["peak"]
    roof["traffic"] = None
    roof["phase"] = dom
    roof["phase_share"] = ph_ms[dom] / max(1e-9, sum(ph_ms.values()))
    roof["launches_per_step"] = ph_calls[dom] / max(1, args.steps)
    roof["peak_source"] = ("GB300 FP64 nominal 1.25 TFLOP/s (probe measured 1.185)" if roof.get("alu") == "fp64"
                           else ("GB300 FP32 FMA probe 74 TFLOP/s" if roof.get("alu") == "fp32"
                                 else f"MEASURED_PEAKS.json hbm_gbs ({pk_kind})"))

    # end to end through the same public call with pinned host buffers
    Xh = X.cpu().pin_memory()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        r = step(Xh)
    t_e2e = time.perf_counter() - t0
    e2e_applies = args.steps * (r.stats["band_applies_fp64"] + r.stats["band_applies_fp32"])
    t_e2e = max_over_ranks(t_e2e, ws)
    e2e = {"value": sum_over_ranks(e2e_applies, ws) / t_e2e, "unit": UNIT,
           "h2d_bytes_per_step": 16 * npw * w.nbands, "d2h_bytes_per_step": 16 * npw * w.nbands + 16 * w.nbands}

    # standalone apply_H throughput on all bands
    applyh = {}
    for dt, name in ((torch.complex128, "c128"), (torch.complex64, "c64")):
        Xa = X.to(dt)
        Ya = torch.empty_like(Xa)
        for _ in range(2):
            s.apply_H(0, Xa, Ya)
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        reps = 3
        for _ in range(reps):
            s.apply_H(0, Xa, Ya)
        a1.record(stream)
        torch.cuda.synchronize()
        applyh[f"{name}_band_applies_per_s"] = reps * w.nbands / (a0.elapsed_time(a1) / 1e3)
    s.close()

    # time to tolerance, FP64 vs mixed, from the same start
    ttt = None
    if not args.no_ttt:
        ttt = {"tol": 1e-8}
        for prec in ("mixed", "fp64"):
            s2 = solver_for(w, prec, timing=False, max_sweeps=args.ttt_max_sweeps, tol=1e-8)
            X2 = start_block(w, s2)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            r2 = s2.solve([X2])
            el = time.perf_counter() - t0
            ttt[f"{prec}_s"] = el
            ttt[f"{prec}_sweeps"] = r2.stats["sweeps"]
            ttt[f"{prec}_converged"] = bool(r2.status == 0)
            ttt[f"{prec}_max_resid"] = float(r2.resid.max())
            ttt[f"{prec}_band_applies"] = {"fp64": r2.stats["band_applies_fp64"], "fp32": r2.stats["band_applies_fp32"]}
            if prec == "mixed":
                eig_mixed = r2.eig.copy()
            else:
                ttt["max_eig_diff_mixed_vs_fp64_Ha"] = float(np.abs(r2.eig - eig_mixed).max())
            s2.close()
        ttt["speedup_mixed_vs_fp64"] = ttt["fp64_s"] / ttt["mixed_s"]

    cpu = None
    if rank == 0 and not args.no_cpu:
        v, el, reps = oracle_sample(w, 15.0)
        cpu = {"value": v, "unit": UNIT, "cores": cpu_cores(), "kind": "oracle",
               "sample": f"oracle block LOBPCG on the same cell: first block of {w.block} bands, one Algorithm 1 "
                         f"iteration (2 x {w.block} band-applies + Gram + RR + update) x {reps} in {el:.1f} s"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": max(args.warmup, 3), "ms_per_step": 1e3 * t_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "c128/f64" if args.precision == "fp64" else "mixed c64/f32 + c128/f64",
            "data": "synthetic",
            "config": {"workload": w.name, "a_bohr": w.a, "N": w.N, "npw": npw, "kpt": list(map(float, w.kpts[0])),
                       "natoms": len(w.pos), "nproj": w.nproj, "nbands": w.nbands, "block": w.block,
                       "nline": w.nline, "precision": args.precision, "step": "one LOBPCG sweep",
                       "l2": f"inputs larger than L2 (X is {16 * npw * w.nbands / 1e6:.0f} MB)",
                       "parallelism": f"replicas x{ws}"},
            "gpu_launches": launches,
            "clocks": clk,
            "roofline": roof,
            "e2e": e2e,
            "cpu_baseline": cpu,
            "apply_H": applyh,
            "time_to_tol": ttt,
            "phases_ms_per_step": {p: ph_ms[p] / args.steps for p in lg.PHASES},
        }
        print(json.dumps(line))
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
