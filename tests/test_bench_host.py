"""Host-side logic of bench.py, on CPU: the replica aggregation at world size 2 over gloo, the
reference arm's JSON line (rank 0 only under a multi-rank launch), the roofline object of the
dominant kernel, the oracle extrapolation and the per-phase rates."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _replica_worker(rank, ws, port, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    # rank r did (r + 1) * 100 band-applies in (r + 1) * 2 s
    rate, t_max = bench.whole_job_rate(100.0 * (rank + 1), 2.0 * (rank + 1), ws)
    mx = bench.max_over_ranks(float(rank), ws)
    sm = bench.sum_over_ranks(float(rank + 1), ws)
    with open(os.path.join(out_dir, f"r{rank}.json"), "w") as f:
        json.dump({"rate": rate, "t_max": t_max, "max": mx, "sum": sm}, f)
    dist.barrier()
    dist.destroy_process_group()


def test_replica_aggregation_world_size_2_gloo(tmp_path):
    import torch.multiprocessing as mp
    ws = 2
    mp.spawn(_replica_worker, args=(ws, _free_port(), str(tmp_path)), nprocs=ws, join=True)
    res = [json.load(open(tmp_path / f"r{r}.json")) for r in range(ws)]
    for r in res:
        # whole job: (100 + 200) applies over the slowest rank's 4 s
        assert r["rate"] == pytest.approx(75.0)
        assert r["t_max"] == pytest.approx(4.0)
        assert r["max"] == 1.0 and r["sum"] == 3.0


def test_single_rank_aggregation_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.whole_job_rate(300.0, 1.5, 1) == (200.0, 1.5)
    assert bench.dist_init(1) == (0, 1)


def _run_reference(env_extra):
    env = dict(os.environ)
    env.update(env_extra)
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                           "--workload", "gamma24", "--steps", "1", "--warmup", "0"],
                          capture_output=True, text=True, env=env, timeout=600, cwd=ROOT)


def test_reference_arm_prints_one_contract_line():
    p = _run_reference({"RANK": "0", "WORLD_SIZE": "1"})
    assert p.returncode == 0, p.stderr
    lines = [ln for ln in p.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference"
    assert d["value"] > 0 and d["higher_is_better"] is False and d["unit"] == "s"
    assert d["config"]["workload"] == "gamma24"
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["value"] == d["value"] and d["e2e"]["unit"] == d["unit"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0


def test_reference_arm_other_ranks_exit_quietly():
    p = _run_reference({"RANK": "1", "WORLD_SIZE": "2"})
    assert p.returncode == 0, p.stderr
    assert p.stdout.strip() == ""


def _phases(**ms):
    names = ("fft", "nonlocal", "gram", "constraint", "rr", "update")
    return {p: float(ms.get(p, 0.0)) for p in names}


def test_roofline_reports_the_dominant_kernel():
    sys.path.insert(0, ROOT)
    import bench
    kr = {"fp64class_gemm": {"kernel": "k", "shape": [1, 2, 3], "bound": "tensor", "unit": "TFLOP/s",
                             "ms": 2.0, "achieved": 40.0, "peak": 80.0, "frac": 0.5, "work_per_launch": "x",
                             "peak_source": "MEASURED_PEAKS.json bf16_tflops"},
          "fft_c64": {"error": "boom"}}
    roof = bench.roofline_of(kr, "fp64class_gemm")
    assert roof["bound"] == "tensor" and roof["frac"] == 0.5 and roof["achieved"] == 40.0
    assert roof["traffic"] is None and "of measured" in roof["peak_source"]
    bad = bench.roofline_of(kr, "fft_c64")
    assert bad["frac"] is None and bad["error"] == "boom"


def test_oracle_extrapolation_counts_every_block_visit():
    sys.path.insert(0, ROOT)
    import bench
    import synth
    w = synth.make_workload("gamma120")
    # 9 sweeps x (1024 + 128) / 128 blocks x 1 k-point visits of 20 s
    assert bench.oracle_s_to_tol(w, 20.0, 128) == pytest.approx(9 * 9 * 20.0)
    w4 = synth.make_workload("mp72x10")
    assert bench.oracle_s_to_tol(w4, 1.0, 64) == pytest.approx(6 * 3 * 10)
    assert bench.nbuf_of(w, -1) == 128 and bench.nbuf_of(w, 0) == 0


def test_phase_rates_split_native_fp64_from_the_rest():
    sys.path.insert(0, ROOT)
    import bench
    ms = _phases(fft=50.0, gram=20.0, rr=10.0)
    ms64 = _phases(gram=5.0, rr=10.0)
    fl = _phases(fft=1e12, gram=4e12, rr=1e10)
    fl64 = _phases(gram=1e11, rr=1e10)
    by = _phases(fft=120e9, gram=1e9)
    by64 = _phases(gram=0.5e9)
    out = bench.phase_rates(ms, ms64, fl, fl64, by, by64, 2)
    assert set(out) == {"fft/other", "gram/other", "gram/fp64", "rr/fp64"}
    assert out["fft/other"]["gbs"] == pytest.approx(120e9 / 0.05 / 1e9)
    assert out["fft/other"]["ms_per_step"] == 25.0
    assert out["gram/other"]["tflops"] == pytest.approx((4e12 - 1e11) / 0.015 / 1e12)
    assert out["gram/fp64"]["gbs"] == pytest.approx(0.5e9 / 0.005 / 1e9)
    assert out["rr/fp64"]["tflops"] == pytest.approx(1e10 / 0.01 / 1e12)


def test_kernel_rooflines_never_raise():
    """Without a GPU each side measurement reports its error instead of raising, so a failed
    kernel timing cannot cost the bench line."""
    sys.path.insert(0, ROOT)
    import bench
    import synth
    import torch
    if torch.cuda.is_available():
        pytest.skip("CPU-only check")
    out = bench.kernel_rooflines(synth.make_workload("gamma24"), 925, 16, {"hbm_gbs": 1.0, "bf16_tflops": 1.0})
    assert set(out) == {"fp64class_gemm", "fp64class_gemm_df32", "gram_3xtf32", "update_3xtf32", "fft_c64"}
    assert all("error" in v for v in out.values())
    assert bench.roofline_of(out)["frac"] is None


def test_roofline_traffic_only_at_the_captured_shape():
    sys.path.insert(0, ROOT)
    import bench
    entry = {"kernel": "k_tc_nn<128>", "bound": "tensor", "unit": "TFLOP/s", "ms": 0.33, "achieved": 267.0,
             "peak": 924.0, "frac": 0.29, "work_per_launch": "x", "peak_source": "MEASURED_PEAKS.json bf16_tflops"}
    at = bench.roofline_of({"update_3xtf32": dict(entry, shape=[113081, 128, 256])}, "update_3xtf32")
    assert at["traffic"] == bench.TRAFFIC[("update_3xtf32", (113081, 128, 256))][0]
    assert at["traffic_source"].startswith("profiles/")
    other = bench.roofline_of({"update_3xtf32": dict(entry, shape=[57925, 64, 128])}, "update_3xtf32")
    assert other["traffic"] is None
    assert bench.DOMINANT in ("update_3xtf32", "fp64class_gemm", "gram_3xtf32", "fft_c64")
