"""The host-side tests catch plausible mistakes in the host logic around the library: the
k-point partition (Sec. 5.2), the bench's rate, extrapolation and roofline arithmetic, and the
binding's operand checks.  Each
case plants one mistake with the plugin tests/_oracle_mutant.py and runs the in-process tests
that pin that logic in a child process, which must end with a failed assertion."""
import json
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
KSHARD = ("tests/test_kshard.py", "partition")
BENCH = ("tests/test_bench_host.py", "not reference_arm and not replica")
BINDING = ("tests/test_binding_checks.py", "check")

# (name, module, text, planted replacement, (test file, -k expression))
HOST_MUTANTS = [
    ("partition_to_the_most_loaded_rank", "paper_0707_3405_gb300.kshard", "r = int(np.argmin(load))",
     "r = int(np.argmax(load))", KSHARD),
    ("partition_lightest_first", "paper_0707_3405_gb300.kshard", "key=lambda k: (-c[k], k))", "key=lambda k: (c[k], k))",
     KSHARD),
    ("partition_lists_unsorted", "paper_0707_3405_gb300.kshard", "return [sorted(x) for x in out]", "return out", KSHARD),
    ("phase_time_includes_the_fp64_part", "bench", 't_ms = ph_ms64[p] if prec == "fp64" else ph_ms[p] - ph_ms64[p]',
     't_ms = ph_ms64[p] if prec == "fp64" else ph_ms[p]', BENCH),
    ("phase_time_not_per_step", "bench", '"ms_per_step": t_ms / max(1, steps)', '"ms_per_step": t_ms', BENCH),
    ("oracle_extrapolation_drops_kpoints", "bench", "return SWEEPS_TO_TOL.get(w.name, 10) * nblk * w.nk * t_visit",
     "return SWEEPS_TO_TOL.get(w.name, 10) * nblk * t_visit", BENCH),
    ("oracle_extrapolation_drops_buffer_blocks", "bench", "nblk = (w.nbands + nbuf) // w.block",
     "nblk = w.nbands // w.block", BENCH),
    ("traffic_at_any_shape", "bench", 'TRAFFIC.get((dominant, tuple(d["shape"])), (None, None))',
     'TRAFFIC.get((dominant, (113081, 128, 256)), (None, None))', BENCH),
    ("binding_skips_the_residency_check", "paper_0707_3405_gb300", "    for name, t, _, _ in ops:\n        if not t.is_cuda:",
     "    for name, t, _, _ in ops[:0]:\n        if not t.is_cuda:", BINDING),
    ("binding_skips_the_plane_wave_count", "paper_0707_3405_gb300", "if x.ndim != 2 or x.shape[1] != npw:",
     "if x.ndim != 2:", BINDING),
    ("binding_skips_the_band_count", "paper_0707_3405_gb300", "        if any(x.shape[0] < M for x in X):",
     "        if False:", BINDING),
    ("binding_skips_the_output_shape", "paper_0707_3405_gb300",
     "elif not (isinstance(Y, np.ndarray) and Y.dtype == X.dtype and Y.shape == X.shape",
     "elif not (isinstance(Y, np.ndarray) and Y.dtype == X.dtype", BINDING),
]


def _run(case):
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    env.pop("ORACLE_MUTANT", None)
    if isinstance(case, tuple) and len(case) == 5:
        name, mod, old, new, (path, expr) = case
        env["ORACLE_MUTANT"] = json.dumps([mod, old, new])
    else:
        path, expr = case
    cmd = [sys.executable, "-m", "pytest", path, "-k", expr, "-x", "-q", "-rf", "-p", "tests._oracle_mutant"]
    p = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)
    return p.returncode, p.stdout + p.stderr


@pytest.fixture(scope="module")
def runs():
    cases = [KSHARD, BENCH, BINDING] + HOST_MUTANTS
    with ThreadPoolExecutor(max_workers=max(1, min(8, os.cpu_count() or 1))) as ex:
        out = list(ex.map(_run, cases))
    names = ["clean_kshard", "clean_bench", "clean_binding"] + [m[0] for m in HOST_MUTANTS]
    return dict(zip(names, out))


def test_every_planted_text_occurs_once():
    import importlib.util
    sys.path.insert(0, ROOT)
    for name, mod, old, new, _ in HOST_MUTANTS:
        with open(importlib.util.find_spec(mod).origin) as f:
            assert f.read().count(old) == 1, name


def test_host_tests_pass_as_they_are(runs):
    for key in ("clean_kshard", "clean_bench", "clean_binding"):
        rc, out = runs[key]
        assert rc == 0, out[-3000:]


@pytest.mark.parametrize("name", [m[0] for m in HOST_MUTANTS])
def test_host_tests_catch_the_planted_mistake(runs, name):
    rc, out = runs[name]
    assert rc == 1, out[-3000:]
    assert any(ln.startswith("FAILED") for ln in out.splitlines()), out[-3000:]
