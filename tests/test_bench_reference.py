"""The benchmark's reference arm on the host: `bench.py --impl reference` times
the FP64 oracle's step on a bounded sample and prints one JSON line with the
fields of the benchmark contract, without a GPU and without loading the CUDA
library.  The oracle's sample itself (minutes on the benchmark mesh) is
replaced here by fixed per-unit times, so that the line's arithmetic and
fields are checked on the host in seconds."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

_DRIVER = r"""
import json, sys
sys.path.insert(0, %r)
import bench
bench.oracle_sample = lambda krylov_tol=1e-10, t0=None: {
    "N": 775009, "build_s": 50.0, "t_block": 20.0, "t_sub": 30.0, "tau1": 0.02 / 200.0,
    "t_cg_it_col": 0.25, "cols": 16, "dt": 0.02, "wall_s": 120.0}
sys.argv = ["bench.py", "--impl", "reference", "--steps", "2", "--warmup", "3"]
bench.main()
maps = open("/proc/self/maps").read() if sys.platform.startswith("linux") else ""
print("LIBAFEM_MAPPED" if "libafem" in maps else "LIBAFEM_NOT_MAPPED")
"""


def test_reference_arm_prints_the_contract_line():
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="")
    r = subprocess.run([sys.executable, "-c", _DRIVER % ROOT], capture_output=True, text=True, env=env, cwd=ROOT,
                       timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads([ln for ln in r.stdout.splitlines() if ln.startswith("{")][-1])
    assert line["impl"] == "reference"
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["higher_is_better"] is True
    assert line["steps"] == 2 and line["warmup"] == 3
    # step = block + S substeps + cols x I iterations, S = dt / tau_1 = 200, I = the FP64 path's mean
    import bench
    t_step = 20.0 + 200.0 * 30.0 + 16 * bench.FP64_CG_ITERS_PER_STEP * 0.25
    assert abs(line["value"] - 1.0 / t_step) <= 1e-12 / t_step
    assert abs(line["ms_per_step"] - 1000.0 / line["value"]) <= 1e-9 * line["ms_per_step"]
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == 1 and cb["host_cores"] >= 1 and cb["value"] == line["value"]
    assert f"1 of {cb['host_cores']} host cores" in cb["sample"] and "N=775009" in cb["sample"]
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"], "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
    assert "LIBAFEM_NOT_MAPPED" in r.stdout
