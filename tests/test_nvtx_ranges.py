"""Every compute entry point of liblabs.so opens an NVTX range named after itself (for profiler timelines).

Checked on the CPU: an NVTX injection library (tests/support/nvtx_record.c, built here with gcc) records
the ranges pushed while a child process calls the entry points with a null context, which each rejects
after opening its range -- no GPU is touched.
"""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
LIB = os.path.join(ROOT, "paper_2409_07222_gb300", "liblabs.so")
CUDA_INCLUDE = "/usr/local/cuda/include"

CALLS = {
    "labs_energy_batch": "(None, None, 13, 0, None, None, None)",
    "labs_flip_deltas": "(None, None, None, 13, 0, 0, 0, None, None)",
    "labs_skew_search": "(None, None, None, 0, None, None, None, None)",
    "labs_batched_search": "(None, None, None, None, None, 0, None, None, None, None, None)",
    "labs_pq_refine": "(None, None, None, 0, None, None, None, None)",
    "labs_pq_independent": "(None, None, None, 0, None, None, None, None)",
    "labs_sequence_operators": "(None, None, 13, 0, None, None, None, None, None)",
    "labs_skew_exhaustive": "(None, 13, 0, 0, None, None, None, None, None)",
    "labs_policy_forward": "(None, None, 0, None, None)",
}


@pytest.mark.skipif(not os.path.exists(LIB), reason="liblabs.so is not built")
@pytest.mark.skipif(shutil.which("gcc") is None or not os.path.isdir(os.path.join(CUDA_INCLUDE, "nvtx3")),
                    reason="needs gcc and the NVTX headers")
def test_entry_points_open_named_ranges(tmp_path):
    rec = tmp_path / "libnvtx_record.so"
    subprocess.run(["gcc", "-shared", "-fPIC", "-O2", "-I" + CUDA_INCLUDE, "-o", str(rec),
                    os.path.join(ROOT, "tests", "support", "nvtx_record.c")], check=True)
    log = tmp_path / "nvtx.log"
    code = "from paper_2409_07222_gb300 import _lib\nlib = _lib.load()\n" + "".join(
        "assert lib.%s%s != 0\n" % (name, args) for name, args in CALLS.items())
    env = dict(os.environ, NVTX_INJECTION64_PATH=str(rec), LABS_NVTX_LOG=str(log), PYTHONPATH=ROOT)
    subprocess.run([sys.executable, "-c", code], check=True, env=env, cwd=ROOT, timeout=120)
    lines = log.read_text().split("\n")
    pushes = [l[5:] for l in lines if l.startswith("push ")]
    assert pushes == list(CALLS), pushes
    assert sum(1 for l in lines if l == "pop") == len(CALLS)
