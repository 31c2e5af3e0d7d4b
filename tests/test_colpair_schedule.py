"""Host check of the column-pair kernels' index logic (no GPU): compiles
tests/colpair_schedule_check.cu against the kernel header and runs it -- the
radix schedules, the digit-reversal maps, the partition of every pass into
groups, the shared-memory swizzles' freedom from bank conflicts and the
pair-table row permutation, for ny = 256 .. 4096."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")


@pytest.mark.skipif(not (os.path.exists(NVCC) or shutil.which("nvcc")), reason="needs nvcc")
def test_colpair_index_logic(tmp_path):
    exe = tmp_path / "colpair_schedule_check"
    src = os.path.join(HERE, "colpair_schedule_check.cu")
    subprocess.check_call([NVCC, "-std=c++17", "-gencode", "arch=compute_103a,code=sm_103a", "-o", str(exe), src])
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    assert out.returncode == 0 and out.stdout.strip().endswith("ok"), out.stdout
