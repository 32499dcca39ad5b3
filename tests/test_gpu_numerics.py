"""Device arithmetic of the library checked against CUDA's own: the FP64
reciprocal rcp64 (float seed + cubic correction), which the flux, wave-speed and
Rusanov routines use in place of 1.0 / x, must stay within one unit in the last
place of CUDA's correctly rounded 1.0 / x and agree bit for bit on the inputs it
hands back to 1.0 / x (zero, subnormal, out of range, inf, NaN)."""
import os
import shutil
import subprocess

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_rcp64_within_one_ulp_of_cuda_division(cuda, tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    exe = tmp_path / "rcp64_check"
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17",
                    "-I", os.path.join(ROOT, "paper_2409_12483_gb300", "csrc"),
                    "-o", str(exe), os.path.join(ROOT, "tests", "gpu_src", "rcp64_check.cu")],
                   check=True, timeout=300)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr
    fields = dict(kv.split("=") for kv in r.stdout.split())
    assert int(fields["maxulp"]) <= 1
    assert int(fields["special_mismatch"]) == 0
    assert float(fields["exact_fraction"]) > 0.999
