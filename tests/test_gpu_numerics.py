"""Device arithmetic of the library checked against CUDA's own.  The flux,
wave-speed and Rusanov routines use rcp64 (float seed + cubic correction) in
place of 1.0 / x and sqrt64 (float inverse-square-root seed + cubic correction)
in place of sqrt(x): rcp64 must stay within one unit in the last place of CUDA's
correctly rounded 1.0 / x, sqrt64 within two of sqrt(x), and both must agree bit
for bit on the inputs they hand back to CUDA (zero, subnormal, out of range,
inf, NaN, negative for sqrt64).  d2f_trunc, the integer-pipe double -> float
conversion of the CFL screening values, must stay within one float ulp of
(float)x and never exceed |x|."""
import os
import shutil
import subprocess

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_device_math_against_cuda(cuda, tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    exe = tmp_path / "device_math_check"
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17",
                    "-I", os.path.join(ROOT, "paper_2409_12483_gb300", "csrc"),
                    "-o", str(exe), os.path.join(ROOT, "tests", "gpu_src", "device_math_check.cu")],
                   check=True, timeout=300)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr
    lines = {ln.split()[0]: dict(kv.split("=") for kv in ln.split()[1:]) for ln in r.stdout.splitlines()}
    assert int(lines["rcp64"]["maxulp"]) <= 1 and float(lines["rcp64"]["exact_fraction"]) > 0.999
    assert int(lines["sqrt64"]["maxulp"]) <= 2 and float(lines["sqrt64"]["exact_fraction"]) > 0.5
    assert int(lines["rcp64"]["special_mismatch"]) == 0 and int(lines["sqrt64"]["special_mismatch"]) == 0
    assert int(lines["d2f_trunc"]["bad"]) == 0
