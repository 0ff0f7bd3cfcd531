"""FP64 FMA issue rate of the GPU, the denominator of the FP64 ALU roofline.

The benchmark reports the SVD, the FP64 H_eff psi and the environment
updates against 152 SMs x 2 FP64 FMA per clock x 2.07 GHz.  This test
builds a clock64() probe and checks that the rate it sees with enough warps
in flight is 2 FMA lanes per clock per SM (16 cycles per warp-wide FMA per
SM, within 30 %), and prints the dependent-chain latency.
"""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.mark.gpu
def test_fp64_issue_rate(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    exe = tmp_path / "fp64_rate"
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-o", str(exe),
                    os.path.join(HERE, "gpu_probes", "fp64_rate.cu")], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    print(out)
    rates = {}
    for line in out.splitlines():
        if line.startswith("dfma 4 chains/thread"):
            warps = int(line.split(",")[1].split()[0])
            rates[warps] = float(line.split(":")[1].split()[0])
    assert 16 in rates
    assert 16.0 * 0.7 <= rates[16] <= 16.0 * 1.3
