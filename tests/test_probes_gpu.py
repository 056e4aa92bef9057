"""GPU probes of device helpers that the end-to-end parity tests only see
indirectly: the integer double <-> float conversions of the mixed path are
compared bit for bit with the hardware conversions, and the reciprocals of the
WENO7 weights with correctly rounded division."""
import os
import subprocess

import pytest

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def test_integer_conversions_match_hardware(tmp_path):
    exe = str(tmp_path / "convert_check")
    subprocess.run(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17",
                    "-I", os.path.join(ROOT, "paper_2203_12866_gb300", "csrc"),
                    os.path.join(HERE, "gpu_probes", "convert_check.cu"), "-o", exe], check=True)
    out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout.strip()
    assert out == f"mismatches 0 0 of {1 << 22}", out


def test_weno_reciprocals_against_division(tmp_path):
    exe = str(tmp_path / "rcp_check")
    subprocess.run(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17",
                    "-I", os.path.join(ROOT, "paper_2203_12866_gb300", "csrc"),
                    os.path.join(HERE, "gpu_probes", "rcp_check.cu"), "-o", exe], check=True)
    out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout.split()
    n, ulp_d, ulp_f = int(out[0]), int(out[1]), int(out[2])
    assert n == 1 << 22
    # two Newton steps from the SFU estimate: within a few ulp of 1/d
    assert ulp_d <= 4, ulp_d
    # the SFU float reciprocal: within 2 ulp of 1/f
    assert ulp_f <= 2, ulp_f
