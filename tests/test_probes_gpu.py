"""GPU probes of device helpers that the end-to-end parity tests only see
indirectly: the integer double <-> float conversions of the mixed path are
compared bit for bit with the hardware conversions, the reciprocals of the
WENO7 weights with correctly rounded division, and the bounded device-side wait
is made to run out (a barrier nothing completes) without faulting the GPU."""
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


def test_bounded_wait_gives_up_and_raises_abort(tmp_path):
    """Failure detection on the device without a fault: the stage kernels' bounded
    mbarrier wait on a barrier that nothing completes returns false after the wait
    limit (about 2 s of SM clocks) and sets the timeout bit that cosenu_sync reports
    as COSENU_ETIMEOUT; a second warp waiting elsewhere leaves on the abort flag
    before its own limit; the context stays usable."""
    exe = str(tmp_path / "wait_check")
    subprocess.run(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17",
                    "-I", os.path.join(ROOT, "paper_2203_12866_gb300", "csrc"),
                    os.path.join(HERE, "gpu_probes", "wait_check.cu"), "-o", exe], check=True)
    out = subprocess.run([exe], check=True, capture_output=True, text=True,
                         timeout=120).stdout.split()
    ok0, ok1, err, waited1, limit = (int(x) for x in out[:5])
    assert ok0 == 0 and ok1 == 0
    assert err == 2  # the timeout bit (kErrTimeout), nothing else
    assert 0 < waited1 < limit  # warp 1 left on the abort flag, before its own limit
    assert out[5] == "usable"


def test_fma_peaks(tmp_path):
    """Measured FMA throughput of the GPU (FP64 and FP32), the ALU peaks against
    which the FP64 stage kernels (and the instruction-bound mixed WENO7 kernels)
    are reported.  From the unit counts at 2.07 GHz: FP64 1.26 TFLOP/s (152 SMs x 2
    FP64 FMA lanes per clock x 2 flops), FP32 80.5 TFLOP/s (152 SMs x 128 lanes x 2)."""
    exe = str(tmp_path / "fma_peak")
    subprocess.run(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17",
                    os.path.join(HERE, "gpu_probes", "fma_peak.cu"), "-o", exe], check=True)
    out = subprocess.run([exe], check=True, capture_output=True, text=True,
                         timeout=120).stdout.split()
    fp64, fp32, sms = float(out[1]), float(out[3]), int(out[5])
    print(f"FMA peaks: fp64 {fp64:.3f} TFLOP/s, fp32 {fp32:.2f} TFLOP/s on {sms} SMs")
    assert 0.5 < fp64 < 2.0 and 30.0 < fp32 < 120.0
