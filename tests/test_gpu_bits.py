"""The step kernels' integer-only binary32 <-> binary64 conversions agree bit for bit with
the hardware conversions on normal values, zeros, subnormals, Inf and overflow
(binary64 -> binary32 rounds toward zero; magnitudes below the binary32 normal range
become signed zero, by design); NaN stays NaN. The FP32-force form's bit-split binary64
state (binary32 truncation + the 29 dropped mantissa bits) rebuilds every binary64 in
[2^-126, 2^128) exactly, holds smaller magnitudes as signed zero and reports the rest as
out of range."""
import os
import subprocess

import pytest

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


def test_conversions_match_hardware(tmp_path):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    exe = str(tmp_path / "conv_check")
    subprocess.check_call(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17",
                           "-o", exe, os.path.join(HERE, "conv_check.cu")])
    r = subprocess.run([exe], capture_output=True, text=True)
    print(r.stdout)
    assert r.returncode == 0, r.stdout + r.stderr
