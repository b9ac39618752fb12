"""The FP64 sweep takes its reciprocals and divisions from a Newton-Raphson
refinement of the hardware's approximate reciprocal (drcp_newton), not from
the IEEE division.  Here it is compared with CUDA's correctly rounded
1.0 / y on 16.7 M values spread over every binade from 2^-1000 to 2^1000
(both signs): at most 1 unit in the last place apart (measured: 0, every
value equal).  (The oracle parity
tests bound its effect on whole steps.)"""
import os
import subprocess

import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


def test_newton_reciprocal_within_one_ulp_of_ieee(tmp_path):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    exe = str(tmp_path / "rcp_check")
    src = os.path.join(HERE, "gpu_checks", "rcp_check.cu")
    subprocess.run([os.environ.get("NVCC", "nvcc"), "-gencode", "arch=compute_103a,code=sm_103a", "-O3",
                    "-std=c++17", "-o", exe, src], check=True)
    out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout.split()
    assert out[0] == "max_ulp" and int(out[3]) == 1 << 24
    assert int(out[1]) <= 1, out
