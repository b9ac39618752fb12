"""The product path has no CPU fallback: without the built library the
binding refuses to import, and without a CUDA device the first call that
needs device memory returns a CUDA error instead of computing on the host."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_binding_refuses_to_import_without_the_library():
    env = dict(os.environ, W5CT_LIB=os.path.join(ROOT, "no-such-dir", "libw5ct.so"))
    r = subprocess.run([sys.executable, "-c", "import paper_1812_04278_gb300.w5ct"], cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=120)
    assert r.returncode != 0
    assert "ImportError" in r.stderr and "missing" in r.stderr


def test_no_device_means_a_cuda_error():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    from paper_1812_04278_gb300 import build
    build.build()
    from paper_1812_04278_gb300 import w5ct
    ctx = w5ct.w5ct_create(w5ct.w5ct_config_default())
    try:
        with pytest.raises(w5ct.W5ctError) as e:
            w5ct.w5ct_init_grid(ctx, (8, 8, 8), (0.125, 0.125, 0.125))
        assert e.value.code == w5ct.W5CT_ERR_CUDA
    finally:
        w5ct.w5ct_destroy(ctx)
