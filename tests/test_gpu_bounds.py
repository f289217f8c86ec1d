"""Bounds-checked build: the streaming kernels compiled with every global
store tested against its buffer (DWT_BOUNDS_CHECK); every scheme, wavelet,
storage type, fusion depth and direction at many shapes must record no
out-of-range store.  The checked library is built next to the product one and
loaded in a process of its own (DWT2D_LIBRARY)."""
import os
import subprocess
import sys

import pytest
import torch

from paper_1705_08266_gb300 import build as B

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_no_store_out_of_bounds():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    lib = B.build_bounds_checked()
    env = dict(os.environ, DWT2D_LIBRARY=lib, PYTHONPATH=ROOT)
    r = subprocess.run([sys.executable, "-m", "tests.bounds_run"], cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=1200)
    assert r.returncode == 0 and r.stdout.strip().splitlines()[-1].startswith("ok"), \
        r.stdout[-3000:] + r.stderr[-3000:]
