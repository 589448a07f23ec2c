"""The Z-slab traversal of full-lattice launches gives the same results as
lexicographic order: the D / D^H / Dhat parity tests rerun in a fresh process
with slabs of depth 2 forced (DD_ZBLOCK=2), which the small test lattices
would otherwise not use."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_parity_with_z_slabs_of_two():
    env = dict(os.environ, DD_ZBLOCK="2")
    res = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "tests/test_gpu_parity.py", "-k",
                          "D_and_DH or Dhat or native_layout"], cwd=ROOT, env=env, capture_output=True, text=True,
                         timeout=600)
    assert res.returncode == 0, res.stdout[-2000:] + res.stderr[-2000:]


def test_parity_with_three_row_fp32_links():
    """The same parity tests with the FP32 links kept at three rows
    (DD_RECON=0), the path taken for links that are not SU(3)."""
    env = dict(os.environ, DD_RECON="0")
    res = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "tests/test_gpu_parity.py", "-k",
                          "D_and_DH or Dhat or native_layout"], cwd=ROOT, env=env, capture_output=True, text=True,
                         timeout=600)
    assert res.returncode == 0, res.stdout[-2000:] + res.stderr[-2000:]
