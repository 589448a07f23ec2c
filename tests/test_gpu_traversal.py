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


def test_parity_with_three_row_links():
    """The same parity tests and the reduced-precision solves with the FP32
    and FP16 links kept at three rows (DD_RECON=0), the path taken for links
    that are not SU(3)."""
    env = dict(os.environ, DD_RECON="0")
    for args in (["tests/test_gpu_parity.py", "-k", "D_and_DH or Dhat or native_layout"],
                 ["tests/test_gpu_solver.py", "-k", "solve_to_1e10 or fused"]):
        res = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", *args], cwd=ROOT, env=env,
                             capture_output=True, text=True, timeout=600)
        assert res.returncode == 0, res.stdout[-2000:] + res.stderr[-2000:]


def test_parity_and_solve_with_eight_real_fp32_links():
    """The parity tests and the FP32-inner solves with the eight-real FP32
    links made at gauge creation (DD_RECON=8)."""
    env = dict(os.environ, DD_RECON="8")
    for args in (["tests/test_gpu_parity.py", "-k", "D_and_DH or Dhat or native_layout"],
                 ["tests/test_gpu_solver.py", "-k", "solve_to_1e10 or multi_rhs or fused"]):
        res = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", *args], cwd=ROOT, env=env,
                             capture_output=True, text=True, timeout=600)
        assert res.returncode == 0, res.stdout[-2000:] + res.stderr[-2000:]
