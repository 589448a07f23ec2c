"""Seeded synthetic inputs shared by the CPU oracle and the CUDA library.

Nothing here computes the Wilson-clover operator: it draws SU(3) gauge links
U = exp(i*eps*H) (H a traceless Hermitian Gaussian matrix) and Gaussian spinor
fields from a counter-based generator (SplitMix64 + Box-Muller, see
``synth.c``), so every site can be drawn on its own and both sides see the same
numbers.

Conventions (shared with the library's canonical layout):
  * ``dims = (nT, nZ, nY, nX)``; site index ``((t*nZ + z)*nY + y)*nX + x``.
  * links ``[V, 4, 3, 3]`` complex128, direction order T, Z, Y, X.
  * spinors ``[nrhs, V, 4, 3]`` complex128 (spin, colour), component 3*spin+colour.

Default seeds: gauge 20240700, right-hand side k uses 20240701 + k, the
adjoint's test field phi uses 20240800.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import tempfile

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "synth.c")
_LIB = os.path.join(_HERE, "libsynth.so")
_lib = None

SEED_GAUGE = 20240700
SEED_RHS = 20240701
SEED_PHI = 20240800


def build(force: bool = False) -> str:
    """Compile ``synth.c`` into ``libsynth.so`` next to it (gcc, OpenMP)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    fd, tmp = tempfile.mkstemp(suffix=".so", dir=_HERE)
    os.close(fd)
    cmd = ["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        i64, u64, dbl, ptr = ctypes.c_int64, ctypes.c_uint64, ctypes.c_double, ctypes.c_void_p
        lib.synth_links.argtypes = [u64, dbl, i64, i64, ctypes.c_int, ptr]
        lib.synth_gaussian.argtypes = [u64, i64, i64, ptr]
        lib.synth_spinor_sites.argtypes = [u64, i64, i64, ptr, i64, ptr]
        lib.synth_links_sites.argtypes = [u64, dbl, ptr, i64, ptr]
        for f in (lib.synth_links, lib.synth_gaussian, lib.synth_spinor_sites, lib.synth_links_sites):
            f.restype = None
        _lib = lib
    return _lib


def volume(dims) -> int:
    v = 1
    for d in dims:
        v *= int(d)
    return v


def gauge(dims, seed: int = SEED_GAUGE, eps: float = 0.3) -> np.ndarray:
    """All links of the lattice: complex128 ``[V, 4, 3, 3]``."""
    V = volume(dims)
    out = np.empty((V, 4, 3, 3), dtype=np.complex128)
    _load().synth_links(seed, eps, 0, V, 4, out.ctypes.data)
    return out


def gauge_sites(sites, seed: int = SEED_GAUGE, eps: float = 0.3) -> np.ndarray:
    """Links of the listed sites only: complex128 ``[len(sites), 4, 3, 3]``."""
    s = np.ascontiguousarray(sites, dtype=np.int64)
    out = np.empty((s.size, 4, 3, 3), dtype=np.complex128)
    _load().synth_links_sites(seed, eps, s.ctypes.data, s.size, out.ctypes.data)
    return out


def su3_field(dims, seed: int, eps: float = 1.0) -> np.ndarray:
    """One SU(3) matrix per site (e.g. a gauge transformation): ``[V, 3, 3]``."""
    V = volume(dims)
    out = np.empty((V, 3, 3), dtype=np.complex128)
    _load().synth_links(seed, eps, 0, V, 1, out.ctypes.data)
    return out


def spinor(dims, nrhs: int = 1, seed: int = SEED_RHS) -> np.ndarray:
    """Gaussian spinor fields ``[nrhs, V, 4, 3]``; field r draws from counters of index r."""
    V = volume(dims)
    out = np.empty((nrhs, V, 4, 3), dtype=np.complex128)
    _load().synth_gaussian(seed, 0, nrhs * V * 12, out.ctypes.data)
    return out


def spinor_sites(dims, sites, r: int = 0, seed: int = SEED_RHS) -> np.ndarray:
    """Field r of :func:`spinor` restricted to the listed sites: ``[len(sites), 4, 3]``."""
    V = volume(dims)
    s = np.ascontiguousarray(sites, dtype=np.int64)
    out = np.empty((s.size, 4, 3), dtype=np.complex128)
    _load().synth_spinor_sites(seed, V, r, s.ctypes.data, s.size, out.ctypes.data)
    return out


def gaussian(n: int, seed: int, counter0: int = 0) -> np.ndarray:
    """n complex Gaussian numbers (Re, Im i.i.d. N(0,1))."""
    out = np.empty(n, dtype=np.complex128)
    _load().synth_gaussian(seed, counter0, n, out.ctypes.data)
    return out
