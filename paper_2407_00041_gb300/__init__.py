"""GB300 (sm_103a) Wilson-clover Dirac operator and FGMRES solver.

The compute path is ``libddwilson.so`` (hand-written CUDA, C ABI declared in
``include/dd_wilson.h``); this package is its thin Python binding.  Importing
it loads the library and fails loudly if it cannot be built or loaded.
"""
from .binding import *  # noqa: F401,F403
from .binding import load, Lattice, Gauge, Operator, SolveParams, Stats, DDError, Decomposition, Amg  # noqa: F401

lib = load()
from .autograd import dirac, su3_force, DiracApply  # noqa: E402,F401
