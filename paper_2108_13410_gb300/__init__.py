"""GB300-native engine for the Trotterised adiabatic evolution of the Z2 gauge-Higgs model.

The compute path is libqsim.so (hand-written sm_103a CUDA behind the C ABI of
include/qsim.h); qsim.py is its ctypes binding.  Importing the binding loads (or
builds, with nvcc) the library and fails loudly if that is impossible.
"""
from .qsim import (Simulator, QsError, library, library_path, qs_couplings,  # noqa: F401
                   QS_NORM, QS_PLAQUETTE, QS_WILSON, QS_X, QS_ENERGY, QS_ENERGY_S,
                   QS_GAUSS, QS_THOOFT, QS_OPT_METHOD, QS_OPT_RENORM_EVERY,
                   QS_OPT_PROFILE, QS_OPT_GRAPH, QS_OPT_XPASS, QS_OPT_TMA_BUFFERS)
