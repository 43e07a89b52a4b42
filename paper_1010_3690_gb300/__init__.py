"""GB300-native CT-AUX submatrix-update hot path (sm_103a CUDA behind a C ABI).

The computation lives in the CUDA library _ctaux.so (sources in csrc/, ABI in
include/ctaux.h); `ctaux` is the ctypes binding.  The binding is imported on
first use of a name below (so that `paper_1010_3690_gb300.build` can run before
the library exists); using it without the library raises ImportError: there
is no other code path.
"""
_EXPORTS = ("CTAUX_FP64", "CTAUX_MIXED", "Context", "CtauxError", "ctaux_philox_uniforms", "lib")


def __getattr__(name):
    if name in _EXPORTS:
        from . import ctaux
        return getattr(ctaux, name)
    raise AttributeError(name)
