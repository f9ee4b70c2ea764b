"""GB300-native STG wall-modelled MRT-LES lattice Boltzmann channel step.

The compute path is the CUDA library liblbm_gb300.so behind the C ABI declared
in include/lbm.h; this package is its thin Python binding.  Importing the
package loads nothing: the library is opened on first use and the binding
raises if it is missing -- there is no CPU fallback.
"""
__all__ = ["LBMChannel", "STGAdjoint", "lib"]


def __getattr__(name):
    if name in ("LBMChannel", "STGAdjoint"):
        from . import channel
        return getattr(channel, name)
    if name == "lib":
        from . import _abi
        return _abi.lib()
    raise AttributeError(name)
