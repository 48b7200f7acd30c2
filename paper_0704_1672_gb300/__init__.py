"""GB300-native two-center multipole (TCM) method for the Coulomb energy of two charge systems.

The compute path is hand-written CUDA for sm_103a behind a C ABI (``include/tcm.h``,
``libtcm.so``); :mod:`.tcm` is the thin Python binding.  Importing the package does
not load the library; the first call into :mod:`.tcm` does, and raises if it is
missing.
"""
__all__ = ["synth"]
