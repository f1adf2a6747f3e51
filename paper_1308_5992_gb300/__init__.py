"""GB300-native bootstrap AMG solver for the odd-even reduced 2D Wilson-Dirac
system (Brannick & Kahl).  The compute path is the CUDA library
libwilson_amg.so (C ABI: include/wilson_amg.h); wilson_amg is its binding."""
from . import wilson_amg  # noqa: F401

__all__ = ["wilson_amg"]
