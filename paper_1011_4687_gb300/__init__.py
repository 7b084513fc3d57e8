"""GB300-native environment electrostatic potential for QM/MM quantum Monte Carlo.

The hot path of the FMO-QMC calculation in "Acceleration of a QM/MM-QMC
simulation using GPU" (Sec. II.B, Eq. ElectrostaticField): the potential of
fixed environment charges at every electron position of every walker, at
every Monte Carlo step.  The compute runs in the CUDA library built from
csrc/ (C ABI in include/esp.h); `esp` is its Python binding.

Importing the package loads nothing; `esp.load()` loads the compiled library
and raises if it is missing.
"""
__all__ = ["esp", "build_lib"]
