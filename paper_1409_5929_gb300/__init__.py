"""GB300-native axisymmetric MRT lattice Boltzmann solver for thermal flow in
porous media (Liu, He & Li, arXiv 1409.5929).

The compute path is the CUDA library ``liblbm.so`` behind the C ABI declared in
``include/lbm.h``; :mod:`paper_1409_5929_gb300.lbm` is its thin ctypes binding.
Importing this package loads nothing; the binding loads the library on first use
and raises if it is missing (there is no CPU fallback).
"""
