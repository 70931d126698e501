"""GB300-native model-based iterative reconstruction for spectral-domain OCT.

The ISAM system operator, its adjoint and the FISTA solver run as hand-written
CUDA kernels for sm_103a behind a C-ABI library (``include/mbir.h``); the
Python layer in :mod:`paper_2108_01438_gb300.mbir` only marshals arguments.
Importing this package loads nothing: the library is opened on first use.
"""
__version__ = "0.1.0"
