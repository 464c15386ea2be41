"""GB300-native butterfly spherical harmonic transform (Tygert, "Fast
algorithms for spherical harmonic expansions, III").

The compute path is a C-ABI shared library (``include/sht.h``) with CUDA
kernels for sm_103a; ``paper_0910_5435_gb300.sht`` is the thin ctypes
binding over it.  Importing this package does not load the library; the
first use of ``paper_0910_5435_gb300.sht`` does, and fails loudly if it
has not been built.
"""
