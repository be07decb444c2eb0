"""GB300-native (sm_103a) implementation of one predictor-corrector time step
of the GEA pressure-based finite-volume solver for the dry compressible Euler
equations (Girfoglio, Quaini & Rozza, arXiv 2303.10499, Section 3).

The compute path is a C-ABI CUDA library (include/gea.h); gea.py is its thin
ctypes binding. workloads.py produces the seeded synthetic initial states.
"""
