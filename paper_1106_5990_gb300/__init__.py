"""GB300-native algebraic-distance strength of connection (arXiv 1106.5990).

``amgd``   -- thin ctypes binding of the C-ABI library ``include/amgd.h``
              (hand-written sm_103a CUDA kernels); loads the in-tree build and
              raises if it is missing.
``inputs`` -- seeded synthetic input matrices and colorings.

Importing the package loads nothing; ``from paper_1106_5990_gb300 import amgd``
loads the CUDA library.
"""
