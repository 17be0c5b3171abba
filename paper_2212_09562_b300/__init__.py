"""B300-native RecSplit construction (rotation fitting) behind a C-ABI library.

The CUDA library is loaded lazily by :mod:`paper_2212_09562_b300.mphf`; importing
the package itself loads nothing.
"""
