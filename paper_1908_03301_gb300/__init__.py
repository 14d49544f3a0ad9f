"""GB300-native Kirchhoff network solver (arXiv:1908.03301 hot path).

The CUDA library is loaded lazily by :mod:`paper_1908_03301_gb300.netsolve`;
importing the package itself loads nothing.
"""
