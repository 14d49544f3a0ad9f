"""FP64 CPU oracle for the Kirchhoff network solve (test infrastructure only).

Only the test suite, the package smoke check and the benchmark's CPU-baseline
and reference legs may import this package.  The CUDA solver never does.
"""
from .oracle import (  # noqa: F401
    CLS_FACE_IN, CLS_FACE_OUT, CLS_INLET, CLS_ISOLATED, CLS_OUTLET, CLS_SPANNING,
    backbone, backbone_blocks, build, close_smallest, fbm_bonds, fbm_field, labels, max_threads, residual, solve,
)
