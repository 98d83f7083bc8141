"""GB300 near-field direct-sum library (the near field of the Abacus N-body
method, Maksimova et al. 2021, Sec. 3.1).

The compute path is libnf (CUDA for sm_103a, C ABI in include/nf.h); this
package is its thin Python binding. Build the library with
``python -m paper_2110_11398_gb300.build``.
"""
from ._native import EXPORTS, NFError, PRECISIONS, load  # noqa: F401
from .nearfield import NearField, accel  # noqa: F401

__all__ = ["NearField", "accel", "NFError", "load", "EXPORTS", "PRECISIONS"]
