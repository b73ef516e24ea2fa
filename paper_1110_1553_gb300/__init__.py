"""GB300-native hierarchical tile Householder QR (HQR).

The numeric path lives in ``libhqr.so`` (C ABI declared in include/hqr.h);
``paper_1110_1553_gb300.hqr`` is its Python binding and
``paper_1110_1553_gb300.inputs`` the seeded synthetic input generators.
"""
from . import hqr  # noqa: F401
