"""GB300-native Sinkhorn solver for dynamic multi-commodity network flow by graph-structured
multi-marginal optimal transport (Haasler, Ringh, Chen, Karlsson, arXiv 2106.14485).

``ots`` is the Python binding of the C ABI (``include/ots.h``), ``instances`` builds seeded
synthetic problems, ``build`` compiles ``libots.so`` for sm_103a.
"""
from . import instances  # noqa: F401

__all__ = ["instances", "ots", "build"]
