"""All-edge spanning centrality (TGT / TGT+) on one GB300 GPU.

The computation lives in libsc.so (CUDA C++ for sm_103a) behind the C ABI of
include/sc.h; ``binding`` is its thin ctypes binding. Build with
``paper_2305_16086_gb300.build.build()``.
"""
from .binding import Graph, ScError, load  # noqa: F401

__all__ = ["Graph", "ScError", "load"]
